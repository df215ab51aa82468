"""Helpers shared by the GPU parity tests: run one epoch of Algorithm 1 on the
CUDA library and on the CPU oracle from the same committed state and compare
every intermediate result."""
import numpy as np

import oracle

# tolerances (spec parity bar): one FP64 propagation epoch agrees to
# 1e-10 relative per particle; resampling indices are bit-exact given the same
# cumulative weights.
TOL_STATE = 1e-10
TOL_LOGLIK = 1e-9
TOL_CUM = 1e-12


def sync_oracle_from_gpu(g, o):
    st = g.pf_get_ensemble()
    o.set_state(**st)
    tb, Cm, _ = g.pf_estimates()
    o.set_moments(tb, Cm)
    h = g.pf_get_history()
    o.set_history(h["epoch"], h["depth"], h["t_prev"], h["hprev1"], h["hprev2"])
    return st


def rel_state_err(a, b):
    """max over particles of ||a_n - b_n||_inf / ||b_n||_inf"""
    scale = np.maximum(np.max(np.abs(b), axis=1), 1e-300)
    return float(np.max(np.max(np.abs(a - b), axis=1) / scale))


def close_loglik(a, b, tol=TOL_LOGLIK):
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    return bool(np.all(np.abs(a[fin] - b[fin]) <= tol * (1.0 + np.abs(b[fin]))))


def check_epoch(g, o, t, y, tol_state=TOL_STATE):
    """One epoch on both sides from the GPU's committed state; returns a dict
    of the observed maximum deviations."""
    sync_oracle_from_gpu(g, o)
    g.pf_assimilate(t, y)
    gw = g.pf_get_work()
    tab, S = o.substeps(t)
    assert o.stage1(tab, S, y) == oracle.OK
    ow = o.work()
    assert close_loglik(gw["ll1"], ow["ll1"]), "stage 1 log-likelihoods differ"
    assert close_loglik(gw["lg"], ow["lg"]), "first-stage log weights differ"
    assert o.cumulative() == oracle.OK
    ow = o.work()
    c_gpu, c_or = gw["c"], ow["c"]
    assert np.all(np.diff(c_gpu) >= 0.0), "cumulative weights not monotone"
    assert np.allclose(c_gpu, c_or, rtol=TOL_CUM, atol=TOL_CUM * c_or[-1])
    u = o.resample_u()
    idx = oracle.resample_systematic(c_gpu, u)
    assert np.array_equal(idx, gw["idx"]), "resampling indices differ"
    # the oracle's own cumulative sums give the same indices here
    same_own = np.array_equal(oracle.resample_systematic(c_or, u), gw["idx"])
    assert o.stage2(tab, S, y, idx) == oracle.OK
    assert o.commit(t) == oracle.OK
    gs, os_ = g.pf_get_ensemble(), o.state()
    errs = {}
    for key in ("x", "h1", "h2"):
        errs[key] = rel_state_err(gs[key], os_[key])
        assert errs[key] <= tol_state, (key, errs[key])
    errs["phi"] = rel_state_err(gs["phi"], os_["phi"])
    assert errs["phi"] <= 1e-12
    wg, wo = np.exp(gs["lw"]), np.exp(os_["lw"])
    errs["w"] = float(np.max(np.abs(wg - wo)) / np.max(wo))
    assert errs["w"] <= 1e-9
    tb, Cm, xb = g.pf_estimates()
    om = o.moments()
    def rel(a, b):
        return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
    errs["phibar"] = rel(tb, om["phibar"])
    # C is a difference of second moments: compare on the scale of the
    # parameter spread, which is zero for a single particle
    errs["C"] = float(np.max(np.abs(Cm - om["C"]))) / max(np.max(np.abs(om["C"])), 1e-280)
    errs["xbar"] = rel(xb, om["xbar"])
    assert errs["phibar"] <= 1e-12 and errs["C"] <= 1e-8 and errs["xbar"] <= 1e-10, errs
    stats = g.pf_stats()
    assert stats["unique_parents"] == len(np.unique(gw["idx"]))
    assert abs(stats["ess"] - om["ess"]) <= 1e-9 * om["ess"]
    errs["same_indices_from_own_scan"] = same_own
    return errs
