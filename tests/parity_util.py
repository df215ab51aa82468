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


def max_log_dev(a, b, live=None):
    """largest |a - b| over the entries finite on both sides (the log weights
    must be finite on the same entries, which close_loglik checks), and live
    when a mask is given"""
    fin = np.isfinite(a) & np.isfinite(b)
    if live is not None:
        fin = fin & live
    return float(np.max(np.abs(a[fin] - b[fin]))) if fin.any() else 0.0


def cumulative_reference(lg):
    """Step 3a's cumulative weights from given log weights, summed in order."""
    fin = np.isfinite(lg)
    if not fin.any():
        return np.zeros_like(lg)
    e = np.where(fin, np.exp(np.where(fin, lg, 0.0) - np.max(lg[fin])), 0.0)
    return np.cumsum(e)


def close_loglik(a, b, tol=TOL_LOGLIK, live=None):
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    if live is not None:
        fin = fin & live
    return bool(np.all(np.abs(a[fin] - b[fin]) <= tol * (1.0 + np.abs(b[fin]))))


def dead_mask(lw):
    """Entries whose weight exp(lw - max lw) underflows to exactly zero."""
    fin = np.isfinite(lw)
    top = np.max(lw[fin]) if fin.any() else 0.0
    return ~fin | (lw - top < -700.0)


def check_epoch(g, o, t, y, tol_state=TOL_STATE, exempt_dead=False):
    """One epoch on both sides from the GPU's committed state; returns a dict
    of the observed maximum deviations.

    exempt_dead: a particle whose weight underflows to zero on both sides
    (log weight more than 700 below the largest, so exp(lw - max) is exactly
    0 in FP64) is exempt from the per-particle bounds on its log-likelihood
    and state; which particles are dead must agree exactly.  Such a particle
    had an ill-conditioned propagation that amplifies rounding without bound
    -- an explicit step on a stiff parameter (unstable), or a Newton iteration
    of the Michaelis-Menten system thrown toward the pole of its flux by an
    extreme parameter -- and it has no effect on any output: it adds nothing
    to the cumulative weights, is never resampled and has zero weight in
    every moment."""
    sync_oracle_from_gpu(g, o)
    tb_prev, C_prev, _ = g.pf_estimates()   # the shift of the one-pass covariance
    g.pf_assimilate(t, y)
    gw = g.pf_get_work()
    tab, S = o.substeps(t)
    assert o.stage1(tab, S, y) == oracle.OK
    ow = o.work()
    live1 = None
    if exempt_dead:
        assert np.array_equal(dead_mask(gw["lg"]), dead_mask(ow["lg"])), "zero first-stage weights differ"
        live1 = ~dead_mask(ow["lg"])
    assert close_loglik(gw["ll1"], ow["ll1"], live=live1), "stage 1 log-likelihoods differ"
    assert close_loglik(gw["lg"], ow["lg"], live=live1), "first-stage log weights differ"
    assert o.cumulative() == oracle.OK
    ow = o.work()
    c_gpu, c_or = gw["c"], ow["c"]
    assert np.all(np.diff(c_gpu) >= 0.0), "cumulative weights not monotone"
    # Step 3a's weights inherit the propagated state's rounding through
    # log pi(y | xbar): each term exp(lg - max lg) moves by at most twice the
    # largest log-weight deviation, so the two sides' sums agree to that
    dlg = max_log_dev(gw["lg"], ow["lg"], live1)
    tol_c = max(TOL_CUM, 4.0 * dlg)
    assert np.allclose(c_gpu, c_or, rtol=tol_c, atol=tol_c * c_or[-1])
    # the scan itself, from the GPU's own log weights, to the scan's rounding
    c_ref = cumulative_reference(gw["lg"])
    assert np.allclose(c_gpu, c_ref, rtol=TOL_CUM, atol=TOL_CUM * c_ref[-1])
    u = o.resample_u()
    idx = oracle.resample_systematic(c_gpu, u)
    assert np.array_equal(idx, gw["idx"]), "resampling indices differ"
    # the oracle's own cumulative sums give the same indices here
    same_own = np.array_equal(oracle.resample_systematic(c_or, u), gw["idx"])
    assert o.stage2(tab, S, y, idx) == oracle.OK
    assert o.commit(t) == oracle.OK
    gs, os_ = g.pf_get_ensemble(), o.state()
    errs = {}
    live = np.ones(len(os_["lw"]), dtype=bool)
    if exempt_dead:
        dg, do = dead_mask(gs["lw"]), dead_mask(os_["lw"])
        assert np.array_equal(dg, do), "zero-weight particles differ"
        live = ~do
        errs["dead"] = int(np.sum(do))
    for key in ("x", "h1", "h2"):
        errs[key] = rel_state_err(gs[key][live], os_[key][live]) if live.any() else 0.0
        assert errs[key] <= tol_state, (key, errs[key])
    errs["phi"] = rel_state_err(gs["phi"], os_["phi"])
    # Step 4a uses chol(C): for a (near-)singular C -- weights collapsed onto a
    # few particles -- the factor's trailing pivots are rounding residues, and
    # two correct factorisations of the same C may differ by up to
    # sqrt(p eps |C|) in those columns (the backward error of Cholesky), which
    # proliferation scales by s |z|
    a = o.cfg.a
    s = np.sqrt(max(1.0 - a * a, 0.0))
    p = len(tb_prev)
    chol_floor = 8.0 * s * np.sqrt(p * np.finfo(float).eps * max(float(np.max(np.abs(C_prev))), 0.0))
    dphi = float(np.max(np.abs(gs["phi"] - os_["phi"])))
    assert errs["phi"] <= 1e-12 or dphi <= chol_floor, (errs["phi"], dphi, chol_floor)
    # Step 5's weights carry the state's rounding the same way (log pi(y | x))
    dlw = max_log_dev(gs["lw"], os_["lw"], live if exempt_dead else None)
    wg, wo = np.exp(gs["lw"]), np.exp(os_["lw"])
    errs["w"] = float(np.max(np.abs(wg - wo)) / np.max(wo))
    assert errs["w"] <= max(1e-9, 4.0 * dlw)
    tb, Cm, xb = g.pf_estimates()
    om = o.moments()
    def rel(a, b):
        return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
    # normalised weights move by at most ~2 dlw relative, so a weighted mean
    # moves by at most ~4 dlw times the spread of what is averaged
    def spread(v):
        return float(np.max(np.abs(v - np.mean(v, axis=0)))) if len(v) else 0.0
    errs["phibar"] = rel(tb, om["phibar"])
    tol_pb = max(1e-12, 4.0 * dlw * spread(os_["phi"][live]) / max(np.max(np.abs(om["phibar"])), 1e-300))
    # C is a difference of second moments about the previous mean (the
    # kernel's shift): its rounding is relative to the larger of C and the
    # squared distance the mean moved, which dominates when the weights
    # collapse onto a few particles (C -> 0)
    # (and, when the ensemble has collapsed onto clones of one particle, C is
    # itself rounding: the differences phi - shift carry eps |phi| each, so C
    # carries (eps |phi|)^2 from their products)
    shift2 = float(np.max((tb - tb_prev) ** 2)) if len(tb) else 0.0
    eps_phi2 = 64.0 * (np.finfo(float).eps * max(float(np.max(np.abs(os_["phi"]))), 1e-300)) ** 2
    dC = float(np.max(np.abs(Cm - om["C"])))
    errs["C"] = max(dC - eps_phi2, 0.0) / max(np.max(np.abs(om["C"])), shift2, 1e-280)
    errs["xbar"] = rel(xb, om["xbar"])
    tol_xb = max(1e-10, 4.0 * dlw * spread(os_["x"][live]) / max(np.max(np.abs(om["xbar"])), 1e-300))
    tol_C = max(1e-8, 8.0 * dlw)
    assert errs["phibar"] <= tol_pb and errs["C"] <= tol_C and errs["xbar"] <= tol_xb, errs
    stats = g.pf_stats()
    assert stats["unique_parents"] == len(np.unique(gw["idx"]))
    assert abs(stats["ess"] - om["ess"]) <= max(1e-9, 8.0 * dlw) * om["ess"]
    errs["same_indices_from_own_scan"] = same_own
    errs["dlg"], errs["dlw"] = dlg, dlw
    return errs
