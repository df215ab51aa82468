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


def loglik_bound(ll, tol=TOL_LOGLIK):
    """Ceiling on the deviation of a log-likelihood (or of a log weight built
    from one): the stated parity tolerance tol (1 + |ll|), a fixed bound that
    does not depend on the deviation observed."""
    with np.errstate(invalid="ignore"):
        return tol * (1.0 + np.abs(ll))


def _loglik_rows(cfg, y, X):
    """log pi(y | x) of every row of X (only its magnitude is used: it sizes
    the tolerance of the log weights built from it)."""
    m = cfg.m
    obs = [cfg.obs_idx[i] for i in range(m)]
    y = np.asarray(y, dtype=np.float64)
    sig = np.array([cfg.sigma[i] for i in range(m)], dtype=np.float64)
    if cfg.noise == oracle.NOISE_RELATIVE:
        sig = sig * np.maximum(np.abs(y), 1e-300)
    with np.errstate(invalid="ignore", over="ignore"):
        r = (y[None, :] - np.asarray(X)[:, obs]) / sig[None, :]
        return -0.5 * np.sum(r * r, axis=1)


def check_epoch(g, o, t, y, tol_state=TOL_STATE, exempt_dead=False):
    """One epoch of the library filter g (pf_assimilate) and of the oracle o
    from g's committed state, compared stage by stage (finish_epoch)."""
    pre = begin_epoch(g, o)
    g.pf_assimilate(t, y)
    return finish_epoch(g, o, t, y, pre, tol_state=tol_state, exempt_dead=exempt_dead)


def begin_epoch(g, o):
    """Start the oracle o from the library filter g's committed state; call
    before the library runs the epoch (alone, batched or served)."""
    sync_oracle_from_gpu(g, o)
    tb_prev, C_prev, _ = g.pf_estimates()   # the shift of the one-pass covariance
    return dict(tb_prev=tb_prev, C_prev=C_prev)


def finish_epoch(g, o, t, y, pre, tol_state=TOL_STATE, exempt_dead=False, stats=True):
    """After the library's epoch (begin_epoch before it): the oracle's epoch
    from the same committed state, every intermediate result compared;
    returns a dict of the observed maximum deviations and the tolerances.

    stats: also compare pf_stats (the distinct parents and the ESS); a
    server session's borrowed filter serves only the read-only calls, so its
    check passes stats=False.

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
    tb_prev, C_prev = pre["tb_prev"], pre["C_prev"]
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
    b1 = loglik_bound(ow["ll1"])
    fin1 = np.isfinite(ow["lg"]) & (live1 if live1 is not None else True)
    assert o.cumulative() == oracle.OK
    ow = o.work()
    c_gpu, c_or = gw["c"], ow["c"]
    assert np.all(np.diff(c_gpu) >= 0.0), "cumulative weights not monotone"
    # Step 3a's weights inherit those deviations: g_k = exp(lg_k - M) moves
    # by at most g_k (b1_k + b1 of the maximum), to first order, so c_k by the
    # cumulative sum of that (with a factor 2 for the second-order terms)
    dlg = max_log_dev(gw["lg"], ow["lg"], live1)
    g_or = np.exp(np.where(fin1, ow["lg"] - np.max(ow["lg"][fin1]), -np.inf))
    bM = b1[np.argmax(np.where(fin1, ow["lg"], -np.inf))]
    tol_ck = 2.0 * np.cumsum(np.where(fin1, g_or * (b1 + bM), 0.0)) + TOL_CUM * c_or
    assert np.all(np.abs(c_gpu - c_or) <= tol_ck + TOL_CUM * c_or[-1])
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
    # Step 5's log weights: lw = log pi(y | x) - ll1[l], then normalised.
    # Each raw ratio deviates by at most b2_n + b1_{l_n} (the log-likelihood
    # tolerance at both ends), and the normalisation constant by at most
    # their weighted mean; every tolerance below follows from these ceilings
    # by first-order propagation, from the oracle's values alone.
    wo = np.exp(os_["lw"])
    wg = np.exp(gs["lw"])
    b2 = loglik_bound(_loglik_rows(o.cfg, y, os_["x"]))
    bl = b2 + b1[idx]
    usew = live & (wo > 0.0) & np.isfinite(bl)
    bl = np.where(usew, bl, 0.0)
    bL = float(np.sum(wo * bl))
    B = bl + bL                                    # per-particle ceiling
    dlw = max_log_dev(gs["lw"], os_["lw"], live if exempt_dead else None)
    devw = np.abs(gs["lw"] - os_["lw"])
    assert np.all(devw[usew] <= B[usew] + 1e-13 * (1.0 + np.abs(os_["lw"][usew]))), \
        float(np.max((devw - B)[usew]))
    assert close_loglik(gs["lw"], os_["lw"], live=live if exempt_dead else None), "log weights differ"
    # w_n = exp(lw_n) moves by at most w_n (e^B_n - 1)
    dW = wo * np.expm1(np.minimum(B, 1.0))
    errs["w"] = float(np.max(np.abs(wg - wo)) / np.max(wo))
    assert errs["w"] <= 1.01 * float(np.max(dW)) / np.max(wo) + 1e-13, errs["w"]
    tb, Cm, xb = g.pf_estimates()
    om = o.moments()
    def rel(a, b):
        return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
    # a weighted mean moves, to first order, by sum_n dW_n |v_n - vbar| (the
    # normalised weights' changes sum to zero), plus for x the states' own
    # deviation sum_n w_n tol_state ||x_n||; factor 2 for the second order
    php = np.where(usew[:, None], os_["phi"], 0.0)
    xp = np.where(usew[:, None], os_["x"], 0.0)
    errs["phibar"] = rel(tb, om["phibar"])
    # and by sum_n w_n |dphi_n|, each particle's phi being within the bound
    # asserted above: 1e-12 relative, or the Cholesky floor
    bphi = np.maximum(1e-12 * np.max(np.abs(os_["phi"]), axis=1), chol_floor)
    wphi = float(np.sum(np.where(usew, wo * bphi, 0.0)))
    dpb = 2.0 * np.sum(dW[:, None] * np.abs(php - om["phibar"]), axis=0) + 2.0 * wphi
    tol_pb = max(1e-12, float(np.max(dpb)) / max(np.max(np.abs(om["phibar"])), 1e-300))
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
    Cden = max(np.max(np.abs(om["C"])), shift2, 1e-280)
    errs["C"] = max(dC - eps_phi2, 0.0) / Cden
    dev_phi = np.max(np.abs(php - om["phibar"]), axis=1)
    dCw = 2.0 * float(np.sum(dW * dev_phi ** 2)) + 4.0 * float(np.sum(np.where(usew, wo * bphi * dev_phi, 0.0)))
    tol_C = max(1e-8, dCw / Cden)
    errs["xbar"] = rel(xb, om["xbar"])
    dxb = 2.0 * (np.sum(dW[:, None] * np.abs(xp - om["xbar"]), axis=0)
                 + tol_state * float(np.sum(wo[usew] * np.max(np.abs(os_["x"][usew]), axis=1))))
    tol_xb = max(1e-10, float(np.max(dxb)) / max(np.max(np.abs(om["xbar"])), 1e-300))
    assert errs["phibar"] <= tol_pb and errs["C"] <= tol_C and errs["xbar"] <= tol_xb, \
        (errs, tol_pb, tol_C, tol_xb)
    # ESS = 1 / sum w^2 moves by at most 2 sum w_n dW_n / sum w^2, relative
    tol_ess = max(1e-9, 2.0 * float(np.sum(wo * dW)) / float(np.sum(wo * wo)))
    if stats:
        st = g.pf_stats()
        assert st["unique_parents"] == len(np.unique(gw["idx"]))
        assert abs(st["ess"] - om["ess"]) <= tol_ess * om["ess"]
    errs["tol"] = dict(pb=tol_pb, C=tol_C, xbar=tol_xb, ess=tol_ess, lw=bL, w=float(np.max(dW)) / float(np.max(wo)))
    errs["same_indices_from_own_scan"] = same_own
    errs["dlg"], errs["dlw"] = dlg, dlw
    return errs


def _posterior_runs(make, seeds, gpu, pf=None):
    """Whole runs, one per filter seed (the data stay fixed): the final
    posterior mean and the diagonal of C of each."""
    pb, dc = [], []
    for seed in seeds:
        w = make(seed)
        if gpu:
            g = pf.Filter.from_workload(w)
            for k in range(w.T):
                g.pf_assimilate(w.t_obs[k], w.y_obs[k])
            tb, Cm, _ = g.pf_estimates()
            g.close()
        else:
            o = oracle.Filter(w)
            o.init()
            for k in range(w.T):
                assert o.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
            m = o.moments()
            tb, Cm = m["phibar"], m["C"]
        pb.append(tb)
        dc.append(np.diag(Cm))
    return np.array(pb), np.array(dc)


def assert_within_three_mc_se(pf, make, R=16):
    """The GPU over filter seeds 0..R-1 and the oracle over the disjoint seeds
    1000..1000+R-1: the means over runs of the posterior mean and of diag C
    differ by at most 3 Monte Carlo standard errors of that difference.  The
    two sides never share a random stream, so this is a statistical check of
    the posterior, not a repeat of the same-seed agreement."""
    g_pb, g_dc = _posterior_runs(make, range(R), True, pf)
    o_pb, o_dc = _posterior_runs(make, range(1000, 1000 + R), False)
    for a, b in ((g_pb, o_pb), (g_dc, o_dc)):
        se = np.sqrt(a.var(axis=0, ddof=1) / R + b.var(axis=0, ddof=1) / R)
        assert np.all(np.abs(a.mean(axis=0) - b.mean(axis=0)) <= 3.0 * se), \
            (a.mean(axis=0), b.mean(axis=0), se)
