"""Pins of the oracle's Algorithm 1 steps as composed in one epoch.

The building blocks (random numbers, LMM steps, Newton, Cholesky, the
systematic search) are pinned in test_oracle_pins.py.  Here each step of the
epoch that the oracle composes from them is recomputed by hand, in NumPy,
from the same stored inputs and the same draws, on tiny ensembles with
deliberately unequal particles -- distinct first-stage log-likelihoods, a
non-identity parent map with repeats, a correlated C, a shrinkage a far from
1 and a kappa far from 1 -- so that a slip in the composition (the parent's
ll1 replaced by the child's, s^2 in place of s, L applied as an upper factor,
kappa outside the square root, a history left untranslated, the 1/2 of the
log-likelihood dropped, |x| in place of |y| in the relative noise) fails:

* Step 3a / Step 5 log pi(y | x): against -1/2 sum ((y_i - x_{o_i}) / s_i)^2
  with s_i = sigma_i (additive) or sigma_i |y_i| (relative, reading 8);
* Step 2 and 3a: log g = log w + log pi(y | Psi(x, theta(shrink(phi))));
* Step 3a's cumulative weights: c = cumsum(exp(lg - max lg));
* Steps 3c-5: phi = shrink(phi^l) + sqrt(1 - a^2) L z with L L^T = C,
  x = Psi(x^l) + sqrt(kappa E) z', history translated by the same v,
  log w = log pi(y | x) - ll1[l];
* Step 5 normalisation and Step 6 moments with unequal weights: against
  np.average and np.cov(aweights=w, bias=True);
* Step 4a as a whole (the proliferation pin): after shrinkage and
  the kernel draw the ensemble covariance is a^2 C + s^2 C = C, within Monte
  Carlo standard errors.
"""
import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import workloads as W


def _np_loglik(w, y, x):
    """Gaussian log-likelihood without its constants (reading 8)."""
    s = 0.0
    for i, o in enumerate(w.obs_idx):
        sig = w.sigma[i] * (max(abs(y[i]), 1e-300) if w.noise == W.NOISE_RELATIVE else 1.0)
        s += ((y[i] - x[o]) / sig) ** 2
    return -0.5 * s


# ------------------------------------------------------------ log-likelihood
@pytest.mark.parametrize("noise", [W.NOISE_ADDITIVE, W.NOISE_RELATIVE])
def test_loglik_against_numpy(oracle_lib, noise):
    rng = np.random.default_rng(40 + noise)
    w = W.robertson(N=4, T=2).with_(noise=noise, obs_idx=[2, 0], sigma=[0.03, 0.2])
    cfg = oracle.make_config(w)
    for _ in range(20):
        x = rng.normal(size=3) * 2.0
        y = rng.normal(size=2) * 3.0
        ref = _np_loglik(w, y, x)
        got = oracle.loglik(cfg, y, x)
        assert got == pytest.approx(ref, rel=1e-14, abs=0)
        # an independent closed form of the same quantity
        sig = np.array(w.sigma) * (np.abs(y) if noise == W.NOISE_RELATIVE else 1.0)
        closed = -0.5 * float(np.sum(((y - x[[2, 0]]) / sig) ** 2))
        assert got == pytest.approx(closed, rel=1e-13)
    # at the data the likelihood is maximal (zero), for both models
    x = np.array([1.5, -0.2, 0.7])
    assert oracle.loglik(cfg, [0.7, 1.5], x) == 0.0


# ----------------------------------------------------- a staged tiny epoch
def _tiny_state(w, n_epochs, rng):
    """A realistic committed state after a few real epochs of the oracle,
    then unequal log weights and a correlated C chosen by the test."""
    f = oracle.Filter(w)
    f.init()
    for k in range(n_epochs):
        assert f.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
    st = f.state()
    lw = rng.normal(size=w.N) * 0.8
    lw -= np.log(np.sum(np.exp(lw)))
    st["lw"] = lw
    # distinct histories, so a missing translation or a wrong slot shows
    st["h1"] = st["h1"] * (1.0 + 1e-3 * rng.normal(size=st["h1"].shape))
    st["h2"] = st["h2"] * (1.0 + 1e-3 * rng.normal(size=st["h2"].shape))
    f.set_state(**st)
    p = w.p
    B = rng.normal(size=(p, p)) * 0.05
    Cm = B @ B.T + 0.002 * np.eye(p)
    pb = np.mean(st["phi"], axis=0) + 0.01 * rng.normal(size=p)
    f.set_moments(pb, Cm)
    return f, st, pb, Cm


CASES = [
    ("linear2", dict(a=0.6, kappa=2.5), 2),
    ("robertson", dict(a=0.55, kappa=4.0), 3),
]


@pytest.mark.parametrize("name,over,k", CASES)
def test_stage1_and_scan_by_hand(oracle_lib, name, over, k):
    rng = np.random.default_rng(7)
    w = W.get(name, N=5, T=k + 1).with_(**over)
    f, st, pb, Cm = _tiny_state(w, k, rng)
    t, y = w.t_obs[k], w.y_obs[k]
    tab, S = f.substeps(t)
    assert f.stage1(tab, S, y) == oracle.OK
    wk = f.work()
    a = w.a
    for n in range(w.N):
        shr = a * st["phi"][n] + (1.0 - a) * pb
        xp, _, _, _ = oracle.propagate(w.ode, w.newton_iters, np.exp(shr), tab, S,
                                       st["x"][n], st["h1"][n], st["h2"][n])
        ll = _np_loglik(w, y, xp)
        assert wk["ll1"][n] == pytest.approx(ll, rel=1e-9, abs=1e-9)
        assert wk["lg"][n] == pytest.approx(st["lw"][n] + ll, rel=1e-9, abs=1e-9)
    assert len(set(np.round(wk["ll1"], 6))) == w.N   # distinct, so slot slips show
    assert f.cumulative() == oracle.OK
    c = f.work()["c"]
    lg = wk["lg"]
    assert np.allclose(c, np.cumsum(np.exp(lg - lg.max())), rtol=1e-13, atol=0)
    assert c[-1] >= 1.0


@pytest.mark.parametrize("name,over,k", CASES)
def test_stage2_by_hand(oracle_lib, name, over, k):
    """Steps 3c-5 recomputed from the stored draws for every slot."""
    rng = np.random.default_rng(11)
    w = W.get(name, N=5, T=k + 1).with_(**over)
    f, st, pb, Cm = _tiny_state(w, k, rng)
    t, y = w.t_obs[k], w.y_obs[k]
    epoch = f.history()["epoch"]
    tab, S = f.substeps(t)
    assert f.stage1(tab, S, y) == oracle.OK
    ll1 = f.work()["ll1"].copy()
    idx = np.array([3, 3, 0, 4, 1], dtype=np.int32)      # repeats, not the identity
    assert f.stage2(tab, S, y, idx) == oracle.OK
    assert f.commit(t) == oracle.OK
    new = f.state()
    a, kappa = w.a, w.kappa
    s = np.sqrt(1.0 - a * a)
    L = np.linalg.cholesky(Cm)
    raw = np.zeros(w.N)
    for n in range(w.N):
        l = idx[n]
        z = np.array([oracle.normal(w.seed, w.stream, oracle.RNG_THETA, n, epoch, i) for i in range(w.p)])
        phi = a * st["phi"][l] + (1.0 - a) * pb + s * (L @ z)
        assert np.allclose(new["phi"][n], phi, rtol=1e-13, atol=1e-14), n
        x, h1, h2, E = oracle.propagate(w.ode, w.newton_iters, np.exp(phi), tab, S,
                                        st["x"][l], st["h1"][l], st["h2"][l], with_error=True)
        zi = np.array([oracle.normal(w.seed, w.stream, oracle.RNG_INNOV, n, epoch, i) for i in range(w.d)])
        v = np.sqrt(kappa * E) * zi
        # the innovation is resolvable in every component
        assert np.all(np.abs(v) > 1e-12 * np.abs(x))
        scale = np.max(np.abs(x))
        for key, ref in (("x", x + v), ("h1", h1 + v), ("h2", h2 + v)):
            assert np.max(np.abs(new[key][n] - ref)) <= 1e-12 * scale, (key, n)
        # the innovation itself, to its own relative accuracy
        assert np.allclose(new["x"][n] - x, v, rtol=1e-6, atol=1e-13 * np.abs(x) + 1e-300)
        raw[n] = _np_loglik(w, y, x + v) - ll1[l]
    # committed log weights are the raw Step 5 ratios, normalised (Step 5)
    ref = raw - (raw.max() + np.log(np.sum(np.exp(raw - raw.max()))))
    assert np.allclose(new["lw"], ref, rtol=1e-9, atol=1e-9)
    assert np.sum(np.exp(new["lw"])) == pytest.approx(1.0, rel=1e-14)


def test_commit_moments_with_unequal_weights(oracle_lib):
    """Step 6 after a real epoch (weights far from equal) against NumPy's
    weighted mean and biased weighted covariance; ESS = 1 / sum w^2."""
    w = W.robertson(N=600, T=3)
    f = oracle.Filter(w)
    f.init()
    for k in range(3):
        assert f.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
        st, m = f.state(), f.moments()
        wt = np.exp(st["lw"])
        assert wt.max() / wt[wt > 0].min() > 10.0          # genuinely unequal
        assert np.sum(wt) == pytest.approx(1.0, rel=1e-13)
        assert np.allclose(m["phibar"], np.average(st["phi"], axis=0, weights=wt), rtol=1e-13, atol=1e-15)
        Cref = np.cov(st["phi"].T, aweights=wt, bias=True)
        assert np.allclose(m["C"], Cref, rtol=1e-10, atol=1e-14 * np.max(np.abs(Cref)))
        assert np.allclose(m["xbar"], np.average(st["x"], axis=0, weights=wt), rtol=1e-13, atol=1e-16)
        assert m["ess"] == pytest.approx(1.0 / np.sum(wt ** 2), rel=1e-12)


def test_moments_skip_zero_weight_particles(oracle_lib):
    """A particle whose propagation failed has weight zero and a non-finite
    state: the moments are those of the others."""
    w = W.linear2(N=200, T=2)
    f = oracle.Filter(w)
    f.init()
    st = f.state()
    st["x"][13] = np.nan
    f.set_state(**st)
    assert f.epoch(w.t_obs[0], w.y_obs[0]) == oracle.OK
    st, m = f.state(), f.moments()
    wt = np.exp(st["lw"])
    dead = wt == 0.0
    assert dead.any()
    live = ~dead
    assert np.allclose(m["xbar"], np.average(st["x"][live], axis=0, weights=wt[live]), rtol=1e-13)
    assert np.allclose(m["phibar"], np.average(st["phi"][live], axis=0, weights=wt[live]), rtol=1e-13)


@pytest.mark.parametrize("a", [0.5, 0.9])
def test_proliferation_restores_covariance(oracle_lib, a):
    """Step 4a on an equally weighted ensemble with sample mean phibar and
    sample covariance C: shrinkage leaves covariance a^2 C and the kernel
    draw adds s^2 C, so the new ensemble has mean phibar and covariance C
    within Monte Carlo standard errors (s^2 = 1 - a^2)."""
    N = 20000
    rng = np.random.default_rng(int(a * 100))
    w = W.linear2(N=N, T=2).with_(a=a, kappa=0.0)
    f = oracle.Filter(w)
    f.init()
    st = f.state()
    mu = np.log(np.array([1.0, 1000.0]))
    C0 = np.array([[0.04, 0.018], [0.018, 0.02]])
    phi = rng.multivariate_normal(mu, C0, size=N)
    st["phi"] = phi
    st["lw"] = np.full(N, -np.log(N))
    f.set_state(**st)
    pb = phi.mean(axis=0)
    Cs = np.cov(phi.T, bias=True)
    f.set_moments(pb, Cs)
    tab, S = f.substeps(w.t_obs[0])
    assert f.stage2(tab, S, w.y_obs[0], np.arange(N, dtype=np.int32)) == oracle.OK
    assert f.commit(w.t_obs[0]) == oracle.OK
    new = f.state()["phi"]
    m = new.mean(axis=0)
    Cn = np.cov(new.T, bias=True)
    se_mean = np.sqrt(np.diag(Cs) * (1.0 - a * a) / N)
    assert np.all(np.abs(m - pb) <= 4.0 * se_mean + 1e-15)
    se_cov = np.sqrt((np.outer(np.diag(Cs), np.diag(Cs)) + Cs ** 2) * (1.0 - a ** 4) / N)
    assert np.all(np.abs(Cn - Cs) <= 4.0 * se_cov), (Cn, Cs)
    # what a plausible slip would give is far outside that band: s^2 = (1-a^2)^2
    wrong = a * a * Cs + (1.0 - a * a) ** 2 * Cs
    assert np.any(np.abs(wrong - Cs) > 8.0 * se_cov)
