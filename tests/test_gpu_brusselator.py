"""GPU parity of the Brusselator (d = 64) path against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import build as B
from paper_1411_1702_gb300 import workloads as W
from parity_util import check_epoch, rel_state_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    B.build()
    oracle.build()
    from paper_1411_1702_gb300 import pf as _pf
    _pf.load()
    return _pf


@pytest.mark.parametrize("N,T", [(137, 3), (33, 2)])
def test_brusselator_epoch_parity(pf, N, T):
    w = W.brusselator(N=N, T=T)
    g = pf.Filter.from_workload(w, N=N)
    o = oracle.Filter(w, N=N)
    o.init()
    for k in range(T):
        errs = check_epoch(g, o, w.t_obs[k], w.y_obs[k])
        assert errs["x"] <= 1e-10


def test_brusselator_deterministic_special_case(pf):
    w = W.brusselator(N=70, T=4)
    th = w.theta_true
    w = w.with_(a=1.0, kappa=0.0, prior_lo=list(th), prior_hi=list(th))
    g = pf.Filter.from_workload(w)
    cfg = oracle.make_config(w)
    x = np.array(w.x0, dtype=float)
    h1, h2 = x.copy(), x.copy()
    depth, hp1, hp2, t = 0, 0.0, 0.0, 0.0
    for k in range(w.T):
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
        tab, S, dout = oracle.build_substeps(cfg, t, w.t_obs[k], depth, hp1, hp2)
        x, h1, h2, _ = oracle.propagate(w.ode, w.newton_iters, th, tab, S, x, h1, h2)
        hp1, hp2 = tab[S - 1].h, tab[S - 2].h
        depth, t = dout, w.t_obs[k]
        _, _, xb = g.pf_estimates()
        assert np.max(np.abs(xb - x)) <= 1e-10 * np.max(np.abs(x))


def test_brusselator_full_size_sampled(pf):
    """The full workload (N = 65536, 20 substeps): every output the oracle can
    compute one particle at a time is checked on a sample of particles, and
    the resampling indices on all of them."""
    w = W.brusselator()
    N, d, p = w.N, w.d, w.p
    g = pf.Filter.from_workload(w)
    g.pf_assimilate(w.t_obs[0], w.y_obs[0])
    k = 1
    pre = g.pf_get_ensemble()
    phibar, Cm, _ = g.pf_estimates()
    hist = g.pf_get_history()
    g.pf_assimilate(w.t_obs[k], w.y_obs[k])
    work = g.pf_get_work()
    post = g.pf_get_ensemble()
    cfg = oracle.make_config(w)
    tab, S, _ = oracle.build_substeps(cfg, hist["t_prev"], w.t_obs[k], hist["depth"],
                                      hist["hprev1"], hist["hprev2"])
    rng = np.random.default_rng(5)
    sample = rng.choice(N, size=24, replace=False)
    # stage 1: propagate with the shrunk parameters, compare log-likelihoods
    for n in sample:
        ph = oracle.liu_west_shrink(w.a, pre["phi"][n], phibar)
        xb, _, _, _ = oracle.propagate(w.ode, w.newton_iters, np.exp(ph), tab, S, pre["x"][n],
                                       pre["h1"][n], pre["h2"][n])
        z = (w.y_obs[k] - xb[w.obs_idx]) / np.array(w.sigma)
        assert work["ll1"][n] == pytest.approx(-0.5 * np.sum(z * z), rel=1e-9, abs=1e-9)
    # cumulative weights and all indices
    c = work["c"]
    assert np.all(np.diff(c) >= 0)
    lg = work["lg"]
    assert c[-1] == pytest.approx(np.sum(np.exp(lg - lg.max())), rel=1e-12)
    u = oracle.uniform(w.seed, 0, oracle.RNG_RESAMPLE, 0, k, 0)
    assert np.array_equal(oracle.resample_systematic(c, u), work["idx"])
    # stage 2 on sampled slots: proliferation, repropagation, innovation
    L = oracle.cholesky_psd(Cm)
    s = np.sqrt(1.0 - w.a * w.a)
    for n in sample:
        l = work["idx"][n]
        zt = np.array([oracle.normal(w.seed, 0, oracle.RNG_THETA, n, k, i) for i in range(p)])
        ph = oracle.liu_west_shrink(w.a, pre["phi"][l], phibar) + s * (L @ zt)
        assert np.allclose(post["phi"][n], ph, rtol=1e-12, atol=1e-14)
        x, h1, h2, E = oracle.propagate(w.ode, w.newton_iters, np.exp(post["phi"][n]), tab, S,
                                        pre["x"][l], pre["h1"][l], pre["h2"][l], with_error=True)
        zi = np.array([oracle.normal(w.seed, 0, oracle.RNG_INNOV, n, k, i) for i in range(d)])
        v = np.sqrt(w.kappa * E) * zi
        for got, want in ((post["x"][n], x + v), (post["h1"][n], h1 + v), (post["h2"][n], h2 + v)):
            assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))
