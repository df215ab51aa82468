"""GPU parity of the 2D advection-diffusion path (the paper's Sec. 4 system,
spectral solve of each implicit step) against the CPU oracle (dense LU)."""
import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import build as B
from paper_1411_1702_gb300 import workloads as W
from parity_util import check_epoch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    B.build()
    oracle.build()
    from paper_1411_1702_gb300 import pf as _pf
    _pf.load()
    return _pf


@pytest.mark.parametrize("n,N,T", [(20, 40, 3), (20, 300, 2), (4, 7, 3), (12, 5, 2)])
def test_advdiff_epoch_parity(pf, n, N, T):
    """Cold start (two BDF1 substeps) and BDF2 epochs, every stage output."""
    w = W.advdiff(n=n, N=N, T=T, seed=n)
    g = pf.Filter.from_workload(w)
    o = oracle.Filter(w)
    o.init()
    for k in range(T):
        errs = check_epoch(g, o, w.t_obs[k], w.y_obs[k])
        assert errs["x"] <= 1e-10


def test_advdiff_large_grid_parity(pf):
    """n = 40 (d = 1521): the largest grid of the paper."""
    w = W.advdiff(n=40, N=6, T=2, seed=1)
    g = pf.Filter.from_workload(w)
    o = oracle.Filter(w)
    o.init()
    for k in range(w.T):
        check_epoch(g, o, w.t_obs[k], w.y_obs[k])


def test_advdiff_deterministic_special_case(pf):
    """a = 1, kappa = 0, point-mass prior: every particle follows the plain
    BDF2 solve; the weighted mean equals the oracle's propagation and the total
    mass of x0 is conserved."""
    w = W.advdiff(n=20, N=33, T=4)
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
        assert abs(xb.sum() - w.x0.sum()) <= 1e-11 * np.abs(w.x0).sum()


def test_advdiff_tracks_the_truth(pf):
    """A short full-size-N run: the posterior mean of the state follows the
    truth at the sensors within a few noise levels."""
    w = W.advdiff(n=20, N=5000, T=5, seed=2)
    g = pf.Filter.from_workload(w)
    for k in range(w.T):
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
    _, Cm, xb = g.pf_estimates()
    err = np.abs(xb[w.obs_idx] - w.x_true[w.T - 1][w.obs_idx])
    assert np.max(err) < 5 * w.sigma[0]
    assert np.all(np.isfinite(Cm))


def test_advdiff_argument_rules(pf):
    w = W.advdiff(n=8, N=4, T=1)
    with pytest.raises(pf.PfError) as ei:
        pf.Filter(w.ode, 64, w.p, 4, w.lmm, w.dt, w.prior_kind, w.prior_lo, w.prior_hi,
                  np.zeros(64), 0.0, a=w.a, newton_iters=1, spacing=w.spacing,
                  substeps=w.substeps, q0=0.0, history=w.history, transform=w.transform,
                  obs_idx=w.obs_idx, noise=w.noise, sigma=w.sigma, kappa=1.0, seed=0)
    assert ei.value.status == pf.PF_ERR_INVALID_ARG          # 8 x 8 is an even grid
    f = pf.Filter.from_workload(w)
    with pytest.raises(pf.PfError):
        pf.Batch([f])                                         # no batched M2 kernels
