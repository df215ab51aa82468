"""GPU parity of the BDF3, Adams-Moulton and Adams-Bashforth propagation
kernels (the first three methods of each family, Sec. 3, Tables 1-2) and of
the paper's M1 Michaelis-Menten system (Sec. 2.1), through the C ABI, against
the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import build as B
from paper_1411_1702_gb300 import workloads as W
from parity_util import assert_within_three_mc_se, check_epoch

pytestmark = pytest.mark.gpu

NEW_LMMS = [W.LMM_BDF3, W.LMM_AM1, W.LMM_AM2, W.LMM_AM3, W.LMM_AB1, W.LMM_AB2, W.LMM_AB3]


@pytest.fixture(scope="module")
def pf():
    B.build()
    oracle.build()
    from paper_1411_1702_gb300 import pf as _pf
    _pf.load()
    return _pf


def _pair(pf, w, N=None):
    g = pf.Filter.from_workload(w, N=N)
    o = oracle.Filter(w, N=N)
    o.init()
    return g, o


@pytest.mark.parametrize("lmm", [W.LMM_BDF1, W.LMM_BDF2] + NEW_LMMS)
def test_michaelis_epoch_parity(pf, lmm):
    """Cold start (the order ramp), carried history and every stage output,
    at a ragged N over several tiles."""
    w = W.michaelis(N=1537, T=4, lmm=lmm)
    g, o = _pair(pf, w)
    for k in range(w.T):
        errs = check_epoch(g, o, w.t_obs[k], w.y_obs[k], exempt_dead=True)
        assert errs["x"] <= 1e-10 and errs["dead"] < w.N


@pytest.mark.parametrize("lmm", NEW_LMMS)
def test_linear2_epoch_parity(pf, lmm):
    """The stiff linear system (AB steps amplify its stiff mode on part of
    the prior; those particles get zero weight on both sides)."""
    w = W.linear2(N=1029, T=3).with_(lmm=lmm)
    g, o = _pair(pf, w)
    for k in range(w.T):
        check_epoch(g, o, w.t_obs[k], w.y_obs[k], exempt_dead=True)


@pytest.mark.parametrize("lmm", [W.LMM_BDF1, W.LMM_BDF2] + NEW_LMMS)
def test_robertson_uniform_epoch_parity(pf, lmm):
    """Robertson on a uniform grid (2e-6 steps) with each of the nine methods."""
    w = W.robertson(N=300, T=3)
    w = w.with_(lmm=lmm, spacing=W.SPACING_UNIFORM, dt=2e-6,
                t_obs=np.array([1e-4, 2e-4, 3e-4]), y_obs=w.y_obs[:3], x_true=w.x_true[:3])
    g, o = _pair(pf, w)
    for k in range(w.T):
        check_epoch(g, o, w.t_obs[k], w.y_obs[k], exempt_dead=True)


@pytest.mark.parametrize("lmm", [W.LMM_BDF2, W.LMM_AM3, W.LMM_AB3])
def test_michaelis_full_size(pf, lmm):
    """The benchmark's M1 size (N = 50000): full per-particle parity over the
    first epochs and one after a GPU-only stretch."""
    w = W.michaelis(lmm=lmm)
    g, o = _pair(pf, w)
    for k in range(2):
        check_epoch(g, o, w.t_obs[k], w.y_obs[k], exempt_dead=True)
    for k in range(2, 12):
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
    check_epoch(g, o, w.t_obs[12], w.y_obs[12], exempt_dead=True)


@pytest.mark.parametrize("lmm", [W.LMM_BDF3, W.LMM_AM2, W.LMM_AB3])
def test_michaelis_deterministic_special_case(pf, lmm):
    """a = 1, kappa = 0, point-mass prior: the GPU's weighted mean equals the
    oracle's plain solve by the same method."""
    w = W.michaelis(N=97, T=6, lmm=lmm)
    th = w.theta_true
    w = w.with_(a=1.0, kappa=0.0, prior_lo=list(th), prior_hi=list(th))
    g = pf.Filter.from_workload(w)
    cfg = oracle.make_config(w)
    x = np.array(w.x0)
    h1, h2 = x.copy(), x.copy()
    depth, hp1, hp2, t = 0, 0.0, 0.0, 0.0
    for k in range(w.T):
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
        tab, S, dout = oracle.build_substeps(cfg, t, w.t_obs[k], depth, hp1, hp2)
        x, h1, h2, _ = oracle.propagate(w.ode, w.newton_iters, th, tab, S, x, h1, h2)
        hp1, hp2, depth, t = tab[S - 1].h, tab[S - 2].h, dout, w.t_obs[k]
        _, _, xb = g.pf_estimates()
        assert np.max(np.abs(xb - x) / np.abs(x)) <= 1e-12


def test_michaelis_tracks_truth(pf):
    """A whole run of each family at the benchmark size: the posterior mean
    of the state follows the truth and the identifiable ratios V/k approach
    their true values."""
    for lmm in (W.LMM_BDF2, W.LMM_AM3, W.LMM_AB3):
        w = W.michaelis(lmm=lmm)
        g = pf.Filter.from_workload(w)
        for k in range(w.T):
            g.pf_assimilate(w.t_obs[k], w.y_obs[k])
        tb, _, xb = g.pf_estimates()
        assert np.allclose(xb, w.x_true[-1], rtol=0.05)
        ratio = np.exp(tb[[0, 1]] - tb[[2, 3]])
        true = np.array(W.MM_THETA)[[0, 1]] / np.array(W.MM_THETA)[[2, 3]]
        assert np.all(np.abs(np.log(ratio / true)) < 0.4), (lmm, ratio)


def test_lmm_argument_rules(pf):
    w = W.michaelis(N=16, T=2, lmm=W.LMM_AM2)
    # the new families need uniform spacing
    with pytest.raises(pf.PfError) as ei:
        pf.Filter.from_workload(W.robertson(N=8, T=2).with_(lmm=W.LMM_AB2))
    assert ei.value.status == pf.PF_ERR_INVALID_ARG
    # and one of the small problems
    with pytest.raises(pf.PfError) as ei:
        pf.Filter.from_workload(W.brusselator(N=8, T=2).with_(lmm=W.LMM_BDF3))
    assert ei.value.status == pf.PF_ERR_INVALID_ARG
    # M1 and every family batch (the batch launches one group per problem and family)
    f = pf.Filter.from_workload(w)
    f2 = pf.Filter.from_workload(W.linear2(N=8, T=2).with_(lmm=W.LMM_AM3))
    b = pf.Batch([f, f2])
    assert b.pf_batch_assimilate([w.t_obs[0], 0.1], [w.y_obs[0], [1.0]]) == [pf.PF_OK] * 2


@pytest.mark.parametrize("lmm", [W.LMM_BDF2, W.LMM_AM3])
def test_long_substep_table(pf, lmm):
    """600 substeps per interval: the staged step table needs more than the
    default 48 KB of dynamic shared memory."""
    w = W.linear2(N=300, T=2).with_(lmm=lmm, dt=0.1 / 600)
    g, o = _pair(pf, w)
    for k in range(w.T):
        check_epoch(g, o, w.t_obs[k], w.y_obs[k])


@pytest.mark.parametrize("lmm", [W.LMM_BDF3, W.LMM_AM3, W.LMM_AB3])
def test_michaelis_independent_runs_agree(pf, lmm):
    """GPU and oracle each run the whole M1 filter on their own (own scan and
    resampling) with the same seed: the same resampled indices every epoch,
    and the same posterior."""
    w = W.michaelis(N=3000, lmm=lmm)
    g, o = _pair(pf, w)
    for k in range(w.T):
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
        assert o.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
        assert np.array_equal(g.pf_get_work()["idx"], o.work()["idx"]), k
    tb, Cm, xb = g.pf_estimates()
    om = o.moments()
    assert np.allclose(tb, om["phibar"], rtol=1e-9, atol=1e-12)
    assert np.allclose(xb, om["xbar"], rtol=1e-9)


def test_michaelis_posterior_within_three_mc_standard_errors(pf):
    """M1 (AM2): the GPU's posterior mean and diag C over 16 filter seeds
    against the oracle's over 16 disjoint seeds, within 3 Monte Carlo
    standard errors."""
    w0 = W.michaelis(N=2000, lmm=W.LMM_AM2)
    assert_within_three_mc_se(pf, lambda s: w0.with_(seed=s))


@pytest.mark.parametrize("lmm", [W.LMM_BDF3, W.LMM_AM3, W.LMM_AB2])
def test_michaelis_restart_history_parity(pf, lmm):
    """RESTART history (a cold start every interval, the literal Psi(x_j)
    reading): the order ramp runs in every interval."""
    w = W.michaelis(N=700, T=3, lmm=lmm).with_(history=W.HIST_RESTART)
    g, o = _pair(pf, w)
    for k in range(w.T):
        check_epoch(g, o, w.t_obs[k], w.y_obs[k], exempt_dead=True)


@pytest.mark.parametrize("lmm", [W.LMM_BDF3, W.LMM_AM2, W.LMM_AB3])
def test_device_series_equals_host_calls(pf, lmm):
    """pf_load_observations + pf_run (M1's inputs tabulated for the whole
    series up front) give the same ensemble as one pf_assimilate per
    observation."""
    w = W.michaelis(N=1500, T=12, lmm=lmm)
    a = pf.Filter.from_workload(w)
    for k in range(w.T):
        a.pf_assimilate(w.t_obs[k], w.y_obs[k])
    b = pf.Filter.from_workload(w)
    b.pf_load_observations(w.t_obs, w.y_obs)
    b.pf_run(0, w.T)
    b.pf_synchronize()
    ea, eb = a.pf_get_ensemble(), b.pf_get_ensemble()
    for key in ea:
        assert np.array_equal(ea[key], eb[key], equal_nan=True), key
