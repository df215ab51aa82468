"""The particle-sharded filter on the GPU: G shards of one filter (pf_shard_*
calls through the C ABI), driven by threads of one process on one GPU and
exchanging through host-ordered copies (ThreadComm), against one filter of
all particles from the same committed state.  The resampled parents and the
propagated states must agree bit for bit (the shards use the whole
ensemble's scan tiling and random streams keyed by the global slot), the log
weights and moments to rounding (they are added in shard order).  Every shard
is also compared with the CPU oracle's epoch through the parity checker."""
import threading

import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import build as B
from paper_1411_1702_gb300 import shard as SH
from paper_1411_1702_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    B.build()
    oracle.build()
    from paper_1411_1702_gb300 import pf
    pf.load()
    return pf, torch


def _run(G, fn, hub):
    errs = []

    def body(r):
        try:
            fn(r)
        except BaseException as ex:   # noqa: BLE001 - re-raised below
            errs.append(ex)
            hub.abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(G)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    if errs:
        raise errs[0]


def _make(pf, torch, w, G):
    N = w.N
    tile = pf.pf_shard_tile(N)
    bounds = SH.shard_bounds(N, G, tile)
    engines = [SH.LibraryShard(pf, w, N, lo, hi - lo) for lo, hi in zip(bounds[:-1], bounds[1:])]
    torch.cuda.synchronize()
    hub = SH.ThreadComm(G, timeout=300.0)
    fs = [None] * G

    def mk(r):
        fs[r] = SH.ShardedFilter(engines[r], hub.view(r), bounds, tile)

    _run(G, mk, hub)
    return engines, fs, hub, bounds


def _sync(g, engines, bounds):
    st = g.pf_get_ensemble()
    tb, Cm, _ = g.pf_estimates()
    h = g.pf_get_history()
    g.pf_set_ensemble(**st)
    g.pf_set_moments(tb, Cm)
    for e, lo, hi in zip(engines, bounds[:-1], bounds[1:]):
        e.f.pf_set_ensemble(**{k: v[lo:hi] for k, v in st.items()})
        e.f.pf_set_moments(tb, Cm)
        e.f.pf_set_history(h["epoch"], h["depth"], h["t_prev"], h["hprev1"], h["hprev2"])


@pytest.mark.parametrize("name,N,G", [("robertson", 131072, 4), ("robertson", 3001, 3),
                                      ("linear2", 2000, 2), ("michaelis", 5000, 3),
                                      ("brusselator", 1100, 2), ("robertson", 4096, 1)])
def test_shards_equal_one_filter(env, name, N, G):
    pf, torch = env
    w = W.get(name, N=N, T=4)
    g = pf.Filter.from_workload(w)
    engines, fs, hub, bounds = _make(pf, torch, w, G)
    moved = 0
    for k in range(w.T):
        _sync(g, engines, bounds)
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
        _run(G, lambda r: fs[r].assimilate(w.t_obs[k], w.y_obs[k]), hub)
        idx = g.pf_get_work()["idx"]
        ge = g.pf_get_ensemble()
        tb, Cm, xb = g.pf_estimates()
        for e, lo, hi in zip(engines, bounds[:-1], bounds[1:]):
            par = e.f.pf_shard_parents()
            assert np.array_equal(par, idx[lo:hi]), (name, k, "parents")
            moved += int(np.sum((par < lo) | (par >= hi)))
            se = e.f.pf_get_ensemble()
            for key in ("x", "h1", "h2", "phi"):
                assert np.array_equal(se[key], ge[key][lo:hi], equal_nan=True), (name, k, key)
            fin = np.isfinite(ge["lw"][lo:hi])
            assert np.array_equal(np.isfinite(se["lw"]), fin)
            assert np.allclose(se["lw"][fin], ge["lw"][lo:hi][fin], rtol=1e-12, atol=1e-12)
            stb, sC, sxb = e.f.pf_estimates()
            assert np.allclose(stb, tb, rtol=1e-12, atol=1e-14)
            assert np.allclose(sC, Cm, rtol=1e-8, atol=1e-12 * max(np.max(np.abs(Cm)), 1e-300))
            assert np.allclose(sxb, xb, rtol=1e-12, atol=1e-15)
    if G > 1:
        assert moved > 0          # offspring crossed shard boundaries


def test_shards_against_oracle(env):
    """Each shard's epoch against the oracle's epoch of the whole ensemble
    from the same committed state (the same check as a filter's parity)."""
    pf, torch = env
    w = W.robertson(N=3001, T=3)
    G = 3
    engines, fs, hub, bounds = _make(pf, torch, w, G)
    o = oracle.Filter(w)
    o.init()
    for k in range(w.T):
        st = {key: np.concatenate([e.f.pf_get_ensemble()[key] for e in engines])
              for key in ("x", "h1", "h2", "phi", "lw")}
        tb, Cm, _ = engines[0].f.pf_estimates()
        for e, lo, hi in zip(engines, bounds[:-1], bounds[1:]):
            e.f.pf_set_ensemble(**{key: v[lo:hi] for key, v in st.items()})
            e.f.pf_set_moments(tb, Cm)
        o.set_state(**st)
        o.set_moments(tb, Cm)
        h = engines[0].f.pf_get_history()
        o.set_history(h["epoch"], h["depth"], h["t_prev"], h["hprev1"], h["hprev2"])
        _run(G, lambda r: fs[r].assimilate(w.t_obs[k], w.y_obs[k]), hub)
        tab, S = o.substeps(w.t_obs[k])
        assert o.stage1(tab, S, w.y_obs[k]) == oracle.OK
        assert o.cumulative() == oracle.OK
        c = o.work()["c"]
        par = np.concatenate([e.f.pf_shard_parents() for e in engines])
        # the shards' parents are the systematic indices of their own
        # cumulative weights, which agree with the oracle's to rounding
        c_gpu = np.concatenate([e.f.pf_get_work()["c"] for e in engines])
        assert np.allclose(c_gpu, c, rtol=1e-9, atol=1e-12 * c[-1])
        assert np.array_equal(par, oracle.resample_systematic(c_gpu, o.resample_u()))
        assert o.stage2(tab, S, w.y_obs[k], par.astype(np.int32)) == oracle.OK
        assert o.commit(w.t_obs[k]) == oracle.OK
        os_ = o.state()
        x = np.concatenate([e.f.pf_get_ensemble()["x"] for e in engines])
        scale = np.maximum(np.max(np.abs(os_["x"]), axis=1), 1e-300)
        assert np.max(np.max(np.abs(x - os_["x"]), axis=1) / scale) <= 1e-10
        tb2, _, _ = engines[0].f.pf_estimates()
        assert np.allclose(tb2, o.moments()["phibar"], rtol=1e-9)


def test_shard_rules(env):
    pf, torch = env
    w = W.robertson(N=5000, T=2)
    tile = pf.pf_shard_tile(5000)
    with pytest.raises(pf.PfError):            # not on a tile boundary
        pf.Filter.from_workload(w, N=100, shard=(5000, 1))
    s = pf.Filter.from_workload(w, N=tile, shard=(5000, 0))
    with pytest.raises(pf.PfError) as ei:      # whole-filter calls are closed
        s.pf_assimilate(w.t_obs[0], w.y_obs[0])
    assert ei.value.status == pf.PF_ERR_STATE
    with pytest.raises(pf.PfError) as ei:      # Step 1's commit comes first
        s.pf_shard_stage1(w.t_obs[0], w.y_obs[0])
    assert ei.value.status == pf.PF_ERR_STATE
    with pytest.raises(pf.PfError):
        pf.Batch([s])
