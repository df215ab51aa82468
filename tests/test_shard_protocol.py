"""The particle-sharded filter's protocol on the CPU (paper_1411_1702_gb300/shard.py).

* The planning of the output ranges against the definition of systematic
  resampling on adversarial cumulative weights (runs of zero weight, a total
  reached early, shards without any weight).
* G = 2..5 oracle shards driven by threads, and world_size 2 and 4 gloo
  ranks, against one oracle filter of all particles from the same committed
  state: the resampled parents and every propagated state bit for bit, the
  log weights and moments to rounding (they are added in shard order).
"""
import math
import os
import threading

import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import shard as SH
from paper_1411_1702_gb300 import workloads as W
from shard_engines import OracleShard


def _definition(c, u):
    return oracle.resample_systematic(np.asarray(c, dtype=np.float64), u)


# ----------------------------------------------------------------- planning
def test_shard_bounds():
    assert SH.shard_bounds(10, 3, 1) == [0, 3, 6, 10]
    b = SH.shard_bounds(5000, 4, 1024)
    assert b[0] == 0 and b[-1] == 5000 and all(x % 1024 == 0 for x in b[1:-1])
    assert all(b[q] < b[q + 1] for q in range(4))
    with pytest.raises(ValueError):
        SH.shard_bounds(3000, 4, 1024)       # only 3 tiles


@pytest.mark.parametrize("case", range(60))
def test_plan_ranges_resolve_every_output_where_its_parent_lives(case):
    rng = np.random.default_rng(case)
    N = int(rng.integers(1, 300))
    g = rng.random(N) ** 3
    g[rng.random(N) < 0.4] = 0.0
    if case % 5 == 0:
        g[N // 2:] = 0.0                      # the total is reached early
    if case % 7 == 0:
        g[:] = 0.0
        g[int(rng.integers(N))] = 1.0         # one heavy particle
    if g.sum() == 0.0:
        g[0] = 1.0
    c = np.cumsum(g)
    u = float(rng.random()) if case % 3 else (0.0 if case % 2 else 1.0 - 2.0 ** -53)
    idx = _definition(c, u)
    G = int(rng.integers(1, min(6, N) + 1))
    cuts = sorted(rng.choice(np.arange(1, N), size=G - 1, replace=False).tolist()) if G > 1 else []
    bounds = [0] + cuts + [N]
    ranges, i_fb = SH.plan_ranges(bounds, 1, c, float(c[-1]), u)
    # the ranges tile [0, N) in shard order
    assert ranges[0][0] == 0 and max(r[1] for r in ranges) == N
    for q in range(G - 1):
        assert ranges[q][1] <= ranges[q + 1][0] or ranges[q + 1] == (N, N)
    covered = np.zeros(N, dtype=int)
    for q, (lo, hi) in enumerate(ranges):
        covered[lo:hi] += 1
        # every output of shard q's range has its parent among q's slots
        assert np.all((idx[lo:hi] >= bounds[q]) & (idx[lo:hi] < bounds[q + 1])), (q, ranges, bounds)
    assert np.all(covered == 1)
    assert i_fb == sum(1 for i in range(N) if SH.threshold(i, u, N, float(c[-1])) < c[-1])
    # the exchange: each shard receives exactly its slots, once
    for me in range(G):
        send, recv = SH.exchange_counts(ranges, bounds, me)
        assert sum(recv) == bounds[me + 1] - bounds[me]
        assert sum(send) == ranges[me][1] - ranges[me][0]


# ------------------------------------------------- oracle shards, threads
def _sync(shard_engines, bounds, ref, state, mom, hist):
    """Give every shard and the reference the same committed state."""
    ref.set_state(**state)
    ref.set_moments(mom["phibar"], mom["C"])
    ref.set_history(**hist)
    for e, lo, hi in zip(shard_engines, bounds[:-1], bounds[1:]):
        e.o.set_state(**{k: v[lo:hi] for k, v in state.items()})
        e.o.set_moments(mom["phibar"], mom["C"])
        e.o.set_history(**hist)


def _run_threads(engines, bounds, t, y):
    hub = SH.ThreadComm(len(engines), timeout=120.0)
    errs = []
    filters = [None] * len(engines)

    def body(r):
        try:
            if filters[r] is None:
                filters[r] = SH.ShardedFilter.__new__(SH.ShardedFilter)
                filters[r].e, filters[r].comm = engines[r], hub.view(r)
                filters[r].bounds, filters[r].tile = bounds, 1
                filters[r].N, filters[r].rec = bounds[-1], engines[r].info["record"]
            filters[r].assimilate(t, y)
        except BaseException as ex:   # noqa: BLE001 - reported below
            errs.append(ex)
            hub.abort()

    th = [threading.Thread(target=body, args=(r,)) for r in range(len(engines))]
    for x in th:
        x.start()
    for x in th:
        x.join()
    if errs:
        raise errs[0]


def _reference_epoch(ref, t, y):
    tab, S = ref.substeps(t)
    assert ref.stage1(tab, S, y) == oracle.OK
    assert ref.cumulative() == oracle.OK
    idx = oracle.resample_systematic(ref.work()["c"], ref.resample_u())
    assert ref.stage2(tab, S, y, idx) == oracle.OK
    assert ref.commit(t) == oracle.OK
    return idx


def _compare(engines, bounds, ref, idx):
    st = ref.state()
    for e, lo, hi in zip(engines, bounds[:-1], bounds[1:]):
        assert np.array_equal(e.parents, idx[lo:hi]), "resampled parents differ"
        s = e.o.state()
        for k in ("x", "h1", "h2", "phi"):
            assert np.array_equal(s[k], st[k][lo:hi]), k
        assert np.allclose(s["lw"], st["lw"][lo:hi], rtol=1e-12, atol=1e-12)
    m = ref.moments()
    for e in engines:
        me = e.o.moments()
        assert np.allclose(me["phibar"], m["phibar"], rtol=1e-12, atol=1e-14)
        assert np.allclose(me["C"], m["C"], rtol=1e-8, atol=1e-13 * np.max(np.abs(m["C"])))
        assert np.allclose(me["xbar"], m["xbar"], rtol=1e-12, atol=1e-15)
        assert me["ess"] == pytest.approx(m["ess"], rel=1e-10)


@pytest.mark.parametrize("name,N,G", [("linear2", 700, 2), ("robertson", 901, 3),
                                      ("michaelis", 640, 4), ("linear2", 333, 5)])
def test_oracle_shards_equal_one_filter(oracle_lib, name, N, G):
    w = W.get(name, N=N, T=4)
    ref = oracle.Filter(w)
    ref.init()
    bounds = SH.shard_bounds(N, G, 1)
    engines = [OracleShard(w, N, lo, hi - lo) for lo, hi in zip(bounds[:-1], bounds[1:])]
    for k in range(w.T):
        _sync(engines, bounds, ref, ref.state(), ref.moments(), ref.history())
        _run_threads(engines, bounds, w.t_obs[k], w.y_obs[k])
        idx = _reference_epoch(ref, w.t_obs[k], w.y_obs[k])
        _compare(engines, bounds, ref, idx)
        assert len(np.unique(idx)) < N      # resampling moved particles between shards
        moved = sum(np.sum((e.parents < lo) | (e.parents >= hi))
                    for e, lo, hi in zip(engines, bounds[:-1], bounds[1:]))
        if k > 0:
            assert moved > 0


def test_oracle_shards_run_alone(oracle_lib):
    """The shards from Step 1 on, with no syncing: Step 1 draws the same
    particles as one filter (random streams keyed by the global slot), every
    shard commits the same moments each epoch, and the posterior ends near
    one filter's (the moments are added in shard order, so the runs agree to
    rounding only, and a rounding difference can move a resampling index)."""
    w = W.robertson(N=1000, T=8)
    G = 3
    bounds = SH.shard_bounds(w.N, G, 1)
    engines = [OracleShard(w, w.N, lo, hi - lo) for lo, hi in zip(bounds[:-1], bounds[1:])]
    ref = oracle.Filter(w)
    ref.init()
    phi0 = np.concatenate([e.o.state()["phi"] for e in engines])
    assert np.array_equal(phi0, ref.state()["phi"])
    hub = SH.ThreadComm(G, timeout=120.0)
    fs = [None] * G

    def make(r):
        fs[r] = SH.ShardedFilter(engines[r], hub.view(r), bounds, 1)

    th = [threading.Thread(target=make, args=(r,)) for r in range(G)]
    [x.start() for x in th]
    [x.join() for x in th]
    m0 = ref.moments()
    for e in engines:
        assert np.allclose(e.o.moments()["phibar"], m0["phibar"], rtol=1e-13)
        assert np.allclose(e.o.moments()["C"], m0["C"], rtol=1e-10)
    for k in range(w.T):
        th = [threading.Thread(target=fs[r].assimilate, args=(w.t_obs[k], w.y_obs[k])) for r in range(G)]
        [x.start() for x in th]
        [x.join() for x in th]
        assert ref.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
        ms = [e.o.moments() for e in engines]
        for m in ms[1:]:
            assert np.array_equal(m["phibar"], ms[0]["phibar"]) and np.array_equal(m["C"], ms[0]["C"])
        lw = np.concatenate([e.o.state()["lw"] for e in engines])
        assert np.sum(np.exp(lw)) == pytest.approx(1.0, rel=1e-12)
    assert np.all(np.abs(ms[0]["phibar"] - ref.moments()["phibar"]) < 0.1)


def test_degenerate_epoch_is_aborted_on_every_shard(oracle_lib):
    w = W.linear2(N=300, T=3)
    bounds = SH.shard_bounds(w.N, 2, 1)
    engines = [OracleShard(w, w.N, lo, hi - lo) for lo, hi in zip(bounds[:-1], bounds[1:])]
    hub = SH.ThreadComm(2, timeout=120.0)
    fs = [None, None]
    th = [threading.Thread(target=lambda r=r: fs.__setitem__(r, SH.ShardedFilter(engines[r], hub.view(r), bounds, 1)))
          for r in range(2)]
    [x.start() for x in th]
    [x.join() for x in th]
    for e in engines:
        st = e.o.state()
        st["x"][:] = np.nan                    # every particle fails: no weight anywhere
        e.o.set_state(**st)
    before = [e.o.state() for e in engines]
    out = []

    def run(r):
        try:
            fs[r].assimilate(w.t_obs[0], w.y_obs[0])
            out.append(None)
        except SH.DegenerateEpoch as ex:
            out.append(ex)

    th = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    [x.start() for x in th]
    [x.join() for x in th]
    assert len(out) == 2 and all(isinstance(v, SH.DegenerateEpoch) for v in out)
    for e, b in zip(engines, before):
        assert np.array_equal(e.o.state()["phi"], b["phi"])


# --------------------------------------------------------------- gloo ranks
def _gloo_rank(rank, world, port, name, N, T, q):
    """One gloo rank: an oracle shard, and (on every rank alike) one oracle
    filter of all particles as the reference.  Before each epoch the shard
    takes its slots of the reference's committed state; after it, its
    parents and states are compared with the reference's epoch."""
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    out = []
    try:
        oracle.build()
        w = W.get(name, N=N, T=T)
        bounds = SH.shard_bounds(N, world, 1)
        lo, hi = bounds[rank], bounds[rank + 1]
        eng = OracleShard(w, N, lo, hi - lo)
        f = SH.ShardedFilter(eng, SH.TorchComm(), bounds, 1)
        ref = oracle.Filter(w)
        ref.init()
        for k in range(T):
            st, m, h = ref.state(), ref.moments(), ref.history()
            eng.o.set_state(**{key: v[lo:hi] for key, v in st.items()})
            eng.o.set_moments(m["phibar"], m["C"])
            eng.o.set_history(**h)
            f.assimilate(w.t_obs[k], w.y_obs[k])
            idx = _reference_epoch(ref, w.t_obs[k], w.y_obs[k])
            rs, es = ref.state(), eng.o.state()
            same = (np.array_equal(eng.parents, idx[lo:hi]) and
                    all(np.array_equal(es[key], rs[key][lo:hi]) for key in ("x", "h1", "h2", "phi")) and
                    np.allclose(es["lw"], rs["lw"][lo:hi], rtol=1e-12, atol=1e-12) and
                    np.allclose(eng.o.moments()["phibar"], ref.moments()["phibar"], rtol=1e-12))
            moved = int(np.sum((eng.parents < lo) | (eng.parents >= hi)))
            out.append((same, moved))
        q.put((rank, out, None))
    except BaseException as ex:   # noqa: BLE001 - reported to the test
        q.put((rank, out, repr(ex)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_equal_one_filter(oracle_lib, world):
    """world_size 2 and 4 gloo processes, each an oracle shard exchanging
    through torch.distributed (TorchComm): every epoch, from the same
    committed state, the parents and states equal one oracle filter's bit
    for bit, and particles do move between ranks."""
    import multiprocessing as mp
    name, N, T = "robertson", 640, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29600 + 10 * world + (os.getpid() % 300)
    ps = [ctx.Process(target=_gloo_rank, args=(r, world, port, name, N, T, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = {}
    try:
        for _ in range(world):
            r, out, err = q.get(timeout=300)
            assert err is None, (r, err)
            res[r] = out
    finally:
        for p in ps:
            p.join(timeout=60)
            if p.exitcode is None:
                p.kill()
    for p in ps:
        assert p.exitcode == 0
    for k in range(T):
        assert all(res[r][k][0] for r in range(world)), k
    assert sum(res[r][k][1] for r in range(world) for k in range(T)) > 0
