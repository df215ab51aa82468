"""Batches of filters: bit-identical to each filter alone, idle filters,
isolated failures, graph reuse."""
import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import build as B
from paper_1411_1702_gb300 import workloads as W
from parity_util import begin_epoch, finish_epoch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    B.build()
    oracle.build()
    from paper_1411_1702_gb300 import pf as _pf
    _pf.load()
    return _pf


def _mix(T=4):
    specs = [("linear2", 1000, 1), ("robertson", 3001, 2), ("linear2", 2053, 3),
             ("robertson", 129, 4), ("brusselator", 70, 5), ("linear2", 1, 6),
             ("robertson", 20000, 7)]
    return [W.get(name, N=N, T=T, seed=seed) for name, N, seed in specs]


def _same(a, b):
    ea, eb = a.pf_get_ensemble(), b.pf_get_ensemble()
    return all(np.array_equal(ea[k], eb[k], equal_nan=True) for k in ea)


def test_batched_equals_alone(pf):
    ws = _mix(T=4)
    alone = [pf.Filter.from_workload(w) for w in ws]
    members = [pf.Filter.from_workload(w) for w in ws]
    batch = pf.Batch(members)
    for k in range(4):
        for f, w in zip(alone, ws):
            f.pf_assimilate(w.t_obs[k], w.y_obs[k])
        st = batch.pf_batch_assimilate([w.t_obs[k] for w in ws], [w.y_obs[k] for w in ws])
        assert st == [pf.PF_OK] * len(ws)
        for a, m in zip(alone, members):
            assert _same(a, m)
            ta, Ca, xa = a.pf_estimates()
            tm, Cm, xm = m.pf_estimates()
            assert np.array_equal(ta, tm) and np.array_equal(Ca, Cm) and np.array_equal(xa, xm)
            assert a.pf_get_history() == m.pf_get_history()
    stats = batch.pf_batch_stats()
    assert stats["epochs"] == 4 and stats["graph_captures"] == 1
    assert stats["last_active"] == len(ws)


def test_idle_filters_and_graph_recapture(pf):
    ws = _mix(T=5)
    alone = [pf.Filter.from_workload(w) for w in ws]
    members = [pf.Filter.from_workload(w) for w in ws]
    batch = pf.Batch(members)
    counts = [0] * len(ws)
    schedule = [[1, 1, 1, 1, 1, 1, 1], [1, 0, 1, 0, 1, 0, 1], [1, 0, 1, 0, 1, 0, 1],
                [0, 1, 1, 1, 0, 1, 0], [1, 1, 1, 1, 1, 1, 1]]
    for row in schedule:
        ts, ys = [], []
        for i, (w, on) in enumerate(zip(ws, row)):
            k = counts[i]
            ts.append(w.t_obs[k] if on else 0.0)
            ys.append(w.y_obs[k] if on else None)
            if on:
                alone[i].pf_assimilate(w.t_obs[k], w.y_obs[k])
                counts[i] += 1
        assert batch.pf_batch_assimilate(ts, ys) == [pf.PF_OK] * len(ws)
    for a, m in zip(alone, members):
        assert _same(a, m)
    # a graph is captured when an active set repeats (row 2 repeats row 1)
    assert batch.pf_batch_stats()["graph_captures"] == 1


def test_failure_is_isolated(pf):
    ws = _mix(T=3)
    alone = [pf.Filter.from_workload(w) for w in ws]
    members = [pf.Filter.from_workload(w) for w in ws]
    batch = pf.Batch(members)
    bad = 2
    st = members[bad].pf_get_ensemble()
    st["x"][:] = np.nan
    members[bad].pf_set_ensemble(**st)
    before = members[bad].pf_get_ensemble()
    ts = [w.t_obs[0] for w in ws]
    ys = [w.y_obs[0] for w in ws]
    ys[4] = np.full_like(ws[4].y_obs[0], np.nan)        # invalid observation
    status = batch.pf_batch_assimilate(ts, ys)
    for i, (a, w) in enumerate(zip(alone, ws)):
        if i == bad:
            assert status[i] == pf.PF_ERR_DEGENERATE
        elif i == 4:
            assert status[i] == pf.PF_ERR_INVALID_ARG
        else:
            assert status[i] == pf.PF_OK
            a.pf_assimilate(w.t_obs[0], w.y_obs[0])
            assert _same(a, members[i])
    after = members[bad].pf_get_ensemble()
    assert np.array_equal(after["phi"], before["phi"]) and np.all(np.isnan(after["x"]))
    assert members[bad].pf_get_history()["epoch"] == 0
    # the failed filters recover and keep advancing with the batch
    good = pf.Filter.from_workload(ws[bad])
    members[bad].pf_set_ensemble(**good.pf_get_ensemble())
    status = batch.pf_batch_assimilate([w.t_obs[0] if i in (bad, 4) else w.t_obs[1]
                                        for i, w in enumerate(ws)],
                                       [w.y_obs[0] if i in (bad, 4) else w.y_obs[1]
                                        for i, w in enumerate(ws)])
    assert status == [pf.PF_OK] * len(ws)


def test_batch_membership_rules(pf):
    ws = _mix(T=2)[:2]
    fs = [pf.Filter.from_workload(w) for w in ws]
    b1 = pf.Batch(fs)
    with pytest.raises(pf.PfError):
        pf.Batch(fs)                      # already in a batch
    b1.close()
    b2 = pf.Batch(fs)                     # free again after the first batch is gone
    b2.close()
    with pytest.raises(pf.PfError):
        pf.Batch([fs[0], fs[0]])


def test_batched_lmm_families_and_m1_equal_alone(pf):
    """Every LMM family and the paper's M1 system in one batch (each family is
    a separate group of launches): bit-identical to each filter alone."""
    ws = [W.michaelis(N=3001, T=4, seed=1, lmm=W.LMM_AM3),
          W.michaelis(N=700, T=4, seed=2, lmm=W.LMM_AB2),
          W.michaelis(N=1500, T=4, seed=3, lmm=W.LMM_BDF3),
          W.michaelis(N=257, T=4, seed=4, lmm=W.LMM_BDF2),
          W.linear2(N=1000, T=4, seed=5).with_(lmm=W.LMM_AM2),
          W.linear2(N=513, T=4, seed=6).with_(lmm=W.LMM_AB3),
          W.robertson(N=2000, T=4, seed=7),
          W.brusselator(N=65, T=4, seed=8)]
    alone = [pf.Filter.from_workload(w) for w in ws]
    members = [pf.Filter.from_workload(w) for w in ws]
    batch = pf.Batch(members)
    for k in range(4):
        for f, w in zip(alone, ws):
            f.pf_assimilate(w.t_obs[k], w.y_obs[k])
        st = batch.pf_batch_assimilate([w.t_obs[k] for w in ws], [w.y_obs[k] for w in ws])
        assert st == [pf.PF_OK] * len(ws)
        for a, m in zip(alone, members):
            assert _same(a, m)
            assert all(np.array_equal(u, v) for u, v in zip(a.pf_estimates(), m.pf_estimates()))


def test_large_member_batched_equals_alone(pf):
    # alone, a filter above one wave of merge tiles resamples in two launches
    # (corners first); in a batch its tiles find their own corners: the
    # indices, and so everything after them, must agree bit for bit
    ws = [W.robertson(N=400000, T=2), W.linear2(N=1000, T=2)]
    alone = [pf.Filter.from_workload(w) for w in ws]
    members = [pf.Filter.from_workload(w) for w in ws]
    batch = pf.Batch(members)
    for k in range(2):
        for f, w in zip(alone, ws):
            f.pf_assimilate(w.t_obs[k], w.y_obs[k])
        st = batch.pf_batch_assimilate([w.t_obs[k] for w in ws], [w.y_obs[k] for w in ws])
        assert st == [pf.PF_OK] * len(ws)
        for a, m in zip(alone, members):
            assert np.array_equal(a.pf_get_work()["idx"], m.pf_get_work()["idx"])
            assert _same(a, m)


def _every_problem_and_family(T=4):
    """One member of each (problem, LMM family) the batched kernels serve."""
    return [W.linear2(N=1000, T=T, seed=31),
            W.linear2(N=513, T=T, seed=32).with_(lmm=W.LMM_AM2),
            W.linear2(N=700, T=T, seed=33).with_(lmm=W.LMM_AB3),
            W.linear2(N=257, T=T, seed=34).with_(lmm=W.LMM_BDF3),
            W.robertson(N=3001, T=T, seed=35),
            W.brusselator(N=70, T=T, seed=36),
            W.michaelis(N=1500, T=T, seed=37, lmm=W.LMM_BDF3),
            W.michaelis(N=2049, T=T, seed=38, lmm=W.LMM_AM3),
            W.michaelis(N=700, T=T, seed=39, lmm=W.LMM_AB2),
            W.michaelis(N=257, T=T, seed=40, lmm=W.LMM_BDF2)]


def test_batched_members_match_oracle(pf):
    """Every member of a mixed batch, epoch by epoch, against the oracle run
    from that member's committed state: every stage output per particle
    (states to 1e-10, indices bit-exact given the member's cumulative
    weights, weights and moments within the derived bounds)."""
    ws = _every_problem_and_family()
    members = [pf.Filter.from_workload(w) for w in ws]
    orcs = [oracle.Filter(w) for w in ws]
    for o in orcs:
        o.init()
    batch = pf.Batch(members)
    for k in range(4):
        pres = [begin_epoch(m, o) for m, o in zip(members, orcs)]
        st = batch.pf_batch_assimilate([w.t_obs[k] for w in ws], [w.y_obs[k] for w in ws])
        assert st == [pf.PF_OK] * len(ws)
        for m, o, w, pre in zip(members, orcs, ws, pres):
            errs = finish_epoch(m, o, w.t_obs[k], w.y_obs[k], pre, exempt_dead=True)
            assert errs["x"] <= 1e-10, (w.name, w.lmm, k, errs["x"])


def test_many_members_parameter_blocks_built_in_parallel(pf):
    """With 128 or more members holding an observation the batch builds their
    parameter blocks on worker threads: 150 members (linear and Robertson,
    ragged N, uneven observation times, one member idle every other epoch and
    one invalid observation) are bit-identical to the same filters alone."""
    ws = []
    for i in range(150):
        name = "linear2" if i % 2 else "robertson"
        ws.append(W.get(name, N=64 + 37 * (i % 9), T=4, seed=100 + i))
    alone = [pf.Filter.from_workload(w) for w in ws]
    members = [pf.Filter.from_workload(w) for w in ws]
    batch = pf.Batch(members)
    for k in range(4):
        ts = [w.t_obs[k] for w in ws]
        ys = [w.y_obs[k] for w in ws]
        idle = 7 if k % 2 else None
        if idle is not None:
            ys[idle] = None
        bad = 11 if k == 2 else None
        if bad is not None:
            ys[bad] = np.full_like(ws[bad].y_obs[k], np.nan)
        st = batch.pf_batch_assimilate(ts, ys)
        for i, (a, w) in enumerate(zip(alone, ws)):
            if i == idle:
                assert st[i] == pf.PF_OK
                continue
            if i == bad:
                assert st[i] == pf.PF_ERR_INVALID_ARG
                continue
            assert st[i] == pf.PF_OK, (i, st[i])
            a.pf_assimilate(w.t_obs[k], w.y_obs[k])
        for a, m in zip(alone, members):
            assert _same(a, m)
            assert a.pf_get_history() == m.pf_get_history()
    batch.close()
