"""Serving: sessions admitted by device-memory budget, continuous batching,
results identical to each filter alone, latency accounting."""
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


def _sessions():
    specs = [("robertson", 4096, 11), ("linear2", 2048, 12), ("brusselator", 64, 13),
             ("robertson", 1000, 14), ("linear2", 1, 15), ("robertson", 8192, 16)]
    return [W.get(name, N=N, T=4, seed=seed) for name, N, seed in specs]


def _sessions_lmm():
    """The paper's M1 system and the other LMM families among the sessions."""
    return [W.michaelis(N=4096, T=4, seed=21, lmm=W.LMM_AM3),
            W.michaelis(N=40000, T=4, seed=22, lmm=W.LMM_AB3),
            W.linear2(N=2048, T=4, seed=23).with_(lmm=W.LMM_BDF3),
            W.robertson(N=1000, T=4, seed=24),
            W.michaelis(N=512, T=4, seed=25, lmm=W.LMM_BDF2)]


def _same(a, b):
    ea, eb = a.pf_get_ensemble(), b.pf_get_ensemble()
    return all(np.array_equal(ea[k], eb[k], equal_nan=True) for k in ea)


@pytest.mark.parametrize("make", [_sessions, _sessions_lmm])
def test_sessions_match_alone_under_interleaved_arrivals(pf, make):
    ws = make()
    srv = pf.Server(budget_bytes=8 << 30)
    sids = [srv.pf_server_open(w, filter_id=i) for i, w in enumerate(ws)]
    rng = np.random.default_rng(3)
    nxt = [0] * len(ws)
    # observations arrive in a random interleaving; the server steps in between
    while any(k < 4 for k in nxt):
        i = int(rng.integers(len(ws)))
        if nxt[i] < 4:
            srv.pf_server_submit(sids[i], ws[i].t_obs[nxt[i]], ws[i].y_obs[nxt[i]])
            nxt[i] += 1
        if rng.random() < 0.5:
            srv.pf_server_step()
    srv.pf_server_drain()
    st = srv.pf_server_stats()
    assert st["assimilations"] == 4 * len(ws)
    assert 0.0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    for i, w in enumerate(ws):
        f, done, last = srv.pf_server_session(sids[i])
        assert done == 4 and last == pf.PF_OK
        alone = pf.Filter.from_workload(w, filter_id=i)
        for k in range(4):
            alone.pf_assimilate(w.t_obs[k], w.y_obs[k])
        assert _same(alone, f)


def _session_bytes(pf, w):
    probe = pf.Server(budget_bytes=1 << 40)
    probe.pf_server_open(w)
    probe.pf_server_step()
    b = probe.pf_server_stats()["device_bytes_in_use"]
    probe.close()
    return b


def test_admission_waits_for_memory(pf):
    ws = _sessions()[:3]
    big = W.robertson(N=200000, T=2, seed=21)
    b_big = _session_bytes(pf, big)
    b_rest = sum(_session_bytes(pf, w) for w in ws)
    # room for the big session or for the rest, not for the big one and the first
    budget = max(b_big, b_rest) + min(_session_bytes(pf, ws[0]), b_big) - 1
    assert b_big + _session_bytes(pf, ws[0]) > budget
    srv = pf.Server(budget_bytes=budget)
    sid_big = srv.pf_server_open(big)
    sids = [srv.pf_server_open(w) for w in ws]
    srv.pf_server_step()
    st = srv.pf_server_stats()
    assert st["admitted"] == 1 and st["waiting"] == 3
    assert st["device_bytes_in_use"] == b_big
    for k in range(2):
        srv.pf_server_submit(sid_big, big.t_obs[k], big.y_obs[k])
    for s, w in zip(sids, ws):
        srv.pf_server_submit(s, w.t_obs[0], w.y_obs[0])
    srv.pf_server_drain()
    assert srv.pf_server_stats()["waiting"] == 3      # still no room
    f, done, _ = srv.pf_server_session(sid_big)
    assert done == 2 and f is not None
    assert srv.pf_server_session(sids[0])[0] is None   # not admitted yet
    srv.pf_server_close(sid_big)                       # frees its memory
    srv.pf_server_drain()
    st = srv.pf_server_stats()
    assert st["waiting"] == 0 and st["assimilations"] == 2 + len(ws)
    assert st["device_bytes_in_use"] == b_rest <= st["budget_bytes"]
    for s, w in zip(sids, ws):
        f, done, _ = srv.pf_server_session(s)
        alone = pf.Filter.from_workload(w)
        alone.pf_assimilate(w.t_obs[0], w.y_obs[0])
        assert done == 1 and _same(alone, f)


def test_session_larger_than_budget_is_rejected(pf):
    srv = pf.Server(budget_bytes=1 << 20)
    with pytest.raises(pf.PfError) as ei:
        srv.pf_server_open(W.robertson(N=100000, T=1))
    assert ei.value.status == pf.PF_ERR_BUDGET
    assert srv.pf_server_stats()["rejected"] == 1


def test_served_sessions_match_oracle(pf):
    """Sessions of every problem and LMM family served together: after each
    round of observations (one per session, then a drain) every session is
    compared with the oracle run from its committed state, stage by stage.
    The session's random streams are those of its filter id."""
    ws = [w.with_(stream=i) for i, w in enumerate(_sessions() + _sessions_lmm())]
    srv = pf.Server(budget_bytes=8 << 30)
    sids = [srv.pf_server_open(w, filter_id=i) for i, w in enumerate(ws)]
    srv.pf_server_step()
    orcs = [oracle.Filter(w) for w in ws]
    for o in orcs:
        o.init()
    for k in range(4):
        views = [srv.pf_server_session(s)[0] for s in sids]
        assert all(v is not None for v in views)
        pres = [begin_epoch(v, o) for v, o in zip(views, orcs)]
        order = np.random.default_rng(k).permutation(len(ws))
        for i in order:
            srv.pf_server_submit(sids[i], ws[i].t_obs[k], ws[i].y_obs[k])
            srv.pf_server_step()
        srv.pf_server_drain()
        for i, (s, o, w, pre) in enumerate(zip(sids, orcs, ws, pres)):
            f, done, last = srv.pf_server_session(s)
            assert done == k + 1 and last == pf.PF_OK
            errs = finish_epoch(f, o, w.t_obs[k], w.y_obs[k], pre, exempt_dead=True, stats=False)
            assert errs["x"] <= 1e-10, (w.name, k, errs["x"])


def test_drain_passes_rejected_observations(pf):
    """Observations the epoch rejects (not finite) leave their queues without
    an epoch; draining steps on past them instead of waiting for a launch
    that never comes, and the valid observations of the other sessions are
    assimilated as usual."""
    ws = [W.linear2(N=512, T=4, seed=41), W.robertson(N=1000, T=4, seed=42)]
    srv = pf.Server(budget_bytes=2 << 30)
    sids = [srv.pf_server_open(w, filter_id=i) for i, w in enumerate(ws)]
    bad = np.full_like(ws[0].y_obs[0], np.nan)
    for k in range(3):
        srv.pf_server_submit(sids[0], ws[0].t_obs[k], bad)
    for k in range(2):
        srv.pf_server_submit(sids[1], ws[1].t_obs[k], ws[1].y_obs[k])
    srv.pf_server_drain()
    f0, done0, last0 = srv.pf_server_session(sids[0])
    f1, done1, last1 = srv.pf_server_session(sids[1])
    assert done0 == 0 and last0 == pf.PF_ERR_INVALID_ARG
    assert done1 == 2 and last1 == pf.PF_OK
    alone = pf.Filter.from_workload(ws[1], filter_id=1)
    for k in range(2):
        alone.pf_assimilate(ws[1].t_obs[k], ws[1].y_obs[k])
    assert _same(alone, f1)
    # the rejected session still takes valid observations afterwards
    srv.pf_server_submit(sids[0], ws[0].t_obs[0], ws[0].y_obs[0])
    srv.pf_server_drain()
    assert srv.pf_server_session(sids[0])[1] == 1
