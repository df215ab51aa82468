"""Checkpoint and resume through the C ABI (pf_checkpoint_size, pf_save,
pf_load): the random streams are counter-based, so a filter restored from a
checkpoint continues bit-identically to one that was never interrupted."""
import numpy as np
import pytest

from paper_1411_1702_gb300 import build as B
from paper_1411_1702_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    B.build()
    from paper_1411_1702_gb300 import pf as _pf
    _pf.load()
    return _pf


def _snapshot(g):
    st = g.pf_get_ensemble()
    tb, Cm, xb = g.pf_estimates()
    s = g.pf_stats()
    return st, (tb, Cm, xb), s, g.pf_get_history()


def _same(a, b):
    (sa, ea, ta, ha), (sb, eb, tb_, hb) = a, b
    for k in sa:
        assert np.array_equal(sa[k], sb[k]), k
    for u, v in zip(ea, eb):
        assert np.array_equal(u, v)
    assert ha == hb
    for k in ("epochs", "ess", "log_weight_sum", "unique_parents", "nonfinite"):
        assert ta[k] == tb_[k], k


@pytest.mark.parametrize("name,N,lmm", [("robertson", 4096, None), ("michaelis", 3001, W.LMM_AM3),
                                        ("linear2", 1029, W.LMM_BDF3), ("brusselator", 513, None),
                                        ("advdiff20", 300, None)])
def test_resume_is_bit_identical(pf, name, N, lmm):
    w = W.get(name, N=N)
    if lmm is not None:
        w = w.with_(lmm=lmm)
    k0, k1 = 5, 10
    a = pf.Filter.from_workload(w)
    for k in range(k0):
        a.pf_assimilate(w.t_obs[k], w.y_obs[k])
    blob = a.pf_save()
    for k in range(k0, k1):
        a.pf_assimilate(w.t_obs[k], w.y_obs[k])
    # a fresh filter of the same configuration, advanced elsewhere first
    b = pf.Filter.from_workload(w)
    b.pf_assimilate(w.t_obs[0], w.y_obs[0])
    b.pf_load(blob)
    assert b.pf_get_history()["epoch"] == k0
    for k in range(k0, k1):
        b.pf_assimilate(w.t_obs[k], w.y_obs[k])
    _same(_snapshot(a), _snapshot(b))


def test_resume_with_device_series(pf):
    w = W.robertson(N=2048, T=12)
    a = pf.Filter.from_workload(w)
    a.pf_load_observations(w.t_obs, w.y_obs)
    a.pf_run(0, 4)
    a.pf_synchronize()
    blob = a.pf_save()
    a.pf_run(4, 12)
    a.pf_synchronize()
    b = pf.Filter.from_workload(w)
    b.pf_load(blob)
    b.pf_load_observations(w.t_obs[4:], w.y_obs[4:])
    b.pf_run(0, 8)
    b.pf_synchronize()
    _same(_snapshot(a), _snapshot(b))


def test_checkpoint_rejects_a_different_filter(pf):
    w = W.linear2(N=256, T=3)
    a = pf.Filter.from_workload(w)
    a.pf_assimilate(w.t_obs[0], w.y_obs[0])
    blob = a.pf_save()
    for other in (pf.Filter.from_workload(w, N=255), pf.Filter.from_workload(w, seed=7),
                  pf.Filter.from_workload(w.with_(lmm=W.LMM_AM2)),
                  pf.Filter.from_workload(W.robertson(N=256, T=2))):
        with pytest.raises(pf.PfError) as ei:
            other.pf_load(blob)
        assert ei.value.status == pf.PF_ERR_INVALID_ARG
    b = pf.Filter.from_workload(w)
    for bad in (blob[:100], blob[:-8], b"x" * len(blob)):
        with pytest.raises(pf.PfError) as ei:
            b.pf_load(bad)
        assert ei.value.status == pf.PF_ERR_INVALID_ARG
    # the failed loads left b untouched: it still runs from its own start
    c = pf.Filter.from_workload(w)
    b.pf_assimilate(w.t_obs[0], w.y_obs[0])
    c.pf_assimilate(w.t_obs[0], w.y_obs[0])
    _same(_snapshot(b), _snapshot(c))


@pytest.mark.parametrize("name", ["robertson", "brusselator", "advdiff20"])
def test_estimates_after_assimilate_equal_a_device_read(pf, name):
    # pf_estimates right after pf_assimilate is served from the values that
    # pf_assimilate's own wait brought back; after any call that may change the
    # device state it reads the device again.  Both must give the same bits,
    # and the mirror must not survive a state change.
    w = W.get(name, N=600 if name != "advdiff20" else 64)
    g = pf.Filter.from_workload(w)
    for k in range(3):
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
        fast = g.pf_estimates()
        blob = g.pf_save()
        g.pf_load(blob)  # the same state, and the mirror is dropped
        slow = g.pf_estimates()
        for u, v in zip(fast, slow):
            assert np.array_equal(u, v)
    # a state change after the mirror was filled is seen
    before = g.pf_estimates()
    phibar, Cm, _ = before
    g.pf_set_moments(phibar + 0.25, Cm)
    after = g.pf_estimates()
    assert np.array_equal(after[0], phibar + 0.25)
    g.close()
