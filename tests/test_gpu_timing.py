"""pf_options.timing and pf_kernel_times: events around every kernel (1) or
around stage 2 alone (2), and results that do not depend on either (the
kernels of an epoch are launched with programmatic dependent launch, which
events between them disable)."""
import numpy as np
import pytest

from paper_1411_1702_gb300 import build as B
from paper_1411_1702_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SLOTS = ["stage1", "scan_tile", "scan_add", "resample", "stage2", "moments"]


@pytest.fixture(scope="module")
def pf():
    B.build()
    from paper_1411_1702_gb300 import pf as _pf
    _pf.load()
    return _pf


def _run(pf, w, timing, epochs):
    f = pf.Filter.from_workload(w, timing=timing)
    f.pf_load_observations(w.t_obs, w.y_obs)
    f.pf_run(0, epochs)
    f.pf_synchronize()
    return f


@pytest.mark.parametrize("name,N", [("robertson", 4099), ("michaelis", 3000), ("linear2", 70000)])
def test_timing_levels_measure_their_kernels_and_change_nothing(pf, name, N):
    w = W.get(name, N=N, T=4)
    f0, f1, f2 = (_run(pf, w, t, 4) for t in (0, 1, 2))
    with pytest.raises(pf.PfError):
        f0.pf_kernel_times()
    k1, k2 = f1.pf_kernel_times(), f2.pf_kernel_times()
    for s in SLOTS:
        n1 = 0 if s == "scan_add" else 4
        assert k1[s][1] == n1 and (k1[s][0] > 0.0) == (n1 > 0), (s, k1[s])
        n2 = 4 if s == "stage2" else 0
        assert k2[s][1] == n2 and (k2[s][0] > 0.0) == (n2 > 0), (s, k2[s])
    # the accumulators were reset by the read
    assert all(v == (0.0, 0) for v in f2.pf_kernel_times().values())
    e = [f.pf_get_ensemble() for f in (f0, f1, f2)]
    for key in e[0]:
        assert np.array_equal(e[0][key], e[1][key]) and np.array_equal(e[0][key], e[2][key]), key
    est = [f.pf_estimates() for f in (f0, f1, f2)]
    for a, b in zip(est[0], est[1]):
        assert np.array_equal(a, b)
    for a, b in zip(est[0], est[2]):
        assert np.array_equal(a, b)
    for f in (f0, f1, f2):
        f.close()


def test_timing_level_out_of_range_is_rejected(pf):
    w = W.get("linear2", N=64, T=2)
    for bad in (3, -1):
        with pytest.raises(pf.PfError) as ei:
            pf.Filter.from_workload(w, timing=bad)
        assert ei.value.status == pf.PF_ERR_INVALID_ARG


def test_assimilate_graph_equals_direct_launches(pf):
    """pf_assimilate runs its epoch as one captured graph when timing is off
    (a few substep counts kept) and as separate calls with timing on: the
    same bits either way, across intervals of seven different lengths (more
    substep counts than the graphs kept, so some are captured again)."""
    w = W.get("linear2", N=3000, T=12)
    gaps = [0.05, 0.1, 0.02, 0.15, 0.05, 0.03, 0.2, 0.1, 0.04, 0.02, 0.05, 0.1]
    w = w.with_(t_obs=np.cumsum(gaps))
    fg, fd = pf.Filter.from_workload(w, timing=0), pf.Filter.from_workload(w, timing=1)
    for k in range(w.T):
        for f in (fg, fd):
            f.pf_assimilate(w.t_obs[k], w.y_obs[k])
        eg, ed = fg.pf_estimates(), fd.pf_estimates()
        for a, b in zip(eg, ed):
            assert np.array_equal(a, b), k
        sg, sd = fg.pf_stats(), fd.pf_stats()
        assert sg["epochs"] == sd["epochs"] == k + 1
        assert sg["h2d_bytes"] == sd["h2d_bytes"] and sg["d2h_bytes"] == sd["d2h_bytes"]
        assert sg["last_epoch_ms"] > 0.0
    e0, e1 = fg.pf_get_ensemble(), fd.pf_get_ensemble()
    for key in e0:
        assert np.array_equal(e0[key], e1[key]), key
    fg.close()
    fd.close()
