"""The allocation-free resampling call against the filter's own resampling.

pf_resample_systematic_noalloc serves callers that cannot allocate device
memory where they resample (a pool allocator that owns all device memory, a
latency-critical loop that cannot afford cudaMalloc's device-wide
synchronisation, a step that must not fail with out-of-memory).  It keeps its
scratch in a fixed array inside the library.  This test hands it the log
fitness weights of real filter epochs -- in buffers the test owns -- and checks
that its cumulative weights and indices equal what pf_assimilate produced,
on consecutive calls (the shared scratch must not leak state between calls).
"""
import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import build as B
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


def _noalloc(pf, torch, lg, u):
    N = len(lg)
    d_lg = torch.tensor(lg, dtype=torch.float64, device="cuda")
    d_c = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
    d_idx = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    pf.pf_resample_systematic_noalloc(d_lg.data_ptr(), N, u, d_c.data_ptr(), d_idx.data_ptr(),
                                      stream or None)
    torch.cuda.synchronize()
    return d_c.cpu().numpy(), d_idx.cpu().numpy()


@pytest.mark.parametrize("N", [5003, 1, 131072])
def test_noalloc_matches_filter_on_consecutive_calls(env, N):
    pf, torch = env
    w = W.robertson(N=N, T=3)
    g = pf.Filter.from_workload(w)
    for k in range(2):
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
        work = g.pf_get_work()
        u = oracle.uniform(w.seed, 0, oracle.RNG_RESAMPLE, 0, k, 0)
        c, idx = _noalloc(pf, torch, work["lg"], u)
        assert np.array_equal(idx, work["idx"]), f"indices differ at call {k}"
        assert np.array_equal(c, work["c"]), f"cumulative weights differ at call {k}"
    g.close()


def test_noalloc_rejects_oversized_and_bad_arguments(env):
    pf, torch = env
    d = torch.zeros(4, dtype=torch.float64, device="cuda")
    i = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(pf.PfError) as ei:
        pf.pf_resample_systematic_noalloc(d.data_ptr(), pf.NOALLOC_MAX_PARTICLES + 1, 0.5,
                                          d.data_ptr(), i.data_ptr())
    assert ei.value.status == pf.PF_ERR_BUDGET
    with pytest.raises(pf.PfError) as ei:
        pf.pf_resample_systematic_noalloc(d.data_ptr(), 4, 1.0, d.data_ptr(), i.data_ptr())
    assert ei.value.status == pf.PF_ERR_INVALID_ARG


def test_noalloc_zero_and_nonfinite_weights(env):
    # every weight zero: c is all zero and every index is 0; NaN and +inf
    # log weights count as zero weights, like -inf
    pf, torch = env
    for N in (1, 700, 70000):
        c, idx = _noalloc(pf, torch, np.full(N, -np.inf), 0.5)
        assert np.all(c == 0.0) and np.all(idx == 0)
    rng = np.random.default_rng(11)
    N = 9000
    lg = rng.standard_normal(N) * 3.0
    bad = rng.choice(N, size=N // 10, replace=False)
    lg[bad] = rng.choice([np.nan, np.inf, -np.inf], size=len(bad))
    u = 0.3
    c, idx = _noalloc(pf, torch, lg, u)
    fin = np.isfinite(lg)
    g = np.where(fin, np.exp(np.where(fin, lg, 0.0) - np.max(lg[fin])), 0.0)
    assert np.allclose(c, np.cumsum(g), rtol=1e-12, atol=0.0)
    assert np.all(np.diff(c) >= 0.0)
    assert np.array_equal(idx, oracle.resample_systematic(c, u))
    assert not np.any(np.isin(idx, np.flatnonzero(~fin)))


def test_noalloc_at_its_maximum_size(env):
    """N = PF_NOALLOC_MAX_PARTICLES (2^24): the scratch layout's largest
    case, two calls in a row, indices against the oracle's systematic search
    on the call's own cumulative weights."""
    pf, torch = env
    N = pf.NOALLOC_MAX_PARTICLES
    rng = np.random.default_rng(24)
    lg = rng.standard_normal(N) * 2.0
    lg[rng.random(N) < 0.05] = -np.inf
    for u in (0.37, 0.0):
        c, idx = _noalloc(pf, torch, lg, u)
        assert np.all(np.diff(c) >= 0.0)
        assert np.array_equal(idx, oracle.resample_systematic(c, u))
        fin = np.isfinite(lg)
        g = np.where(fin, np.exp(np.where(fin, lg, 0.0) - np.max(lg[fin])), 0.0)
        ref = np.cumsum(g)
        assert np.allclose(c, ref, rtol=1e-11, atol=1e-11 * ref[-1])
