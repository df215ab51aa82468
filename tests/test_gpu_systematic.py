"""The filter's systematic search (Algorithm 1, Step 3b) on given cumulative
weights, against the oracle's, index for index.

pf_systematic_indices launches the same merge-path kernel body as
pf_assimilate.  Its comparisons are first decided from an estimate of each
tau_i and fall back to the exact tau_i only for near ties, so the cases here
put cumulative weights exactly on, and one ulp either side of, the tau_i;
they also cover runs of zero weights (equal c), leading and trailing zeros
(a tau past every c), a single heavy particle, u at both ends of [0, 1), tiny
totals, tile edges of the 1024-item merge tiles and a ragged tail.
"""
import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import build as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    B.build()
    oracle.build()
    from paper_1411_1702_gb300 import pf
    pf.load()
    return pf, torch


def _gpu(pf, torch, c, u):
    N = len(c)
    d_c = torch.tensor(c, dtype=torch.float64, device="cuda")
    d_idx = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    pf.pf_systematic_indices(d_c.data_ptr(), N, u, d_idx.data_ptr(), stream or None)
    torch.cuda.synchronize()
    return d_idx.cpu().numpy()


def _taus(N, u, total):
    # the definition, element by element in FP64 (numpy rounds each operation)
    i = np.arange(N, dtype=np.float64)
    return (i + u) / float(N) * total


def _cases():
    rng = np.random.default_rng(1411)
    out = []
    for N in (1, 2, 3, 511, 512, 513, 1023, 1024, 1025, 4097, 20011):
        g = rng.random(N)
        out.append((f"uniform-{N}", np.cumsum(g), float(rng.random())))
    N = 6007
    g = rng.random(N)
    g[rng.random(N) < 0.8] = 0.0
    g[0] = 1.0
    out.append(("sparse", np.cumsum(g), 0.37))
    g = rng.random(N)
    g[: N // 3] = 0.0
    out.append(("leading-zeros", np.cumsum(g), 0.91))
    g = rng.random(N)
    g[-N // 3:] = 0.0
    out.append(("trailing-zeros", np.cumsum(g), 1.0 - 2.0 ** -53))
    g = np.zeros(N)
    g[N // 2] = 1.0
    out.append(("one-heavy", np.cumsum(g), 0.0))
    g = rng.random(N) ** 40
    out.append(("skewed", np.cumsum(g), 0.5))
    out.append(("u-zero", np.cumsum(rng.random(N)), 0.0))
    out.append(("u-max", np.cumsum(rng.random(N)), 1.0 - 2.0 ** -53))
    out.append(("tiny-total", np.cumsum(rng.random(N)) * 1e-305, 0.25))
    out.append(("all-zero", np.zeros(777), 0.5))
    # cumulative weights on the resampling points themselves, and one ulp off
    for name, shift in (("on-tau", 0), ("ulp-below", -1), ("ulp-above", 1)):
        N = 3001
        u = float(rng.random())
        c = np.cumsum(rng.random(N))
        tau = _taus(N, u, c[-1])
        pick = np.sort(rng.choice(N - 1, size=N // 2, replace=False))
        c[pick] = tau[pick]
        if shift:
            c[pick] = np.nextafter(c[pick], np.inf if shift > 0 else -np.inf)
        c = np.maximum.accumulate(c)
        out.append((name, c, u))
    return out


CASES = _cases()


@pytest.mark.parametrize("name,c,u", CASES, ids=[x[0] for x in CASES])
def test_indices_equal_oracle(env, name, c, u):
    pf, torch = env
    c = np.ascontiguousarray(c, dtype=np.float64)
    assert np.all(np.diff(c) >= 0.0) and c[0] >= 0.0
    got = _gpu(pf, torch, c, u)
    want = oracle.resample_systematic(c, u)
    np.testing.assert_array_equal(got, want, err_msg=name)


def test_near_ties_are_exercised():
    # the on-tau cases really place c_k == tau_k (so the exact fallback decides)
    name, c, u = [x for x in CASES if x[0] == "on-tau"][0]
    tau = _taus(len(c), u, c[-1])
    assert np.count_nonzero(c[:-1] == tau[:-1]) > len(c) // 4


def test_full_size_random(env):
    # Robertson's ensemble size and one of 2^22, compared whole
    pf, torch = env
    rng = np.random.default_rng(7)
    for N in (131072, 1 << 22):
        lg = -0.5 * (rng.standard_normal(N) * 6.0) ** 2
        c = np.cumsum(np.exp(lg - lg.max()))
        u = float(rng.random())
        np.testing.assert_array_equal(_gpu(pf, torch, c, u), oracle.resample_systematic(c, u))


def test_same_as_filter_on_its_own_weights(env):
    # real epochs of a Robertson filter: from the filter's cumulative weights
    # and the epoch's u (Philox purpose RESAMPLE, slot 0), the stand-alone
    # call gives the filter's indices
    pf, torch = env
    from paper_1411_1702_gb300 import workloads as W
    w = W.robertson(N=3000, T=3)
    g = pf.Filter.from_workload(w)
    for k in range(w.T):
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
        work = g.pf_get_work()
        u = oracle.uniform(w.seed, 0, oracle.RNG_RESAMPLE, 0, k, 0)
        np.testing.assert_array_equal(_gpu(pf, torch, work["c"], u), work["idx"])
    g.close()


def test_two_phase_paths_equal_oracle(env):
    # above one wave of merge tiles (N > 4 * 152 * 512) the filter and the
    # allocation-free call find every tile corner in a launch of their own;
    # their indices must equal the oracle's and the one-launch form's
    pf, torch = env
    rng = np.random.default_rng(23)
    N = (1 << 20) + 4099
    lg = -0.5 * (rng.standard_normal(N) * 4.0) ** 2
    lg[rng.random(N) < 0.3] = -np.inf
    u = float(rng.random())
    d_lg = torch.tensor(lg, dtype=torch.float64, device="cuda")
    d_c = torch.empty(N, dtype=torch.float64, device="cuda")
    d_idx = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    pf.pf_resample_systematic_noalloc(d_lg.data_ptr(), N, u, d_c.data_ptr(), d_idx.data_ptr(),
                                      stream or None)
    torch.cuda.synchronize()
    c = d_c.cpu().numpy()
    idx = d_idx.cpu().numpy()
    np.testing.assert_array_equal(idx, oracle.resample_systematic(c, u))
    np.testing.assert_array_equal(idx, _gpu(pf, torch, c, u))


@pytest.mark.parametrize("N", [311296, 311297, 400000])
def test_filter_two_phase_resampling_equals_oracle(env, N):
    # Robertson filters on both sides of the two-launch threshold (2N items in
    # more than 4 * 152 tiles of 1024: N > 311296) and beyond it
    pf, torch = env
    from paper_1411_1702_gb300 import workloads as W
    w = W.robertson(N=N, T=2)
    g = pf.Filter.from_workload(w)
    for k in range(w.T):
        g.pf_assimilate(w.t_obs[k], w.y_obs[k])
        work = g.pf_get_work()
        u = oracle.uniform(w.seed, 0, oracle.RNG_RESAMPLE, 0, k, 0)
        np.testing.assert_array_equal(work["idx"], oracle.resample_systematic(work["c"], u))
        assert g.pf_stats()["unique_parents"] == len(np.unique(work["idx"]))
    g.close()


def test_first_stage_ess_matches_the_log_weights(env):
    # pf_stats' ess_stage1 is (sum g)^2 / sum g^2 of the epoch's first-stage
    # weights g = exp(lg - max lg); here from the filter's own lg
    pf, torch = env
    from paper_1411_1702_gb300 import workloads as W
    for name, N in (("robertson", 5000), ("brusselator", 300)):
        w = W.get(name, N=N)
        g = pf.Filter.from_workload(w)
        assert g.pf_stats()["ess_stage1"] == 0.0
        for k in range(3):
            g.pf_assimilate(w.t_obs[k], w.y_obs[k])
            lg = g.pf_get_work()["lg"]
            fin = np.isfinite(lg)
            e = np.exp(lg[fin] - lg[fin].max())
            want = e.sum() ** 2 / (e * e).sum()
            assert 1.0 <= want <= N
            assert g.pf_stats()["ess_stage1"] == pytest.approx(want, rel=1e-12)
        g.close()
