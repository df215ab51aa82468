"""Host-side arithmetic of bench.py's JSON line (no GPU): the launch count it
claims and the support kernels' bandwidth figures."""
import re
from pathlib import Path

import pytest

import bench
from paper_1411_1702_gb300 import workloads as W

ROOT = Path(__file__).resolve().parents[1]


def _cuh_int(name):
    text = (ROOT / "paper_1411_1702_gb300" / "csrc" / "pf_scan.cuh").read_text()
    m = re.search(rf"constexpr int {name} = ([^;]+);", text)
    return m.group(1)


def test_launch_count_follows_the_two_phase_threshold():
    # the library switches to a separate corner launch above 4 merge tiles of
    # kResampleThreads * kRsItems = 1024 items for each SM (608 on a GB300)
    assert _cuh_int("kRsTwoPhaseTilesPerSm") == "4"
    assert _cuh_int("kResampleThreads") == "256" and _cuh_int("kRsItems") == "4"
    w = W.robertson(N=8, T=2)
    for sms in (152, 148, 160):
        edge = 4 * sms * 1024 // 2           # 2N items fill exactly 4 tiles an SM
        assert bench.epoch_launches(w.with_(N=edge), sms) == 5
        assert bench.epoch_launches(w.with_(N=edge + 1), sms) == 6
    assert bench.epoch_launches(W.advdiff20(N=16, T=2), 152) == 6   # + the state mean


def test_support_roofline_arithmetic():
    # 2 ms over 4 launches of resampling at N = 1e6: 12 MB per 0.5 ms
    kt = {"resample": (2.0, 4), "scan_tile": (1.0, 4), "scan_add": (0.0, 4)}
    out = bench.support_roofline(kt, 1_000_000)
    r = out["kernels"]["resample"]
    assert r["us"] == pytest.approx(500.0)
    assert r["achieved"] == pytest.approx(12e6 / 500e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / out["peak"])
    assert out["kernels"]["scan_tile"]["achieved"] == pytest.approx(16e6 / 250e-6 / 1e9)
    assert "scan_add" not in out["kernels"]          # no pass of its own
    assert out["bound"] == "hbm" and out["unit"] == "GB/s"


def test_serving_trace_lengths_and_dilation():
    # sessions carry their problem's T observations by default
    tr = W.serving(n_sessions=12, seed=5)
    for ss in tr:
        assert len(ss.obs_s) == {W.LINEAR2: 50, W.ROBERTSON: 40, W.BRUSSELATOR: 30}[ss.w.ode]
        assert ss.w.T == len(ss.obs_s)
    # the load sweep dilates time: the same sessions, every arrival scaled by D
    a = W.serving(n_sessions=6, obs_per_session=4, seed=1)
    D = 7.5
    b = W.serving(n_sessions=6, obs_per_session=4, seed=1, rate_hz=200.0 / D, mean_gap_ms=5.0 * D)
    for sa, sb in zip(a, b):
        assert (sa.w.ode, sa.w.N) == (sb.w.ode, sb.w.N)
        assert sb.open_s == pytest.approx(D * sa.open_s, rel=1e-12)
        assert sb.obs_s == pytest.approx(D * sa.obs_s, rel=1e-12)
    assert bench.trace_span(b) == pytest.approx(D * bench.trace_span(a), rel=1e-12)
    assert bench.trace_steps(a) == bench.trace_steps(b) == sum(
        ss.w.particle_steps(k) for ss in a for k in range(4))


def test_percentile_rule():
    lat = list(range(1, 101))
    assert bench._pct(lat, 0.5) == 50 and bench._pct(lat, 0.99) == 99
    assert bench._pct([3.0], 0.99) == 3.0


@pytest.mark.gpu
def test_fp64_fma_probe_reaches_the_nominal_peak():
    """The benchmark's FMA probe (its own library, outside the sampler's C
    ABI) sustains close to the FP64 rate the roofline divides by (2 FMA lanes
    per clock per SM at the maximum clock, 1.259 TFLOP/s on a 152-SM GB300):
    between half and 110 % of it."""
    from paper_1411_1702_gb300 import build as B
    B.build()
    r = bench.fp64_fma_rate(50.0, None)
    assert r is not None and 0.5 * 1.259 < r < 1.1 * 1.259, r
    assert bench.fp64_fma_rate(0.0, None) is None
