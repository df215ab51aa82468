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
    # the library switches to a separate corner launch above 4 * 152 merge
    # tiles of kResampleThreads * kRsItems = 1024 items
    assert _cuh_int("kRsTwoPhaseTiles").replace(" ", "") == "4*152"
    assert _cuh_int("kResampleThreads") == "256" and _cuh_int("kRsItems") == "4"
    w = W.robertson(N=8, T=2)
    edge = 4 * 152 * 1024 // 2           # 2N items fill exactly 608 tiles
    assert bench.epoch_launches(w.with_(N=edge)) == 5
    assert bench.epoch_launches(w.with_(N=edge + 1)) == 6
    assert bench.epoch_launches(W.advdiff20(N=16, T=2)) == 6   # + the state mean


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
