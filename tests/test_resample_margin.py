"""The arithmetic behind the resampling search's fast comparisons (no GPU).

Each test tau_i < c_k is first decided from the estimate fma(i, s, u s), with
s = c_{N-1} / N and u s rounded, and falls back to the exact
tau_i = ((i + u) / N) c_{N-1} only within 64 bit patterns of c_k.  That is
sound if the estimate and tau_i, both normal, never differ by more than a few
bit patterns: each lies within a few roundings of the real (i + u) c_{N-1} / N.
Here that claim is checked directly, with the fused multiply-add modelled by
exact rational arithmetic and a single rounding to double.
"""
import math
import struct
from fractions import Fraction

import numpy as np

MARGIN = 64     # kRsUlps
CLAIM = 6       # the bound the comment derives (three + two roundings)


def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _fma(a, b, c):
    # one rounding of the exact a * b + c (Fraction -> float rounds to nearest)
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _tau(i, u, n, total):
    return (float(i) + u) / float(n) * total


def _estimate(i, u, n, total):
    s = total / float(n)
    return _fma(float(i), s, u * s)


def test_estimate_within_claimed_patterns_of_tau():
    rng = np.random.default_rng(1411)
    worst = 0
    for _ in range(20000):
        n = int(rng.integers(1, 1 << 31))
        i = int(rng.integers(0, n))
        u = float(rng.random())
        total = float(rng.random()) * 10.0 ** int(rng.integers(-3, 12)) + 1e-300
        t, e = _tau(i, u, n, total), _estimate(i, u, n, total)
        if t < 2.0 ** -1000 or e < 2.0 ** -1000:
            continue  # the kernel decides tiny estimates exactly
        worst = max(worst, abs(_bits(t) - _bits(e)))
    assert worst <= CLAIM < MARGIN, worst


def test_adversarial_corners():
    # u at the top of [0, 1), the largest N, totals at binade edges
    for n in (1, 2, 3, 1023, (1 << 31) - 1):
        for u in (0.0, 2.0 ** -53, 0.5, 1.0 - 2.0 ** -53):
            for total in (1.0, 2.0 - 2.0 ** -52, 2.0 ** 40, math.nextafter(2.0 ** 20, 0.0), 3.0e-290):
                for i in (0, 1, n // 2, n - 1):
                    t, e = _tau(i, u, n, total), _estimate(i, u, n, total)
                    if t < 2.0 ** -1000 or e < 2.0 ** -1000:
                        continue
                    assert abs(_bits(t) - _bits(e)) <= CLAIM, (n, u, total, i)
