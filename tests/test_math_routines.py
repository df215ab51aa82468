"""The table-driven logarithm and sine/cosine of the Box-Muller transform
(csrc/pf_math.cuh): a host build against mpmath at 40 digits (CPU), and the
device build against the host build, bit for bit (GPU)."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1411_1702_gb300", "csrc")
SHIM = os.path.join(ROOT, "tests", "math_shim.cpp")

TWO53 = 1 << 53


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("mathshim") / "libmath_shim.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                    "-shared", "-I", CSRC, SHIM, "-o", out], check=True)
    L = C.CDLL(out)
    L.shim_log.argtypes = [C.c_void_p, C.c_void_p, C.c_long]
    L.shim_sincospi.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_long]
    return L


def host_log(L, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    L.shim_log(x.ctypes.data, y.ctypes.data, len(x))
    return y


def host_sincospi(L, k):
    k = np.ascontiguousarray(k, dtype=np.uint64)
    s, c = np.empty(len(k)), np.empty(len(k))
    L.shim_sincospi(k.ctypes.data, s.ctypes.data, c.ctypes.data, len(k))
    return s, c


def log_inputs(rng, n):
    """The Box-Muller arguments 1 - u1 = m 2^-53, m in [1, 2^53], plus the
    table's breakpoints and their neighbours, powers of two and 1."""
    m = rng.integers(1, TWO53 + 1, n, dtype=np.uint64)
    x = [float(v) * 2.0 ** -53 for v in m]
    for j in range(129):
        F = 1.0 + j / 128.0
        for s in (0.5, 0.25, 2.0 ** -10, 2.0 ** -40):
            for f in (F, np.nextafter(F, 0.0), np.nextafter(F, 4.0), F + 1.0 / 256.0 - 2.0 ** -52):
                x.append(f * s)
    x += [1.0, np.nextafter(1.0, 0.0), 2.0 ** -53, 0.5, np.nextafter(0.5, 0.0), 0.75]
    return np.array(x)


def trig_inputs(rng, n):
    """k of the Box-Muller angle pi k 2^-52, k < 2^53: random, and around
    every table point j/64 (k = j 2^46) and every rounding boundary between two."""
    k = list(rng.integers(0, TWO53, n, dtype=np.uint64))
    for j in range(129):
        for d in (-(1 << 45), -(1 << 45) + 1, -1, 0, 1, (1 << 45) - 1, 1 << 45):
            v = j * (1 << 46) + d
            if 0 <= v < TWO53:
                k.append(v)
    k += [0, 1, TWO53 - 1]
    return np.array(k, dtype=np.uint64)


def ulp(v):
    return np.spacing(np.abs(v))


def test_log_within_two_ulps(shim):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(11)
    x = log_inputs(rng, 4000)
    y = host_log(shim, x)
    exact = np.array([float(mpmath.log(mpmath.mpf(v))) for v in x])
    err = np.abs(y - exact) / np.maximum(ulp(exact), 2.0 ** -1074)
    assert np.all(np.isfinite(y))
    # the table value, log 2 times e, the polynomial and two sums each round
    # once; below 1/2 the first sum cancels by up to a factor of about 1.5
    assert err.max() <= 2.0, (x[err.argmax()], err.max())
    assert np.mean(err) <= 0.5
    # exact where the logarithm is
    assert host_log(shim, np.array([1.0]))[0] == 0.0
    # and within a rounding or two of the C library's
    lib = np.log(x)
    assert np.max(np.abs(y - lib) / np.maximum(ulp(lib), 2.0 ** -1074)) <= 2.0


def test_sincospi_within_half_an_ulp_of_one(shim):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(12)
    k = trig_inputs(rng, 4000)
    s, c = host_sincospi(shim, k)
    ang = [mpmath.pi * mpmath.mpf(int(v)) / mpmath.mpf(1 << 52) for v in k]
    es = np.array([float(mpmath.sin(a)) for a in ang])
    ec = np.array([float(mpmath.cos(a)) for a in ang])
    # absolute error against the exact values, in units of 2^-53 (half an ulp of 1)
    assert np.max(np.abs(s - es)) <= 2.0 ** -53
    assert np.max(np.abs(c - ec)) <= 2.0 ** -53
    # relative accuracy away from the zeros: the table value, the polynomial
    # and the combining FMA each round once
    big = np.abs(es) > 2.0 ** -4
    assert np.max(np.abs(s - es)[big] / ulp(es[big])) <= 2.0
    big = np.abs(ec) > 2.0 ** -4
    assert np.max(np.abs(c - ec)[big] / ulp(ec[big])) <= 2.0
    # the identities the transform relies on
    assert np.max(np.abs(s * s + c * c - 1.0)) <= 4.0 * 2.0 ** -53
    assert host_sincospi(shim, np.array([0], dtype=np.uint64)) == (np.array([0.0]), np.array([1.0]))


def test_box_muller_radius_and_angle_match_the_library(shim):
    """The normals of one Philox block as the kernels form them, against the
    same formula with the C library's log, cos and sin (the oracle's)."""
    rng = np.random.default_rng(13)
    k1 = rng.integers(0, TWO53, 5000, dtype=np.uint64)
    k2 = rng.integers(0, TWO53, 5000, dtype=np.uint64)
    v = (TWO53 - k1).astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * host_log(shim, v))
    s, c = host_sincospi(shim, k2)
    u2 = k2.astype(np.float64) * 2.0 ** -53
    r_lib = np.sqrt(-2.0 * np.log(1.0 - k1.astype(np.float64) * 2.0 ** -53))
    a = 2.0 * np.pi * u2
    assert np.max(np.abs(r * c - r_lib * np.cos(a))) <= 1e-14
    assert np.max(np.abs(r * s - r_lib * np.sin(a))) <= 1e-14


@pytest.mark.gpu
def test_device_build_is_bit_identical_to_host_build(shim):
    import torch
    from paper_1411_1702_gb300 import build as B
    B.build()
    P = C.CDLL(B.PROBE_LIB)
    P.pf_probe_math.argtypes = [C.c_void_p] * 2 + [C.c_int64] + [C.c_void_p] * 3
    P.pf_probe_math.restype = C.c_int
    rng = np.random.default_rng(14)
    x = log_inputs(rng, 1 << 16)
    k = trig_inputs(rng, len(x))[:len(x)]
    n = min(len(x), len(k))
    x, k = x[:n], k[:n]
    assert np.all(x > 2.0 ** -1022) and np.all(np.isfinite(x)) and np.all(k < TWO53)
    dx = torch.from_numpy(x).cuda()
    dk = torch.from_numpy(k.view(np.int64)).cuda()
    lg, s, c = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    assert P.pf_probe_math(dx.data_ptr(), dk.data_ptr(), n, lg.data_ptr(), s.data_ptr(),
                           c.data_ptr()) == 0
    hs, hc = host_sincospi(shim, k)
    assert np.array_equal(lg.cpu().numpy(), host_log(shim, x))
    assert np.array_equal(s.cpu().numpy(), hs)
    assert np.array_equal(c.cpu().numpy(), hc)
