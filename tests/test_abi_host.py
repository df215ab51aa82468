"""CPU tests of the C-ABI library: it builds, loads, exports every symbol that
include/pf.h declares, rejects bad arguments before touching the GPU, and its
host-side substep grid matches the oracle's (no GPU compute here)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import build as B
from paper_1411_1702_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pf():
    B.build()
    from paper_1411_1702_gb300 import pf as _pf
    _pf.load()
    return _pf


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \*]*?\b(pf_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(pf):
    declared = _declared_functions()
    assert len(declared) >= 15
    lib = C.CDLL(pf.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(pf.ABI_SYMBOLS)


def test_version(pf):
    assert "sm_103a" in pf.pf_version()


def _create(pf, **over):
    w = W.robertson(N=8, T=2)
    args = dict(ode=w.ode, d=w.d, p=w.p, N=8, lmm=w.lmm, dt=w.dt, prior_kind=w.prior_kind,
                prior_lo=w.prior_lo, prior_hi=w.prior_hi, x0=w.x0, t0=w.t0)
    kw = dict(a=w.a, newton_iters=w.newton_iters, spacing=w.spacing, substeps=w.substeps, q0=w.q0,
              history=w.history, transform=w.transform, obs_idx=w.obs_idx, noise=w.noise,
              sigma=w.sigma, kappa=w.kappa, seed=0)
    for k, v in over.items():
        if k in args:
            args[k] = v
        else:
            kw[k] = v
    return pf.Filter(*args.values(), **kw)


@pytest.mark.parametrize("bad", [
    dict(d=4), dict(p=2), dict(N=0), dict(ode=9), dict(lmm=4), dict(lmm=14), dict(lmm=3),
    dict(lmm=12), dict(a=0.0), dict(a=1.5),
    dict(newton_iters=0), dict(obs_idx=[5]), dict(sigma=[0.0, 0.01]), dict(substeps=0),
    dict(substeps=100000), dict(prior_lo=[-1.0, 1.0, 1.0]), dict(kappa=-1.0), dict(spacing=7),
    dict(timing=3), dict(timing=-1),
])
def test_invalid_arguments_rejected_before_gpu(pf, bad):
    with pytest.raises(pf.PfError) as ei:
        _create(pf, **bad)
    assert ei.value.status == pf.PF_ERR_INVALID_ARG


@pytest.mark.parametrize("bad", [
    dict(c=0), dict(idx=0), dict(N=0), dict(N=-3), dict(N=1 << 31), dict(u=1.0), dict(u=-0.5),
    dict(u=float("nan")),
])
def test_systematic_indices_rejects_arguments_before_gpu(pf, bad):
    # the checks come before any launch, so the (never dereferenced) buffer
    # addresses may be placeholders
    a = dict(c=0x1000, N=16, u=0.5, idx=0x2000)
    a.update(bad)
    with pytest.raises(pf.PfError) as ei:
        pf.pf_systematic_indices(a["c"], a["N"], a["u"], a["idx"])
    assert ei.value.status == pf.PF_ERR_INVALID_ARG


def test_device_bytes_cover_the_ensembles(pf):
    w = W.robertson(N=8, T=2)
    a = pf.pf_device_bytes(w.ode, w.d, w.p, 1000)
    b = pf.pf_device_bytes(w.ode, w.d, w.p, 2000)
    # two ping-pong copies of x, h1, h2 (d each), phi (p) and w, at least
    assert a >= 8 * 1000 * 2 * (3 * w.d + w.p + 1)
    assert b > a
    for bad in (dict(ode=9), dict(d=0), dict(p=0), dict(p=6), dict(N=0)):
        args = dict(ode=w.ode, d=w.d, p=w.p, N=1000)
        args.update(bad)
        with pytest.raises(pf.PfError) as ei:
            pf.pf_device_bytes(**args)
        assert ei.value.status == pf.PF_ERR_INVALID_ARG


@pytest.mark.parametrize("case", ["null", "misaligned", "small"])
def test_create_with_buffers_rejects_memory_before_gpu(pf, case):
    # the buffer checks come before any device work, so the (never touched)
    # addresses may be placeholders
    w = W.robertson(N=64, T=2)
    need = pf.pf_device_bytes(w.ode, w.d, w.p, 64)
    buf = {"null": (0, need), "misaligned": (0x100080, need), "small": (0x100000, need - 1)}[case]
    with pytest.raises(pf.PfError) as ei:
        pf.Filter.from_workload(w, N=64, device_buffer=buf)
    assert ei.value.status == pf.PF_ERR_INVALID_ARG


def _compare_tables(w, t_prev, t_next, depth, h1, h2, pf):
    cfg = oracle.make_config(w)
    tab, S, dout = oracle.build_substeps(cfg, t_prev, t_next, depth, h1, h2)
    coef, gdout = pf.pf_substep_table(w.lmm, w.spacing, w.dt, w.substeps, w.q0, t_prev, t_next,
                                      depth, h1, h2)
    assert coef.shape[0] == S and gdout == dout
    o = oracle.substep_dicts(tab, S)
    for i in range(S):
        assert coef[i, 0] == o[i]["kind"]
        assert coef[i, 1] == o[i]["h"]  # the same grid formula gives the same steps
        if o[i]["kind"] > 10:
            # Adams: the library packs the AM weights of f_n, f_{n-1} into
            # rho1, rho2 and the AB weights into pi0..pi2
            want = dict(gamma=o[i]["gamma"], rho1=o[i]["beta"][1], rho2=o[i]["beta"][2],
                        pi0=o[i]["bab"][0], pi1=o[i]["bab"][1], pi2=o[i]["bab"][2], mu=o[i]["mu"],
                        rho3=0.0, pi3=0.0)
        else:
            want = o[i]
        keys = ["gamma", "rho1", "rho2", "pi0", "pi1", "pi2", "mu", "rho3", "pi3"]
        for j, key in enumerate(keys, start=2):
            assert coef[i, j] == pytest.approx(want[key], rel=1e-12, abs=1e-15), (i, key)
    return coef


def test_substep_table_matches_oracle(pf):
    lw = W.linear2(N=4, T=3)
    _compare_tables(lw, 0.0, 0.1, 0, 0.0, 0.0, pf)
    _compare_tables(lw, 0.1, 0.2, 2, 0.005, 0.005, pf)
    _compare_tables(lw, 0.1, 0.2, 2, 0.001, 0.001, pf)        # ratio >= 2: cold start
    _compare_tables(lw.with_(lmm=1), 0.1, 0.2, 2, 0.005, 0.005, pf)
    rw = W.robertson(N=4, T=40)
    t = rw.t_obs
    _compare_tables(rw, 0.0, t[0], 0, 0.0, 0.0, pf)
    coef0, _ = pf.pf_substep_table(rw.lmm, rw.spacing, rw.dt, rw.substeps, rw.q0, 0.0, t[0], 0, 0, 0)
    _compare_tables(rw, t[0], t[1], 2, coef0[-1, 1], coef0[-2, 1], pf)
    _compare_tables(rw, t[20], t[21], 2, 0.3, 0.29, pf)
    bw = W.brusselator(N=4, T=3)
    _compare_tables(bw, 1.0 / 3.0, 2.0 / 3.0, 2, 1.0 / 60.0, 1.0 / 60.0, pf)


@pytest.mark.parametrize("lmm", [3, 11, 12, 13, 21, 22, 23])
def test_substep_table_other_lmms_match_oracle(pf, lmm):
    """BDF3 and the Adams methods: the library's textbook weights against the
    oracle's weights derived from Lagrange polynomials, cold start (the order
    ramp) and carried history."""
    mw = W.michaelis(N=4, T=2, lmm=lmm)
    _compare_tables(mw, 0.0, 0.5, 0, 0.0, 0.0, pf)
    _compare_tables(mw, 0.5, 1.0, 2, 0.05, 0.05, pf)
    _compare_tables(mw, 0.5, 1.0, 1, 0.05, 0.05, pf)
    lw = W.linear2(N=4, T=3).with_(lmm=lmm)
    _compare_tables(lw, 0.1, 0.2, 2, 0.005, 0.005, pf)
    # uniform spacing only
    with pytest.raises(ValueError):
        pf.pf_substep_table(lmm, 1, 0.0, 50, 1.01, 1e-4, 2e-4, 2, 1e-6, 1e-6)


def test_substep_table_rejects_bad_intervals(pf):
    with pytest.raises(ValueError):
        pf.pf_substep_table(2, 0, 0.005, 0, 0.0, 0.1, 0.1013, 2, 0.005, 0.005)
    with pytest.raises(ValueError):
        pf.pf_substep_table(2, 0, 0.005, 0, 0.0, 0.2, 0.1, 2, 0.005, 0.005)
    with pytest.raises(ValueError):
        pf.pf_substep_table(2, 1, 0.0, 50, 0.0, 0.0, 1e-4, 0, 0.0, 0.0)   # q0 missing


def test_substep_coefficients_constant_step(pf):
    coef, _ = pf.pf_substep_table(2, 0, 0.01, 0, 0.0, 1.0, 1.1, 2, 0.01, 0.01)
    assert np.allclose(coef[:, 3], 4.0 / 3.0, rtol=1e-12)
    assert np.allclose(coef[:, 4], -1.0 / 3.0, rtol=1e-12)
    assert np.allclose(coef[:, 2], 2.0 / 3.0 * 0.01, rtol=1e-9)
    assert np.allclose(coef[:, 8], -2.0 / 11.0, rtol=1e-9)
