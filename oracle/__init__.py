"""CPU oracle of the LMM PF-SMC sampler (Algorithm 1 of Arnold, Calvetti,
Somersalo, "Vectorized and Parallel Particle Filter SMC Parameter Estimation
for Stiff ODEs").

TEST INFRASTRUCTURE ONLY.  The oracle is the plain FP64 C restatement of the
method in ``pf_oracle.c``; this module compiles it with gcc and wraps it with
ctypes.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_HDR = os.path.join(_HERE, "pf_oracle.h")
_LIB = os.path.join(_HERE, "liboracle.so")
_OPC_SRC = os.path.join(_HERE, "opcount.cpp")
_OPC_LIB = os.path.join(_HERE, "libopcount.so")
_opc = None
_lock = threading.Lock()
_lib = None

DMAX, PMAX, MMAX, SMAX = 2025, 8, 32, 4096
LINEAR2, ROBERTSON, BRUSSELATOR, ADVDIFF, MICHAELIS = 1, 2, 3, 4, 5
LMM_BDF1, LMM_BDF2, LMM_BDF3 = 1, 2, 3
LMM_AM1, LMM_AM2, LMM_AM3 = 11, 12, 13
LMM_AB1, LMM_AB2, LMM_AB3 = 21, 22, 23
RNG_INIT, RNG_THETA, RNG_INNOV, RNG_RESAMPLE = 1, 2, 3, 4
UNIFORM, LOGUNIFORM = 0, 1
SPACING_UNIFORM, SPACING_GEOMETRIC = 0, 1
HIST_CARRY, HIST_RESTART = 0, 1
TRANSFORM_LOG, TRANSFORM_IDENTITY = 0, 1
NOISE_ADDITIVE, NOISE_RELATIVE = 0, 1
OK, ERR_ARG, ERR_DEGENERATE = 0, 1, 5


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP64, no contraction, OpenMP)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or any(
            os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off",
                   "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB)
        # the op-counting build of the same source (opcount.cpp)
        stale = (not os.path.exists(_OPC_LIB)) or any(
            os.path.getmtime(s) > os.path.getmtime(_OPC_LIB) for s in (_SRC, _HDR, _OPC_SRC))
        if force or stale:
            tmp = _OPC_LIB + f".tmp{os.getpid()}"
            cmd = ["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                   "-shared", "-o", tmp, _OPC_SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _OPC_LIB)
    return _LIB


class Config(C.Structure):
    _fields_ = [
        ("ode", C.c_int), ("d", C.c_int), ("p", C.c_int), ("m", C.c_int),
        ("N", C.c_int64),
        ("lmm", C.c_int), ("newton_iters", C.c_int), ("spacing", C.c_int),
        ("dt", C.c_double), ("substeps", C.c_int), ("q0", C.c_double),
        ("history", C.c_int), ("transform", C.c_int),
        ("obs_idx", C.c_int * MMAX), ("noise", C.c_int), ("sigma", C.c_double * MMAX),
        ("a", C.c_double), ("kappa", C.c_double), ("seed", C.c_uint64), ("stream", C.c_uint32),
        ("prior_kind", C.c_int * PMAX), ("prior_lo", C.c_double * PMAX),
        ("prior_hi", C.c_double * PMAX), ("x0", C.c_double * DMAX), ("t0", C.c_double),
        ("slot0", C.c_uint32),
    ]


class Substep(C.Structure):
    _fields_ = [("kind", C.c_int), ("h", C.c_double), ("gamma", C.c_double),
                ("rho1", C.c_double), ("rho2", C.c_double), ("pi0", C.c_double),
                ("pi1", C.c_double), ("pi2", C.c_double), ("mu", C.c_double),
                ("rho3", C.c_double), ("pi3", C.c_double), ("beta", C.c_double * 3),
                ("bab", C.c_double * 3), ("tn", C.c_double), ("t", C.c_double)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        sig = {
            "or_philox4x32_10": (None, [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
            "or_uniform": (C.c_double, [C.c_uint64, C.c_uint32, C.c_int, C.c_uint32, C.c_uint32, C.c_int]),
            "or_normal": (C.c_double, [C.c_uint64, C.c_uint32, C.c_int, C.c_uint32, C.c_uint32, C.c_int]),
            "or_ode_f": (None, [C.c_int, C.c_int, _dp, C.c_double, _dp, _dp]),
            "or_mm_constants": (None, [_dp]),
            "or_mm_input": (C.c_double, [C.c_double]),
            "or_lmm_coefficients": (C.c_int, [C.c_int, C.c_double, C.POINTER(Substep)]),
            "or_ode_jac": (None, [C.c_int, C.c_int, _dp, _dp, _dp]),
            "or_ode_dims": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "or_ode_check_dim": (C.c_int, [C.c_int, C.c_int]),
            "or_lu_solve": (C.c_int, [C.c_int, _dp, _dp, _dp]),
            "or_lu_factor": (C.c_int, [C.c_int, _dp, C.POINTER(C.c_int)]),
            "or_lu_apply": (None, [C.c_int, _dp, C.POINTER(C.c_int), _dp, _dp]),
            "or_bdf_coefficients": (C.c_int, [C.c_int, C.c_double, C.c_double, C.c_double, C.POINTER(Substep)]),
            "or_build_substeps": (C.c_int, [C.POINTER(Config), C.c_double, C.c_double, C.c_int, C.c_double,
                                            C.c_double, C.POINTER(Substep), C.c_int, C.POINTER(C.c_int)]),
            "or_propagate": (C.c_int, [C.c_int, C.c_int, C.c_int, _dp, C.POINTER(Substep), C.c_int, _dp, _dp,
                                       _dp, _dp]),
            "or_loglik": (C.c_double, [C.POINTER(Config), _dp, _dp]),
            "or_resample_systematic": (None, [C.c_int64, _dp, C.c_double, _ip]),
            "or_cholesky_psd": (None, [C.c_int, _dp, _dp]),
            "or_liu_west_shrink": (None, [C.c_int, C.c_double, _dp, _dp, _dp]),
            "or_create": (C.c_void_p, [C.POINTER(Config)]),
            "or_destroy": (None, [C.c_void_p]),
            "or_init": (C.c_int, [C.c_void_p]),
            "or_epoch": (C.c_int, [C.c_void_p, C.c_double, _dp]),
            "or_epoch_substeps": (C.c_int, [C.c_void_p, C.c_double, C.POINTER(Substep), C.c_int]),
            "or_stage1": (C.c_int, [C.c_void_p, C.POINTER(Substep), C.c_int, _dp]),
            "or_cumulative": (C.c_int, [C.c_void_p]),
            "or_resample_u": (C.c_double, [C.c_void_p]),
            "or_stage2": (C.c_int, [C.c_void_p, C.POINTER(Substep), C.c_int, _dp, _ip]),
            "or_commit": (C.c_int, [C.c_void_p, C.c_double]),
            "or_get_state": (None, [C.c_void_p, _dp, _dp, _dp, _dp, _dp]),
            "or_set_state": (None, [C.c_void_p, _dp, _dp, _dp, _dp, _dp]),
            "or_get_moments": (None, [C.c_void_p, _dp, _dp, _dp, _dp]),
            "or_set_moments": (None, [C.c_void_p, _dp, _dp]),
            "or_get_work": (None, [C.c_void_p, _dp, _dp, _dp, _ip]),
            "or_get_history": (None, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), _dp, _dp, _dp]),
            "or_set_history": (None, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]),
            "or_shard_init": (C.c_int, [C.c_void_p]),
            "or_get_pending_lw": (None, [C.c_void_p, _dp]),
            "or_set_ll1": (None, [C.c_void_p, _dp]),
            "or_shard_nsums": (C.c_int, [C.c_void_p]),
            "or_shard_sums": (None, [C.c_void_p, C.c_int, C.c_double, _dp]),
            "or_shard_commit": (C.c_int, [C.c_void_p, C.c_int, C.c_double, _dp, C.c_double]),
            "or_threads": (C.c_int, []),
            "or_set_threads": (None, [C.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_ip) if a is not None else None


# ---------------------------------------------------------------- primitives
def philox(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def uniform(seed, stream, purpose, n, epoch, k):
    return lib().or_uniform(seed, stream, purpose, n, epoch, k)


def normal(seed, stream, purpose, n, epoch, k):
    return lib().or_normal(seed, stream, purpose, n, epoch, k)


def ode_dims(ode):
    d, p = C.c_int(), C.c_int()
    if lib().or_ode_dims(ode, C.byref(d), C.byref(p)) != 0:
        raise ValueError(ode)
    return d.value, p.value


def ode_check_dim(ode, d):
    return lib().or_ode_check_dim(ode, int(d)) == 0


def ode_f(ode, theta, x, t=0.0):
    xx = np.ascontiguousarray(x, dtype=np.float64)
    d = len(xx)
    if not ode_check_dim(ode, d):
        raise ValueError((ode, d))
    th = np.ascontiguousarray(theta, dtype=np.float64)
    f = np.zeros(d)
    lib().or_ode_f(ode, d, _d(th), float(t), _d(xx), _d(f))
    return f


def mm_constants():
    """M1's known constants (lambda, c0, A0, A, t0, tau) as the oracle reads them."""
    out = np.zeros(6)
    lib().or_mm_constants(_d(out))
    return dict(zip(("lam", "c0", "A0", "A", "t0", "tau"), out.tolist()))


def mm_input(t):
    return lib().or_mm_input(float(t))


def ode_jac(ode, theta, x):
    xx = np.ascontiguousarray(x, dtype=np.float64)
    d = len(xx)
    if not ode_check_dim(ode, d):
        raise ValueError((ode, d))
    th = np.ascontiguousarray(theta, dtype=np.float64)
    J = np.zeros((d, d))
    lib().or_ode_jac(ode, d, _d(th), _d(xx), _d(J))
    return J


def lu_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(len(b))
    if lib().or_lu_solve(len(b), _d(A), _d(b), _d(x)) != 0:
        raise np.linalg.LinAlgError("singular")
    return x


def lu_factor_solve(A, bs):
    """Factor A once (or_lu_factor) and solve for each right-hand side."""
    LU = np.array(A, dtype=np.float64, order="C")
    n = LU.shape[0]
    piv = (C.c_int * n)()
    if lib().or_lu_factor(n, _d(LU), piv) != 0:
        raise np.linalg.LinAlgError("singular")
    out = []
    for b in bs:
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(n)
        lib().or_lu_apply(n, _d(LU), piv, _d(b), _d(x))
        out.append(x)
    return out


def bdf_coefficients(kind, h0, h1=0.0, h2=0.0):
    s = Substep()
    if lib().or_bdf_coefficients(kind, h0, h1, h2, C.byref(s)) != 0:
        raise ValueError(kind)
    return s


def lmm_coefficients(kind, h):
    s = Substep()
    if lib().or_lmm_coefficients(kind, h, C.byref(s)) != 0:
        raise ValueError(kind)
    return s


def substep_dicts(tab, S):
    return [dict(kind=tab[i].kind, h=tab[i].h, gamma=tab[i].gamma, rho1=tab[i].rho1,
                 rho2=tab[i].rho2, pi0=tab[i].pi0, pi1=tab[i].pi1, pi2=tab[i].pi2,
                 mu=tab[i].mu, rho3=tab[i].rho3, pi3=tab[i].pi3, beta=list(tab[i].beta),
                 bab=list(tab[i].bab), tn=tab[i].tn, t=tab[i].t) for i in range(S)]


def build_substeps(cfg: Config, t_prev, t_next, depth, hprev1, hprev2):
    tab = (Substep * SMAX)()
    dout = C.c_int()
    S = lib().or_build_substeps(C.byref(cfg), t_prev, t_next, depth, hprev1, hprev2, tab, SMAX,
                                C.byref(dout))
    if S < 1:
        raise ValueError("bad interval")
    return tab, S, dout.value


def propagate(ode, K, theta, tab, S, x, h1, h2, with_error=False):
    """One particle over S substeps; returns (x, h1, h2, E or None)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.array(x, dtype=np.float64)
    h1 = np.array(h1, dtype=np.float64)
    h2 = np.array(h2, dtype=np.float64)
    E = np.zeros(len(x)) if with_error else None
    rc = lib().or_propagate(ode, len(x), K, _d(th), tab, S, _d(x), _d(h1), _d(h2), _d(E))
    if rc != 0:
        raise np.linalg.LinAlgError("singular Newton matrix")
    return x, h1, h2, E


def count_propagate(ode, K, theta, tab, S, x, h1, h2, with_error=False):
    """Exact operation counts of or_propagate over the S substeps of tab for
    one particle (opcount.cpp): additions/subtractions, multiplications,
    divisions, square roots, elementary functions, and the propagated state."""
    global _opc
    if _opc is None:
        build()
        L = C.CDLL(_OPC_LIB)
        L.or_count_propagate.restype = C.c_int
        L.or_count_propagate.argtypes = [C.c_int, C.c_int, C.c_int, _dp, C.POINTER(Substep), C.c_int,
                                         _dp, _dp, _dp, C.c_int, C.POINTER(C.c_longlong), _dp]
        _opc = L
    th = np.ascontiguousarray(theta, dtype=np.float64)
    x, h1, h2 = (np.ascontiguousarray(v, dtype=np.float64) for v in (x, h1, h2))
    out = (C.c_longlong * 5)()
    xo = np.zeros(len(x))
    rc = _opc.or_count_propagate(ode, len(x), K, _d(th), tab, S, _d(x), _d(h1), _d(h2),
                                 1 if with_error else 0, out, _d(xo))
    if rc != 0:
        raise np.linalg.LinAlgError("singular Newton matrix")
    return dict(add=out[0], mul=out[1], div=out[2], sqrt=out[3], elem=out[4], x=xo)


def loglik(cfg: Config, y, x):
    """Step 3a / Step 5 log-likelihood log pi(y | x) of one state (or_loglik)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    return lib().or_loglik(C.byref(cfg), _d(y), _d(x))


def resample_systematic(c, u):
    c = np.ascontiguousarray(c, dtype=np.float64)
    idx = np.zeros(len(c), dtype=np.int32)
    lib().or_resample_systematic(len(c), _d(c), float(u), _i(idx))
    return idx


def cholesky_psd(Cm):
    Cm = np.ascontiguousarray(Cm, dtype=np.float64)
    p = Cm.shape[0]
    L = np.zeros((p, p))
    lib().or_cholesky_psd(p, _d(Cm), _d(L))
    return L


def liu_west_shrink(a, phi, phibar):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    phibar = np.ascontiguousarray(phibar, dtype=np.float64)
    out = np.zeros_like(phi)
    lib().or_liu_west_shrink(len(phi), float(a), _d(phi), _d(phibar), _d(out))
    return out


def threads():
    return lib().or_threads()


def set_threads(n):
    lib().or_set_threads(int(n))


# -------------------------------------------------------------------- filter
def make_config(w) -> Config:
    """Oracle config from a workload description (paper_1411_1702_gb300.workloads)."""
    c = Config()
    c.ode, c.d, c.p, c.m, c.N = w.ode, w.d, w.p, len(w.obs_idx), w.N
    c.lmm, c.newton_iters = w.lmm, w.newton_iters
    c.spacing, c.dt, c.substeps, c.q0 = w.spacing, w.dt, w.substeps, w.q0
    c.history, c.transform = w.history, w.transform
    for i, o in enumerate(w.obs_idx):
        c.obs_idx[i] = int(o)
        c.sigma[i] = float(w.sigma[i])
    c.noise = w.noise
    c.a, c.kappa, c.seed, c.stream = w.a, w.kappa, w.seed, w.stream
    for i in range(w.p):
        c.prior_kind[i] = int(w.prior_kind[i])
        c.prior_lo[i] = float(w.prior_lo[i])
        c.prior_hi[i] = float(w.prior_hi[i])
    for i in range(w.d):
        c.x0[i] = float(w.x0[i])
    c.t0 = w.t0
    return c


class Filter:
    """Algorithm 1 on the CPU, one epoch per observation."""

    def __init__(self, workload, N=None, slot0=0):
        w = workload
        self.cfg = make_config(w)
        if N is not None:
            self.cfg.N = int(N)
        self.cfg.slot0 = int(slot0)
        self.N, self.d, self.p, self.m = self.cfg.N, w.d, w.p, len(w.obs_idx)
        self._h = lib().or_create(C.byref(self.cfg))
        if not self._h:
            raise ValueError("oracle rejected the configuration")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_destroy(h)
            self._h = None

    def init(self):
        return lib().or_init(self._h)

    def epoch(self, t, y):
        y = np.ascontiguousarray(y, dtype=np.float64)
        return lib().or_epoch(self._h, float(t), _d(y))

    # stage-level access ----------------------------------------------------
    def substeps(self, t):
        tab = (Substep * SMAX)()
        S = lib().or_epoch_substeps(self._h, float(t), tab, SMAX)
        if S < 1:
            raise ValueError("bad interval")
        return tab, S

    def stage1(self, tab, S, y):
        y = np.ascontiguousarray(y, dtype=np.float64)
        return lib().or_stage1(self._h, tab, S, _d(y))

    def cumulative(self):
        return lib().or_cumulative(self._h)

    def resample_u(self):
        return lib().or_resample_u(self._h)

    def stage2(self, tab, S, y, idx):
        y = np.ascontiguousarray(y, dtype=np.float64)
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        return lib().or_stage2(self._h, tab, S, _d(y), _i(idx))

    def commit(self, t):
        return lib().or_commit(self._h, float(t))

    def state(self):
        N, d, p = self.N, self.d, self.p
        x, h1, h2 = np.zeros((N, d)), np.zeros((N, d)), np.zeros((N, d))
        phi, lw = np.zeros((N, p)), np.zeros(N)
        lib().or_get_state(self._h, _d(x), _d(h1), _d(h2), _d(phi), _d(lw))
        return dict(x=x, h1=h1, h2=h2, phi=phi, lw=lw)

    def set_state(self, x=None, h1=None, h2=None, phi=None, lw=None):
        def a(v):
            return None if v is None else np.ascontiguousarray(v, dtype=np.float64)
        x, h1, h2, phi, lw = a(x), a(h1), a(h2), a(phi), a(lw)
        lib().or_set_state(self._h, _d(x), _d(h1), _d(h2), _d(phi), _d(lw))

    def moments(self):
        p, d = self.p, self.d
        pb, Cm, xb, ess = np.zeros(p), np.zeros((p, p)), np.zeros(d), C.c_double()
        lib().or_get_moments(self._h, _d(pb), _d(Cm), _d(xb), C.byref(ess))
        return dict(phibar=pb, C=Cm, xbar=xb, ess=ess.value)

    def set_moments(self, phibar, Cm):
        pb = np.ascontiguousarray(phibar, dtype=np.float64)
        Cm = np.ascontiguousarray(Cm, dtype=np.float64)
        lib().or_set_moments(self._h, _d(pb), _d(Cm))

    def work(self):
        N = self.N
        ll1, lg, c = np.zeros(N), np.zeros(N), np.zeros(N)
        idx = np.zeros(N, dtype=np.int32)
        lib().or_get_work(self._h, _d(ll1), _d(lg), _d(c), _i(idx))
        return dict(ll1=ll1, lg=lg, c=c, idx=idx)

    # a shard of a particle-sharded filter (cfg.slot0 = its first global slot)
    def shard_init(self):
        return lib().or_shard_init(self._h)

    def pending_lw(self):
        out = np.zeros(self.N)
        lib().or_get_pending_lw(self._h, _d(out))
        return out

    def set_ll1(self, ll1):
        lib().or_set_ll1(self._h, _d(np.ascontiguousarray(ll1, dtype=np.float64)))

    def shard_sums(self, pending, M):
        out = np.zeros(lib().or_shard_nsums(self._h))
        lib().or_shard_sums(self._h, int(pending), float(M), _d(out))
        return out

    def shard_commit(self, pending, M, sums, t_next=0.0):
        sums = np.ascontiguousarray(sums, dtype=np.float64)
        return lib().or_shard_commit(self._h, int(pending), float(M), _d(sums), float(t_next))

    def history(self):
        e, dp = C.c_int(), C.c_int()
        t, h1, h2 = C.c_double(), C.c_double(), C.c_double()
        lib().or_get_history(self._h, C.byref(e), C.byref(dp), C.byref(t), C.byref(h1), C.byref(h2))
        return dict(epoch=e.value, depth=dp.value, t_prev=t.value, hprev1=h1.value, hprev2=h2.value)

    def set_history(self, epoch, depth, t_prev, hprev1, hprev2):
        lib().or_set_history(self._h, int(epoch), int(depth), float(t_prev), float(hprev1), float(hprev2))
