"""Thin ctypes binding of the C ABI in include/pf.h (libpf_gb300.so).

Argument marshalling only: every step of the sampler runs in the library's
CUDA kernels.  Importing this module loads the in-tree library and raises if
it is missing -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpf_gb300.so")

PF_OK, PF_ERR_INVALID_ARG, PF_ERR_OOM, PF_ERR_BUDGET, PF_ERR_CUDA = 0, 1, 2, 3, 4
PF_ERR_DEGENERATE, PF_ERR_NUMERIC, PF_ERR_TIMEOUT, PF_ERR_STATE = 5, 6, 7, 8
PF_ODE_LINEAR2, PF_ODE_ROBERTSON, PF_ODE_BRUSSELATOR1D, PF_ODE_ADVDIFF2D = 1, 2, 3, 4
PF_ODE_MICHAELIS3 = 5
PF_LMM_BDF1, PF_LMM_BDF2, PF_LMM_BDF3 = 1, 2, 3
PF_LMM_AM1, PF_LMM_AM2, PF_LMM_AM3 = 11, 12, 13
PF_LMM_AB1, PF_LMM_AB2, PF_LMM_AB3 = 21, 22, 23
PF_SUBSTEP_ROW = 11
MAX_SUBSTEPS = 640

STATUS_NAMES = {0: "PF_OK", 1: "PF_ERR_INVALID_ARG", 2: "PF_ERR_OOM", 3: "PF_ERR_BUDGET",
                4: "PF_ERR_CUDA", 5: "PF_ERR_DEGENERATE", 6: "PF_ERR_NUMERIC",
                7: "PF_ERR_TIMEOUT", 8: "PF_ERR_STATE"}

# every symbol declared in include/pf.h
ABI_SYMBOLS = [
    "pf_create", "pf_assimilate", "pf_estimates", "pf_stats", "pf_last_error", "pf_destroy",
    "pf_load_observations", "pf_run", "pf_synchronize", "pf_reset", "pf_get_ensemble",
    "pf_set_ensemble", "pf_set_moments", "pf_get_work", "pf_get_history", "pf_set_history",
    "pf_substep_table", "pf_version", "pf_kernel_times", "pf_resample_systematic_noalloc",
    "pf_systematic_indices", "pf_device_bytes", "pf_create_with_buffers",
    "pf_batch_create", "pf_batch_assimilate", "pf_batch_stats", "pf_batch_last_error",
    "pf_batch_destroy", "pf_server_create", "pf_server_open", "pf_server_submit",
    "pf_server_step", "pf_server_drain", "pf_server_close", "pf_server_session",
    "pf_server_stats", "pf_server_last_error", "pf_server_destroy", "pf_checkpoint_size",
    "pf_save", "pf_load", "pf_shard_tile", "pf_shard_create", "pf_shard_info", "pf_shard_stage1",
    "pf_shard_scan", "pf_shard_offsets", "pf_shard_resample", "pf_shard_stage2", "pf_shard_moments",
    "pf_shard_commit", "pf_shard_abort", "pf_shard_parents",
]
NOALLOC_MAX_PARTICLES = 1 << 24
KERNEL_SLOTS = ["stage1", "scan_tile", "scan_add", "resample", "stage2", "moments"]


class PfError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Prior(C.Structure):
    _fields_ = [("p", C.c_int), ("kind", C.POINTER(C.c_int)), ("lo", C.POINTER(C.c_double)),
                ("hi", C.POINTER(C.c_double)), ("d", C.c_int), ("x0", C.POINTER(C.c_double)),
                ("t0", C.c_double)]


class Options(C.Structure):
    _fields_ = [("a", C.c_double), ("newton_iters", C.c_int), ("spacing", C.c_int),
                ("substeps", C.c_int), ("q0", C.c_double), ("history", C.c_int),
                ("transform", C.c_int), ("m", C.c_int), ("obs_idx", C.POINTER(C.c_int)),
                ("noise", C.c_int), ("sigma", C.POINTER(C.c_double)), ("kappa", C.c_double),
                ("seed", C.c_uint64), ("filter_id", C.c_uint32), ("stream", C.c_void_p),
                ("timing", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("epochs", C.c_int64), ("ess", C.c_double), ("log_weight_sum", C.c_double),
                ("unique_parents", C.c_int64), ("nonfinite", C.c_int64),
                ("theta_mean", C.c_double * 8), ("last_epoch_ms", C.c_double),
                ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("ess_stage1", C.c_double)]


class BatchStats(C.Structure):
    _fields_ = [("epochs", C.c_int64), ("graph_captures", C.c_int64),
                ("last_device_ms", C.c_double), ("last_active", C.c_int), ("last_tiles", C.c_int),
                ("tile_order", C.c_int), ("concurrent_models", C.c_int), ("tune_ms", C.c_double * 4)]


class ServerStats(C.Structure):
    _fields_ = [("admitted", C.c_int64), ("rejected", C.c_int64), ("waiting", C.c_int64),
                ("active_sessions", C.c_int64), ("queued_observations", C.c_int64),
                ("assimilations", C.c_int64), ("epochs", C.c_int64),
                ("mean_sessions_per_epoch", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("mean_ms", C.c_double), ("max_ms", C.c_double),
                ("particle_steps_per_s", C.c_double), ("device_bytes_in_use", C.c_int64),
                ("budget_bytes", C.c_int64), ("step_calls", C.c_int64),
                ("step_ms_mean", C.c_double), ("step_ms_max", C.c_double),
                ("collect_ms_max", C.c_double), ("admit_ms_max", C.c_double),
                ("launch_ms_max", C.c_double)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_lib = None


def load(path: str = LIB_PATH):
    """Load libpf_gb300.so (build it first with paper_1411_1702_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build the CUDA library first "
                          "(python -m paper_1411_1702_gb300.build)")
    L = C.CDLL(path)
    sig = {
        "pf_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int, C.c_double,
                                C.POINTER(Prior), C.POINTER(Options), C.POINTER(C.c_void_p)]),
        "pf_device_bytes": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int64,
                                      C.POINTER(C.c_size_t)]),
        "pf_create_with_buffers": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int,
                                             C.c_double, C.POINTER(Prior), C.POINTER(Options),
                                             C.c_void_p, C.c_size_t, C.POINTER(C.c_void_p)]),
        # the per-epoch calls take plain addresses: building ctypes pointer
        # objects cost about as much host time as the calls themselves
        "pf_assimilate": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p]),
        "pf_estimates": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
        "pf_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
        "pf_last_error": (C.c_char_p, [C.c_void_p]),
        "pf_destroy": (None, [C.c_void_p]),
        "pf_load_observations": (C.c_int, [C.c_void_p, C.c_int, _dp, _dp]),
        "pf_run": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
        "pf_synchronize": (C.c_int, [C.c_void_p]),
        "pf_reset": (C.c_int, [C.c_void_p]),
        "pf_get_ensemble": (C.c_int, [C.c_void_p, _dp, _dp, _dp, _dp, _dp]),
        "pf_set_ensemble": (C.c_int, [C.c_void_p, _dp, _dp, _dp, _dp, _dp]),
        "pf_set_moments": (C.c_int, [C.c_void_p, _dp, _dp]),
        "pf_get_work": (C.c_int, [C.c_void_p, _dp, _dp, _dp, _ip]),
        "pf_get_history": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int), _dp, _dp, _dp]),
        "pf_set_history": (C.c_int, [C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_double, C.c_double]),
        "pf_checkpoint_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t)]),
        "pf_save": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
        "pf_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
        "pf_substep_table": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_int, C.c_double, C.c_double,
                                       C.c_double, C.c_int, C.c_double, C.c_double, _dp, C.c_int,
                                       C.POINTER(C.c_int)]),
        "pf_version": (C.c_char_p, []),
        "pf_kernel_times": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64), C.c_int]),
        "pf_resample_systematic_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                                                     C.c_void_p, C.c_void_p]),
        "pf_systematic_indices": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                                            C.c_void_p]),
        "pf_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
        "pf_batch_assimilate": (C.c_int, [C.c_void_p, _dp, C.POINTER(_dp), C.POINTER(C.c_int)]),
        "pf_batch_stats": (C.c_int, [C.c_void_p, C.POINTER(BatchStats)]),
        "pf_batch_last_error": (C.c_char_p, [C.c_void_p]),
        "pf_batch_destroy": (None, [C.c_void_p]),
        "pf_server_create": (C.c_int, [C.c_int64, C.c_int, C.POINTER(C.c_void_p)]),
        "pf_server_open": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int,
                                     C.c_double, C.POINTER(Prior), C.POINTER(Options),
                                     C.POINTER(C.c_int64)]),
        "pf_server_submit": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, _dp]),
        "pf_server_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int)]),
        "pf_server_drain": (C.c_int, [C.c_void_p]),
        "pf_server_close": (C.c_int, [C.c_void_p, C.c_int64]),
        "pf_server_session": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_void_p),
                                        C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
        "pf_server_stats": (C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
        "pf_server_last_error": (C.c_char_p, [C.c_void_p]),
        "pf_server_destroy": (None, [C.c_void_p]),
        "pf_shard_tile": (C.c_int64, [C.c_int64]),
        "pf_shard_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int64,
                                      C.c_int, C.c_double, C.POINTER(Prior), C.POINTER(Options),
                                      C.POINTER(C.c_void_p)]),
        "pf_shard_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "pf_shard_stage1": (C.c_int, [C.c_void_p, C.c_double, _dp, _dp]),
        "pf_shard_scan": (C.c_int, [C.c_void_p, C.c_double, _dp, _dp]),
        "pf_shard_offsets": (C.c_int, [C.c_void_p, _dp, C.c_double, _dp, _dp, _dp]),
        "pf_shard_resample": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_int64, C.c_double,
                                        C.c_double, C.c_void_p]),
        "pf_shard_stage2": (C.c_int, [C.c_void_p, C.c_void_p, _dp]),
        "pf_shard_moments": (C.c_int, [C.c_void_p, C.c_double, _dp, C.POINTER(C.c_int)]),
        "pf_shard_commit": (C.c_int, [C.c_void_p, _dp, C.c_int]),
        "pf_shard_abort": (C.c_int, [C.c_void_p]),
        "pf_shard_parents": (C.c_int, [C.c_void_p, _ip]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _d(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(st, handle=None):
    if st != PF_OK:
        msg = load().pf_last_error(handle)
        raise PfError(st, msg.decode() if msg else "")


def pf_version() -> str:
    return load().pf_version().decode()


def pf_resample_systematic_noalloc(log_g_ptr, N, u, cumulative_ptr, idx_ptr, stream=None):
    """Systematic resampling of caller-owned device buffers (raw device
    addresses) without any allocation; asynchronous on `stream`."""
    st = load().pf_resample_systematic_noalloc(C.c_void_p(log_g_ptr), int(N), float(u),
                                               C.c_void_p(cumulative_ptr), C.c_void_p(idx_ptr),
                                               C.c_void_p(stream) if stream else None)
    _check(st, None)


def pf_systematic_indices(cumulative_ptr, N, u, idx_ptr, stream=None):
    """Step 3b's systematic search alone on caller-owned device buffers (raw
    device addresses): the filter's own kernel; asynchronous on `stream`."""
    st = load().pf_systematic_indices(C.c_void_p(cumulative_ptr), int(N), float(u),
                                      C.c_void_p(idx_ptr), C.c_void_p(stream) if stream else None)
    _check(st, None)


def pf_device_bytes(ode, d, p, N):
    """Device bytes a filter of this shape lays out (pf_create_with_buffers)."""
    out = C.c_size_t()
    _check(load().pf_device_bytes(int(ode), int(d), int(p), int(N), C.byref(out)), None)
    return out.value


def pf_substep_table(lmm, spacing, dt, substeps, q0, t_prev, t_next, depth, hprev1, hprev2):
    """Host-only: the substep table of one interval, shape (S, PF_SUBSTEP_ROW):
    kind, h, gamma, rho1, rho2, pi0, pi1, pi2, mu, rho3, pi3."""
    coef = np.zeros((MAX_SUBSTEPS, PF_SUBSTEP_ROW))
    dout = C.c_int()
    S = load().pf_substep_table(lmm, spacing, dt, substeps, q0, t_prev, t_next, depth, hprev1,
                                hprev2, _d(coef), MAX_SUBSTEPS, C.byref(dout))
    if S < 1:
        raise ValueError("invalid interval")
    return coef[:S].copy(), dout.value


class Filter:
    """One LMM PF-SMC filter on the GPU (Algorithm 1), owned by the library."""

    def __init__(self, ode, d, p, N, lmm, dt, prior_kind, prior_lo, prior_hi, x0, t0, *,
                 a, newton_iters, spacing, substeps, q0, history, transform, obs_idx, noise,
                 sigma, kappa, seed, filter_id=0, stream=None, timing=False, device_buffer=None,
                 shard=None):
        L = load()
        self._keep = []
        kind = (C.c_int * len(prior_kind))(*[int(k) for k in prior_kind])
        lo, hi = _f64(prior_lo), _f64(prior_hi)
        x0a = _f64(x0)
        obs = (C.c_int * len(obs_idx))(*[int(o) for o in obs_idx])
        sig = _f64(sigma)
        self._keep += [kind, lo, hi, x0a, obs, sig]
        pr = Prior(p, kind, _d(lo), _d(hi), d, _d(x0a), float(t0))
        op = Options(float(a), int(newton_iters), int(spacing), int(substeps), float(q0),
                     int(history), int(transform), len(obs_idx), obs, int(noise), _d(sig),
                     float(kappa), int(seed), int(filter_id), C.c_void_p(stream) if stream else None,
                     int(timing))  # False/0 off, True/1 every kernel, 2 stage 2 only
        h = C.c_void_p()
        if shard is not None:
            # the slots [first, first + N) of a sharded filter of n_all particles
            n_all, first = shard
            st = L.pf_shard_create(int(ode), int(d), int(p), int(n_all), int(first), int(N),
                                   int(lmm), float(dt), C.byref(pr), C.byref(op), C.byref(h))
        elif device_buffer is None:
            st = L.pf_create(int(ode), int(d), int(p), int(N), int(lmm), float(dt), C.byref(pr),
                             C.byref(op), C.byref(h))
        else:
            # caller-owned device memory: (address, bytes), or an object with
            # data_ptr() and nbytes (a CUDA tensor), kept referenced here
            if hasattr(device_buffer, "data_ptr"):
                ptr, nbytes = device_buffer.data_ptr(), device_buffer.nbytes
            else:
                ptr, nbytes = device_buffer
            self._keep.append(device_buffer)
            st = L.pf_create_with_buffers(int(ode), int(d), int(p), int(N), int(lmm), float(dt),
                                          C.byref(pr), C.byref(op), C.c_void_p(int(ptr)),
                                          int(nbytes), C.byref(h))
        _check(st, None)
        self._h = h
        self.ode, self.d, self.p, self.N, self.m = ode, d, p, N, len(obs_idx)

    @classmethod
    def from_workload(cls, w, N=None, stream=None, seed=None, filter_id=0, timing=False,
                      device_buffer=None, shard=None):
        return cls(w.ode, w.d, w.p, int(N if N is not None else w.N), w.lmm, w.dt, w.prior_kind,
                   w.prior_lo, w.prior_hi, w.x0, w.t0, a=w.a, newton_iters=w.newton_iters,
                   spacing=w.spacing, substeps=w.substeps, q0=w.q0, history=w.history,
                   transform=w.transform, obs_idx=w.obs_idx, noise=w.noise, sigma=w.sigma,
                   kappa=w.kappa, seed=w.seed if seed is None else seed, filter_id=filter_id,
                   stream=stream, timing=timing, device_buffer=device_buffer, shard=shard)

    @classmethod
    def borrowed(cls, handle, ode, d, p, N, m):
        """View of a filter the library owns (e.g. a server session)."""
        obj = cls.__new__(cls)
        obj._h = C.c_void_p(handle)
        obj._owned = False
        obj._keep = []
        obj.ode, obj.d, obj.p, obj.N, obj.m = ode, d, p, N, m
        return obj

    def close(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None and getattr(self, "_owned", True):
            _lib.pf_destroy(h)
        self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- the calls of include/pf.h ---------------------------------------
    def pf_assimilate(self, t, y):
        y = _f64(y)
        if y.size < self.m:
            raise ValueError(f"need {self.m} observed values, got {y.size}")
        _check(load().pf_assimilate(self._h, float(t), y.ctypes.data), self._h)

    def pf_estimates(self):
        # one buffer, every entry written by the call, returned as three
        # disjoint views (theta-bar, C, x-bar)
        p, d = self.p, self.d
        buf = np.empty(p + p * p + d)
        a = buf.ctypes.data
        _check(load().pf_estimates(self._h, a, a + 8 * p, a + 8 * (p + p * p)), self._h)
        return buf[:p], buf[p:p + p * p].reshape(p, p), buf[p + p * p:]

    def pf_stats(self):
        s = Stats()
        _check(load().pf_stats(self._h, C.byref(s)), self._h)
        return dict(epochs=s.epochs, ess=s.ess, log_weight_sum=s.log_weight_sum,
                    unique_parents=s.unique_parents, nonfinite=s.nonfinite,
                    theta_mean=np.array(s.theta_mean[:self.p]), last_epoch_ms=s.last_epoch_ms,
                    h2d_bytes=s.h2d_bytes, d2h_bytes=s.d2h_bytes, ess_stage1=s.ess_stage1)

    def pf_kernel_times(self):
        """Per-kernel device ms and launch counts since the last call."""
        n = len(KERNEL_SLOTS)
        ms = np.zeros(n)
        cnt = (C.c_int64 * n)()
        _check(load().pf_kernel_times(self._h, _d(ms), cnt, n), self._h)
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_SLOTS)}

    def pf_load_observations(self, t, y):
        t, y = _f64(t), _f64(y).reshape(len(t), self.m)
        _check(load().pf_load_observations(self._h, len(t), _d(t), _d(y)), self._h)

    def pf_run(self, k0, k1):
        _check(load().pf_run(self._h, int(k0), int(k1)), self._h)

    def pf_synchronize(self):
        _check(load().pf_synchronize(self._h), self._h)

    def pf_reset(self):
        _check(load().pf_reset(self._h), self._h)

    def pf_get_ensemble(self):
        N, d, p = self.N, self.d, self.p
        x, h1, h2 = np.zeros((N, d)), np.zeros((N, d)), np.zeros((N, d))
        phi, lw = np.zeros((N, p)), np.zeros(N)
        _check(load().pf_get_ensemble(self._h, _d(x), _d(h1), _d(h2), _d(phi), _d(lw)), self._h)
        return dict(x=x, h1=h1, h2=h2, phi=phi, lw=lw)

    def pf_set_ensemble(self, x=None, h1=None, h2=None, phi=None, lw=None):
        a = [None if v is None else _f64(v) for v in (x, h1, h2, phi, lw)]
        _check(load().pf_set_ensemble(self._h, *[_d(v) for v in a]), self._h)

    def pf_set_moments(self, phibar, Cm):
        pb, Cm = _f64(phibar), _f64(Cm)
        _check(load().pf_set_moments(self._h, _d(pb), _d(Cm)), self._h)

    def pf_get_work(self):
        N = self.N
        ll1, lg, c = np.zeros(N), np.zeros(N), np.zeros(N)
        idx = np.zeros(N, dtype=np.int32)
        _check(load().pf_get_work(self._h, _d(ll1), _d(lg), _d(c), idx.ctypes.data_as(_ip)), self._h)
        return dict(ll1=ll1, lg=lg, c=c, idx=idx)

    def pf_get_history(self):
        e, dp = C.c_int64(), C.c_int()
        t, h1, h2 = C.c_double(), C.c_double(), C.c_double()
        _check(load().pf_get_history(self._h, C.byref(e), C.byref(dp), C.byref(t), C.byref(h1),
                                     C.byref(h2)), self._h)
        return dict(epoch=e.value, depth=dp.value, t_prev=t.value, hprev1=h1.value, hprev2=h2.value)

    def pf_set_history(self, epoch, depth, t_prev, hprev1, hprev2):
        _check(load().pf_set_history(self._h, int(epoch), int(depth), float(t_prev), float(hprev1),
                                     float(hprev2)), self._h)

    def pf_save(self) -> bytes:
        """Checkpoint of the committed state (pf_checkpoint_size + pf_save)."""
        n = C.c_size_t()
        _check(load().pf_checkpoint_size(self._h, C.byref(n)), self._h)
        buf = C.create_string_buffer(n.value)
        _check(load().pf_save(self._h, buf, n.value), self._h)
        return buf.raw

    def pf_load(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        _check(load().pf_load(self._h, buf, len(blob)), self._h)


    # ---- a shard of a particle-sharded filter (pf_shard_* in include/pf.h);
    # device buffers are addresses (int), host arrays NumPy
    def pf_shard_info(self):
        tot, first = C.c_int64(), C.c_int64()
        nt, nta, rec = C.c_int(), C.c_int(), C.c_int()
        _check(load().pf_shard_info(self._h, C.byref(tot), C.byref(first), C.byref(nt),
                                    C.byref(nta), C.byref(rec)), self._h)
        return dict(total=tot.value, first=first.value, tiles=nt.value, tiles_all=nta.value,
                    record=rec.value)

    def pf_shard_stage1(self, t, y):
        m = C.c_double()
        _check(load().pf_shard_stage1(self._h, float(t), _d(_f64(y)), C.byref(m)), self._h)
        return m.value

    def pf_shard_scan(self, lg_max, n_tiles):
        tiles = np.zeros(n_tiles)
        cl = C.c_double()
        _check(load().pf_shard_scan(self._h, float(lg_max), _d(tiles), C.byref(cl)), self._h)
        return tiles, cl.value

    def pf_shard_offsets(self, tiles_all, cl_last):
        ta = _f64(tiles_all)
        ends = np.zeros(len(ta))
        tot, u = C.c_double(), C.c_double()
        _check(load().pf_shard_offsets(self._h, _d(ta), float(cl_last), _d(ends), C.byref(tot),
                                       C.byref(u)), self._h)
        return ends, tot.value, u.value

    def pf_shard_resample(self, i_lo, i_hi, i_fb, u, total, send_ptr):
        _check(load().pf_shard_resample(self._h, int(i_lo), int(i_hi), int(i_fb), float(u),
                                        float(total), C.c_void_p(int(send_ptr)) if send_ptr else None),
               self._h)

    def pf_shard_stage2(self, recv_ptr):
        m = C.c_double()
        _check(load().pf_shard_stage2(self._h, C.c_void_p(int(recv_ptr)), C.byref(m)), self._h)
        return m.value

    def pf_shard_moments(self, lw_max):
        sums = np.zeros(128)
        nv = C.c_int()
        _check(load().pf_shard_moments(self._h, float(lw_max), _d(sums), C.byref(nv)), self._h)
        return sums[:nv.value].copy()

    def pf_shard_commit(self, sums):
        sm = _f64(sums)
        _check(load().pf_shard_commit(self._h, _d(sm), len(sm)), self._h)

    def pf_shard_abort(self):
        _check(load().pf_shard_abort(self._h), self._h)

    def pf_shard_parents(self):
        out = np.zeros(self.N, dtype=np.int32)
        _check(load().pf_shard_parents(self._h, out.ctypes.data_as(_ip)), self._h)
        return out


def pf_shard_tile(N):
    return int(load().pf_shard_tile(int(N)))


class Batch:
    """Many filters advanced together by tile-scheduled batched launches."""

    def __init__(self, filters, stream=None):
        L = load()
        self.filters = list(filters)
        arr = (C.c_void_p * len(self.filters))(*[f._h.value for f in self.filters])
        h = C.c_void_p()
        st = L.pf_batch_create(arr, len(self.filters), C.c_void_p(stream) if stream else None,
                               C.byref(h))
        _check(st, None)
        self._h = h
        # one row of observations per member, reused by every call: the
        # pointer array is the rows' addresses (0 for idle members)
        self._m = [f.m for f in self.filters]
        self._ybuf = np.zeros((len(self.filters), max(self._m + [1])), dtype=np.float64)
        self._rows = (self._ybuf.ctypes.data
                      + self._ybuf.strides[0] * np.arange(len(self.filters), dtype=np.uint64))

    def close(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.pf_batch_destroy(h)
        self._h = None

    def __del__(self):
        self.close()

    def pf_batch_assimilate(self, t, ys):
        """t: n times; ys: list of n observation arrays or None (idle).
        Returns the per-filter status codes."""
        n = len(self.filters)
        if len(t) != n or len(ys) != n:
            raise ValueError(f"need {n} times and {n} observations (None for idle)")
        tt = _f64(t)
        addr = np.zeros(n, dtype=np.uint64)
        for i, y in enumerate(ys):
            if y is not None:
                self._ybuf[i, :self._m[i]] = y
                addr[i] = self._rows[i]
        status = np.zeros(n, dtype=np.int32)
        st = load().pf_batch_assimilate(self._h, _d(tt), C.cast(addr.ctypes.data, C.POINTER(_dp)),
                                        status.ctypes.data_as(C.POINTER(C.c_int)))
        if st != PF_OK:
            msg = load().pf_batch_last_error(self._h)
            raise PfError(st, msg.decode() if msg else "")
        return status.tolist()

    def pf_batch_stats(self):
        s = BatchStats()
        _check(load().pf_batch_stats(self._h, C.byref(s)), None)
        return dict(epochs=s.epochs, graph_captures=s.graph_captures,
                    last_device_ms=s.last_device_ms, last_active=s.last_active,
                    last_tiles=s.last_tiles, tile_order=s.tile_order,
                    concurrent_models=s.concurrent_models, tune_ms=list(s.tune_ms))


def _prior_options(w, N=None, seed=None, filter_id=0):
    keep = []
    kind = (C.c_int * len(w.prior_kind))(*[int(k) for k in w.prior_kind])
    lo, hi, x0 = _f64(w.prior_lo), _f64(w.prior_hi), _f64(w.x0)
    obs = (C.c_int * len(w.obs_idx))(*[int(o) for o in w.obs_idx])
    sig = _f64(w.sigma)
    keep += [kind, lo, hi, x0, obs, sig]
    pr = Prior(w.p, kind, _d(lo), _d(hi), w.d, _d(x0), float(w.t0))
    op = Options(float(w.a), int(w.newton_iters), int(w.spacing), int(w.substeps), float(w.q0),
                 int(w.history), int(w.transform), len(w.obs_idx), obs, int(w.noise), _d(sig),
                 float(w.kappa), int(w.seed if seed is None else seed), int(filter_id), None, 0)
    return pr, op, keep


class Server:
    """Filter sessions admitted by device-memory budget and served by
    continuous batching (see include/pf.h)."""

    def __init__(self, budget_bytes, lanes=0):
        h = C.c_void_p()
        _check(load().pf_server_create(int(budget_bytes), int(lanes), C.byref(h)), None)
        self._h = h
        self._shapes = {}

    def _check(self, st):
        if st != PF_OK:
            msg = load().pf_server_last_error(self._h)
            raise PfError(st, msg.decode() if msg else "")

    def close(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.pf_server_destroy(h)
        self._h = None

    def __del__(self):
        self.close()

    def pf_server_open(self, w, N=None, seed=None, filter_id=0):
        N = int(N if N is not None else w.N)
        pr, op, keep = _prior_options(w, N, seed, filter_id)
        sid = C.c_int64()
        self._check(load().pf_server_open(self._h, w.ode, w.d, w.p, N, w.lmm, float(w.dt),
                                          C.byref(pr), C.byref(op), C.byref(sid)))
        self._shapes[sid.value] = (w.ode, w.d, w.p, N, len(w.obs_idx))
        return sid.value

    def pf_server_submit(self, session, t, y):
        y = _f64(y)
        self._check(load().pf_server_submit(self._h, int(session), float(t), _d(y)))

    def pf_server_step(self):
        n = C.c_int()
        self._check(load().pf_server_step(self._h, C.byref(n)))
        return n.value

    def pf_server_drain(self):
        self._check(load().pf_server_drain(self._h))

    def pf_server_close(self, session):
        self._check(load().pf_server_close(self._h, int(session)))

    def pf_server_session(self, session):
        fh = C.c_void_p()
        done = C.c_int64()
        last = C.c_int()
        self._check(load().pf_server_session(self._h, int(session), C.byref(fh), C.byref(done),
                                             C.byref(last)))
        f = Filter.borrowed(fh.value, *self._shapes[int(session)]) if fh.value else None
        return f, done.value, last.value

    def pf_server_stats(self):
        s = ServerStats()
        self._check(load().pf_server_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}
