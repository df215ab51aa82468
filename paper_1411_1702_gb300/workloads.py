"""Seeded synthetic workloads for the LMM PF-SMC sampler.

This module only describes problems and makes data: observation times, noisy
observations of a reference trajectory, priors, the initial state and the
sampler's settings.  It holds none of the sampler's arithmetic: the reference
trajectory comes from a closed form (the linear system) or from SciPy's Radau
integrator at tight tolerances (Robertson, Brusselator), and the observation
noise from NumPy's seeded generator.  Both the CUDA library and the CPU oracle
consume these inputs.

Problems (the paper's own test systems, Sec. 2.1 and Sec. 4, lack constants or
need a different solver, so three textbook stiff systems stand in, sized like
the paper's workloads -- thousands to ~10^5 particles, 30-50 observations):

* ``linear2``      x' = A x, A = [[-th1, th2], [0, -th2]], th* = (1, 1000),
                   x1 observed with sigma = 0.01 at t = 0.1 k, k = 1..50,
                   BDF2 with 20 uniform substeps per interval.
* ``robertson``    Robertson kinetics, th* = (0.04, 3e7, 1e4), y1 and y3
                   observed with 1% relative noise at 40 log-spaced times on
                   [1e-4, 1e4], 50 geometric substeps per interval.
* ``brusselator``  1D Brusselator on 32 interior points (d = 64),
                   th* = (A, B, alpha) = (1, 3, 0.02), u observed at 8 points
                   with sigma = 0.02 at t = k/3, k = 1..30, 20 uniform substeps.
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

LINEAR2, ROBERTSON, BRUSSELATOR, ADVDIFF, MICHAELIS = 1, 2, 3, 4, 5
# LMMs of the paper's Tables 1-2 (the first three of each family)
LMM_BDF1, LMM_BDF2, LMM_BDF3 = 1, 2, 3
LMM_AM1, LMM_AM2, LMM_AM3 = 11, 12, 13
LMM_AB1, LMM_AB2, LMM_AB3 = 21, 22, 23
LMM_NAMES = {"BDF1": LMM_BDF1, "BDF2": LMM_BDF2, "BDF3": LMM_BDF3, "AM1": LMM_AM1,
             "AM2": LMM_AM2, "AM3": LMM_AM3, "AB1": LMM_AB1, "AB2": LMM_AB2, "AB3": LMM_AB3}
UNIFORM, LOGUNIFORM = 0, 1
SPACING_UNIFORM, SPACING_GEOMETRIC = 0, 1
HIST_CARRY, HIST_RESTART = 0, 1
TRANSFORM_LOG, TRANSFORM_IDENTITY = 0, 1
NOISE_ADDITIVE, NOISE_RELATIVE = 0, 1

# Fixed Newton count per problem (no early exit, so every particle costs the
# same).  Each is the smallest K whose result agrees with the fully converged
# Newton solution to 1e-12 relative along the reference trajectory and on the
# particles of a filter run; the test-suite re-checks the reference trajectory.
NEWTON_ITERS = {LINEAR2: 1, ROBERTSON: 2, BRUSSELATOR: 3, ADVDIFF: 1, MICHAELIS: 4}


@dataclasses.dataclass
class Workload:
    name: str
    ode: int
    d: int
    p: int
    N: int
    lmm: int
    newton_iters: int
    spacing: int
    dt: float
    substeps: int
    q0: float
    history: int
    transform: int
    obs_idx: list
    noise: int
    sigma: list
    a: float
    kappa: float
    seed: int
    stream: int
    prior_kind: list
    prior_lo: list
    prior_hi: list
    x0: np.ndarray
    t0: float
    theta_true: np.ndarray
    t_obs: np.ndarray          # (T,)
    y_obs: np.ndarray          # (T, m)
    x_true: np.ndarray         # (T, d) reference states at t_obs

    @property
    def m(self) -> int:
        return len(self.obs_idx)

    @property
    def T(self) -> int:
        return len(self.t_obs)

    def substeps_per_interval(self, k: int) -> int:
        """Substep count of observation interval k (0-based)."""
        if self.spacing == SPACING_GEOMETRIC:
            return self.substeps
        t0 = self.t0 if k == 0 else self.t_obs[k - 1]
        return int(round((self.t_obs[k] - t0) / self.dt))

    def particle_steps(self, k: int) -> int:
        """particle-LMM-steps of epoch k: two propagations (Steps 2 and 4) of
        every particle over the interval's substeps."""
        return 2 * self.substeps_per_interval(k) * self.N

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def _noise(rng, x_obs, sigma, relative):
    eps = rng.standard_normal(x_obs.shape)
    if relative:
        return x_obs * (1.0 + np.asarray(sigma)[None, :] * eps)
    return x_obs + np.asarray(sigma)[None, :] * eps


# ---------------------------------------------------------------- linear2
def linear2_exact(theta, x0, t):
    """Closed-form solution of x' = A x, A = [[-th1, th2], [0, -th2]]."""
    th1, th2 = float(theta[0]), float(theta[1])
    t = np.asarray(t, dtype=np.float64)
    x2 = x0[1] * np.exp(-th2 * t)
    x1 = x0[0] * np.exp(-th1 * t) + th2 * x0[1] * (np.exp(-th2 * t) - np.exp(-th1 * t)) / (th1 - th2)
    return np.stack([x1, x2], axis=-1)


def linear2(N: int = 2000, T: int = 50, seed: int = 0, theta=None) -> Workload:
    theta = np.array([1.0, 1000.0]) if theta is None else np.asarray(theta, dtype=float)
    x0 = np.array([1.0, 1.0])
    t_obs = 0.1 * np.arange(1, T + 1)
    x_true = linear2_exact(theta, x0, t_obs)
    obs_idx, sigma = [0], [0.01]
    rng = np.random.default_rng([seed, 0xDA7A, LINEAR2])
    y = _noise(rng, x_true[:, obs_idx], sigma, False)
    return Workload(
        name="linear2", ode=LINEAR2, d=2, p=2, N=N, lmm=2, newton_iters=NEWTON_ITERS[LINEAR2],
        spacing=SPACING_UNIFORM, dt=0.005, substeps=20, q0=0.0,
        history=HIST_CARRY, transform=TRANSFORM_LOG, obs_idx=obs_idx,
        noise=NOISE_ADDITIVE, sigma=sigma, a=0.98, kappa=1.0, seed=seed, stream=0,
        prior_kind=[LOGUNIFORM, LOGUNIFORM], prior_lo=[0.1, 100.0], prior_hi=[10.0, 1e4],
        x0=x0, t0=0.0, theta_true=theta, t_obs=t_obs, y_obs=y, x_true=x_true)


# -------------------------------------------------------------- robertson
def robertson_rhs(theta):
    k1, k2, k3 = theta

    def f(t, y):
        return np.array([-k1 * y[0] + k3 * y[1] * y[2],
                         k1 * y[0] - k3 * y[1] * y[2] - k2 * y[1] ** 2,
                         k2 * y[1] ** 2])

    def jac(t, y):
        return np.array([[-k1, k3 * y[2], k3 * y[1]],
                         [k1, -k3 * y[2] - 2 * k2 * y[1], -k3 * y[1]],
                         [0.0, 2 * k2 * y[1], 0.0]])
    return f, jac


def robertson_times(T: int = 40):
    k = np.arange(1, T + 1)
    return 10.0 ** (-4.0 + 8.0 * (k - 1) / 39.0)


def robertson(N: int = 131072, T: int = 40, seed: int = 0, theta=None,
              rtol: float = 1e-11) -> Workload:
    from scipy.integrate import solve_ivp
    theta_star = np.array([0.04, 3e7, 1e4])
    theta = theta_star if theta is None else np.asarray(theta, dtype=float)
    x0 = np.array([1.0, 0.0, 0.0])
    t_all = robertson_times(40)
    f, jac = robertson_rhs(theta)
    sol = solve_ivp(f, (0.0, t_all[-1]), x0, method="Radau", t_eval=t_all, rtol=rtol,
                    atol=1e-18 if rtol < 1e-9 else 1e-14, jac=jac)
    x_true = sol.y.T[:T]
    t_obs = t_all[:T]
    obs_idx, sigma = [0, 2], [0.01, 0.01]
    rng = np.random.default_rng([seed, 0xDA7A, ROBERTSON])
    y = _noise(rng, x_true[:, obs_idx], sigma, True)
    S = 50
    q0 = 10.0 ** (8.0 / (39.0 * S))   # the same ratio as the later intervals
    return Workload(
        name="robertson", ode=ROBERTSON, d=3, p=3, N=N, lmm=2, newton_iters=NEWTON_ITERS[ROBERTSON],
        spacing=SPACING_GEOMETRIC, dt=0.0, substeps=S, q0=q0,
        history=HIST_CARRY, transform=TRANSFORM_LOG, obs_idx=obs_idx,
        noise=NOISE_RELATIVE, sigma=sigma, a=0.98, kappa=1.0, seed=seed, stream=0,
        prior_kind=[LOGUNIFORM] * 3, prior_lo=list(theta_star / 10.0),
        prior_hi=list(theta_star * 10.0), x0=x0, t0=0.0, theta_true=theta, t_obs=t_obs, y_obs=y,
        x_true=x_true)


# -------------------------------------------------------------- michaelis
# M1 of Sec. 2.1.  The paper names lambda, c0, A0, A, t0, tau as known but
# prints no values, nor the true (V1, V2, k1, k2), the noise or the time span;
# the values below are this project's reading (see the design notes).
MM_THETA = (3.0, 2.5, 0.5, 0.3)          # (V1, V2, k1, k2)
MM_KNOWN = dict(lam=0.5, c0=2.0, A0=1.0, A=0.5, t0=0.5, tau=4.0)


def mm_input(t):
    k = MM_KNOWN
    s = t - k["t0"]
    return k["A0"] + (k["A"] * s * math.exp(-s / k["tau"]) if s > 0.0 else 0.0)


def michaelis_rhs(theta):
    V1, V2, k1, k2 = (float(v) for v in theta)
    lam, c0 = MM_KNOWN["lam"], MM_KNOWN["c0"]

    def f(t, x):
        j1 = V1 * x[0] / (x[0] + k1)
        j2 = V2 * x[1] / (x[1] + k2)
        return np.array([mm_input(t) - j1, j1 - j2, j2 - lam * (x[2] - c0)])

    def jac(t, x):
        a = V1 * k1 / (x[0] + k1) ** 2
        b = V2 * k2 / (x[1] + k2) ** 2
        return np.array([[-a, 0.0, 0.0], [a, -b, 0.0], [0.0, b, -lam]])
    return f, jac


def michaelis_x0(theta=MM_THETA):
    """The steady state of the true system under the constant input A0 (the
    input is A0 until t0): V1 x1/(x1+k1) = A0, V2 x2/(x2+k2) = A0,
    lambda (x3 - c0) = A0."""
    V1, V2, k1, k2 = theta
    A0, lam, c0 = MM_KNOWN["A0"], MM_KNOWN["lam"], MM_KNOWN["c0"]
    return np.array([A0 * k1 / (V1 - A0), A0 * k2 / (V2 - A0), c0 + A0 / lam])


def michaelis_truth(theta, x0, t_obs, rtol=1e-11):
    """Reference trajectory by Radau, split at t0 where the input's slope jumps."""
    from scipy.integrate import solve_ivp
    f, jac = michaelis_rhs(theta)
    t0 = MM_KNOWN["t0"]
    out = np.empty((len(t_obs), 3))
    first = t_obs <= t0
    x = np.array(x0, dtype=float)
    if first.any():
        sol = solve_ivp(f, (0.0, t0), x, method="Radau", t_eval=t_obs[first], rtol=rtol,
                        atol=1e-14, jac=jac, dense_output=False)
        out[first] = sol.y.T
    rest = ~first
    if not rest.any():
        return out
    sol0 = solve_ivp(f, (0.0, t0), x, method="Radau", rtol=rtol, atol=1e-14, jac=jac)
    x = sol0.y[:, -1]
    sol = solve_ivp(f, (t0, float(t_obs[-1])), x, method="Radau", t_eval=t_obs[rest], rtol=rtol,
                    atol=1e-14, jac=jac)
    out[rest] = sol.y.T
    return out


def michaelis(N: int = 50000, T: int = 50, seed: int = 0, lmm: int = LMM_BDF2,
              theta=None) -> Workload:
    """M1 of Sec. 2.1 as Tables 1-2 run it: all three states observed at 50
    times, fixed step h = 0.05.  Reading: t_k = 0.5 k (10 steps per interval),
    2 % relative noise, log-uniform priors one decade either side of
    theta* = (V1, V2, k1, k2) = (3, 2.5, 0.5, 0.3), x0 the steady state under
    the input A0.  The prior reaches V/k ~ 600, where h |lambda| ~ 30: stiff
    for part of the ensemble, as the paper describes."""
    theta_star = np.array(MM_THETA)
    theta = theta_star if theta is None else np.asarray(theta, dtype=float)
    x0 = michaelis_x0(MM_THETA)
    t_obs = 0.5 * np.arange(1, T + 1)
    x_true = michaelis_truth(theta, x0, t_obs)
    obs_idx, sigma = [0, 1, 2], [0.02, 0.02, 0.02]
    rng = np.random.default_rng([seed, 0xDA7A, MICHAELIS])
    y = _noise(rng, x_true[:, obs_idx], sigma, True)
    name = "michaelis" + next((k for k, v in LMM_NAMES.items() if v == lmm), str(lmm))
    return Workload(
        name=name, ode=MICHAELIS, d=3, p=4, N=N, lmm=lmm, newton_iters=NEWTON_ITERS[MICHAELIS],
        spacing=SPACING_UNIFORM, dt=0.05, substeps=10, q0=0.0,
        history=HIST_CARRY, transform=TRANSFORM_LOG, obs_idx=obs_idx,
        noise=NOISE_RELATIVE, sigma=sigma, a=0.98, kappa=1.0, seed=seed, stream=0,
        prior_kind=[LOGUNIFORM] * 4, prior_lo=list(theta_star / 10.0),
        prior_hi=list(theta_star * 10.0), x0=x0, t0=0.0, theta_true=theta, t_obs=t_obs,
        y_obs=y, x_true=x_true)


# ------------------------------------------------------------ brusselator
BR_POINTS = 32


def brusselator_rhs(theta):
    A, B, alpha = theta
    D = alpha * 33.0 ** 2

    def f(t, x):
        u, v = x[0::2], x[1::2]
        up = np.concatenate([[1.0], u, [1.0]])
        vp = np.concatenate([[3.0], v, [3.0]])
        du = A + u * u * v - (B + 1) * u + D * (up[:-2] - 2 * u + up[2:])
        dv = B * u - u * u * v + D * (vp[:-2] - 2 * v + vp[2:])
        out = np.empty_like(x)
        out[0::2], out[1::2] = du, dv
        return out

    def jac(t, x):
        u, v = x[0::2], x[1::2]
        n = 2 * BR_POINTS
        J = np.zeros((n, n))
        for i in range(BR_POINTS):
            a, b = 2 * i, 2 * i + 1
            J[a, a] = 2 * u[i] * v[i] - (B + 1) - 2 * D
            J[a, b] = u[i] ** 2
            J[b, a] = B - 2 * u[i] * v[i]
            J[b, b] = -u[i] ** 2 - 2 * D
            if i > 0:
                J[a, a - 2] = D
                J[b, b - 2] = D
            if i < BR_POINTS - 1:
                J[a, a + 2] = D
                J[b, b + 2] = D
        return J
    return f, jac


def brusselator_x0():
    xi = np.arange(1, BR_POINTS + 1) / 33.0
    x0 = np.empty(2 * BR_POINTS)
    x0[0::2] = 1.0 + np.sin(2 * math.pi * xi)
    x0[1::2] = 3.0
    return x0


@functools.lru_cache(maxsize=8)
def _brusselator_truth(T: int) -> np.ndarray:
    from scipy.integrate import solve_ivp
    theta = np.array([1.0, 3.0, 0.02])
    t_obs = np.arange(1, T + 1) / 3.0
    f, jac = brusselator_rhs(theta)
    sol = solve_ivp(f, (0.0, t_obs[-1]), brusselator_x0(), method="Radau", t_eval=t_obs,
                    rtol=1e-11, atol=1e-12, jac=jac)
    x = sol.y.T.copy()
    x.flags.writeable = False
    return x


def brusselator(N: int = 65536, T: int = 30, seed: int = 0) -> Workload:
    theta = np.array([1.0, 3.0, 0.02])
    x0 = brusselator_x0()
    t_obs = np.arange(1, T + 1) / 3.0
    x_true = np.array(_brusselator_truth(T))
    obs_idx = [2 * i for i in range(2, 32, 4)]
    sigma = [0.02] * len(obs_idx)
    rng = np.random.default_rng([seed, 0xDA7A, BRUSSELATOR])
    y = _noise(rng, x_true[:, obs_idx], sigma, False)
    return Workload(
        name="brusselator", ode=BRUSSELATOR, d=64, p=3, N=N, lmm=2, newton_iters=NEWTON_ITERS[BRUSSELATOR],
        spacing=SPACING_UNIFORM, dt=1.0 / 60.0, substeps=20, q0=0.0,
        history=HIST_CARRY, transform=TRANSFORM_LOG, obs_idx=obs_idx,
        noise=NOISE_ADDITIVE, sigma=sigma, a=0.98, kappa=1.0, seed=seed, stream=0,
        prior_kind=[UNIFORM] * 3, prior_lo=list(0.5 * theta), prior_hi=list(1.5 * theta),
        x0=x0, t0=0.0, theta_true=theta, t_obs=t_obs, y_obs=y, x_true=x_true)


def batched(n_filters: int = 256, seed: int = 0, n_min_log2: float = 10.0,
            n_max_log2: float = 17.0):
    """Independent filters of uneven size and mixed problems: N_f =
    round(2^U[10, 17]), problem linear2 or robertson with probability 1/2
    each, the true parameter drawn from that problem's prior, seed and filter
    id f.  Robertson reference trajectories are solved at rtol 1e-8 (ample for
    1 % observation noise)."""
    rng = np.random.default_rng([seed, 0xBA7C])
    out = []
    for f in range(n_filters):
        N = int(round(2.0 ** rng.uniform(n_min_log2, n_max_log2)))
        if rng.random() < 0.5:
            lo, hi = np.array([0.1, 100.0]), np.array([10.0, 1e4])
            th = np.exp(rng.uniform(np.log(lo), np.log(hi)))
            w = linear2(N=N, seed=f, theta=th)
        else:
            star = np.array([0.04, 3e7, 1e4])
            th = np.exp(rng.uniform(np.log(star / 10.0), np.log(star * 10.0)))
            w = robertson(N=N, seed=f, theta=th, rtol=1e-8)
        out.append(w.with_(stream=f))
    return out


# ---- the paper's 2D advection-diffusion system (Sec. 4) --------------------
# Gaussian plumes of the initial state: (standard deviation, x centre,
# y centre), the table of Sec. 4.
AD_PLUMES = ((0.04, 0.20, 0.80), (0.08, 0.30, 0.40), (0.07, 0.40, 0.40),
             (0.10, 0.50, 0.50), (0.05, 0.50, 0.60), (0.06, 0.70, 0.50))
AD_THETA = (9.0, 4.0, 6.0, 2.5, -1.5)   # (k1, k2, k3, c1, c2) of Sec. 4


def advdiff_x0(n: int) -> np.ndarray:
    """u0 on the periodic grid: the n x n grid of [0,1]^2 without its last row
    and column, nt = n - 1 points per side at j / (n - 1), stacked as
    U[iy * nt + ix] (x fastest)."""
    nt = n - 1
    c = np.arange(nt) / (n - 1)
    X, Y = np.meshgrid(c, c, indexing="xy")       # X[iy, ix] = c[ix]
    u = np.zeros((nt, nt))
    for g, xc, yc in AD_PLUMES:
        u += np.exp(-((X - xc) ** 2 + (Y - yc) ** 2) / (2.0 * g * g)) / (g * math.sqrt(2 * math.pi))
    return u.reshape(-1)


def advdiff_eigenvalues(nt: int, theta) -> np.ndarray:
    """Eigenvalues lam[my, mx] of the M2 operator on the Fourier mode
    exp(2 pi i (mx ix + my iy) / nt): the difference matrix ell (u_j - u_{j-1},
    periodic) is circulant with symbol a(m) = 1 - exp(-2 pi i m / nt)."""
    k1, k2, k3, c1, c2 = (float(v) for v in theta)
    a = 1.0 - np.exp(-2j * np.pi * np.arange(nt) / nt)
    ax, ay = a[None, :], a[:, None]
    return (-(k1 * k1 * np.abs(ax) ** 2 + 2.0 * k1 * k3 * np.real(np.conj(ax) * ay)
              + (k2 * k2 + k3 * k3) * np.abs(ay) ** 2) + c1 * ax + c2 * ay)


def advdiff_exact(n: int, theta, x0, t) -> np.ndarray:
    """exp(t L) x0 for each time in t (rows), through the 2D DFT."""
    nt = n - 1
    lam = advdiff_eigenvalues(nt, theta)
    U0 = np.fft.fft2(np.asarray(x0, dtype=np.float64).reshape(nt, nt))
    out = [np.real(np.fft.ifft2(U0 * np.exp(tt * lam))).reshape(-1) for tt in np.atleast_1d(t)]
    return np.array(out)


def advdiff(n: int = 20, N: int = 5000, T: int = 30, seed: int = 0, m: int = 20) -> Workload:
    """M2 of Sec. 4: d = (n-1)^2, theta* = (9, 4, 6, 2.5, -1.5), m = 20 fixed
    sensors drawn without replacement from the grid, observed at t = 1..T with
    additive noise sigma = max |u0 at the sensors| / 50; BDF2 with h = 0.1.
    The prior (not given in the paper) is uniform on theta* -+ |theta*| / 2,
    sampled in theta space (c2 is negative)."""
    theta = np.array(AD_THETA)
    nt = n - 1
    d = nt * nt
    x0 = advdiff_x0(n)
    rng = np.random.default_rng([seed, 0xAD, n])
    m = min(m, d)
    obs_idx = [int(i) for i in np.sort(rng.choice(d, size=m, replace=False))]
    t_obs = np.arange(1, T + 1, dtype=np.float64)
    x_true = advdiff_exact(n, theta, x0, t_obs)
    sig = float(np.max(np.abs(x0[obs_idx]))) / 50.0
    sigma = [sig] * m
    y = _noise(rng, x_true[:, obs_idx], sigma, False)
    half = 0.5 * np.abs(theta)
    return Workload(
        name=f"advdiff{n}", ode=ADVDIFF, d=d, p=5, N=N, lmm=2, newton_iters=NEWTON_ITERS[ADVDIFF],
        spacing=SPACING_UNIFORM, dt=0.1, substeps=10, q0=0.0,
        history=HIST_CARRY, transform=TRANSFORM_IDENTITY, obs_idx=obs_idx,
        noise=NOISE_ADDITIVE, sigma=sigma, a=0.98, kappa=1.0, seed=seed, stream=0,
        prior_kind=[UNIFORM] * 5, prior_lo=list(theta - half), prior_hi=list(theta + half),
        x0=x0, t0=0.0, theta_true=theta, t_obs=t_obs, y_obs=y, x_true=x_true)


def advdiff20(N: int = 5000, T: int = 30, seed: int = 0) -> Workload:
    return advdiff(20, N, T, seed)


def advdiff40(N: int = 5000, T: int = 30, seed: int = 0) -> Workload:
    return advdiff(40, N, T, seed)


@dataclasses.dataclass
class Session:
    """One filter session of a serving trace: its problem and the wall-clock
    arrival time (seconds from the start) of the session and of each of its
    observations."""
    w: Workload
    open_s: float
    obs_s: np.ndarray


def serving(n_sessions: int = 64, rate_hz: float = 200.0, obs_per_session: int = 0,
            mean_gap_ms: float = 5.0, seed: int = 0, n_log2=(12, 18)) -> list:
    """Serving trace: sessions arrive as a Poisson process (rate_hz); each is
    linear2, robertson or brusselator with probability 1/3, N = 2^k with k
    uniform on n_log2 (4096 ... 262144), its true parameter drawn from that
    problem's prior (the Brusselator keeps its reference parameter), and its
    observations arrive at exponential intervals of mean mean_gap_ms, the
    first one a gap after the session opens.  A session has obs_per_session
    observations, or its problem's T (linear2 50, robertson 40, brusselator
    30) when that is 0."""
    rng = np.random.default_rng([seed, 0x5E55])
    out = []
    t = 0.0
    for s in range(n_sessions):
        t += rng.exponential(1.0 / rate_hz)
        N = 2 ** int(rng.integers(n_log2[0], n_log2[1] + 1))
        kind = int(rng.integers(3))
        T = obs_per_session or (50, 40, 30)[kind]
        if kind == 0:
            lo, hi = np.array([0.1, 100.0]), np.array([10.0, 1e4])
            w = linear2(N=N, T=T, seed=s, theta=np.exp(rng.uniform(np.log(lo), np.log(hi))))
        elif kind == 1:
            star = np.array([0.04, 3e7, 1e4])
            w = robertson(N=N, T=T, seed=s, rtol=1e-8,
                          theta=np.exp(rng.uniform(np.log(star / 10.0), np.log(star * 10.0))))
        else:
            w = brusselator(N=N, T=T, seed=s)
        gaps = rng.exponential(mean_gap_ms * 1e-3, size=T)
        out.append(Session(w=w.with_(stream=s), open_s=t, obs_s=t + np.cumsum(gaps)))
    return out


BY_NAME = {"linear2": linear2, "robertson": robertson, "brusselator": brusselator,
           "advdiff20": advdiff20, "advdiff40": advdiff40, "michaelis": michaelis}
for _lname, _lmm in LMM_NAMES.items():
    BY_NAME["michaelis" + _lname] = functools.partial(michaelis, lmm=_lmm)
# Robertson at 2^22 particles: the scan and resampling kernels at a size where
# they move enough data for their bandwidth to show
BY_NAME["robertson22"] = functools.partial(robertson, N=1 << 22)


def get(name: str, **kw) -> Workload:
    return BY_NAME[name](**kw)
