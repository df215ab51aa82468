"""Pins of the CPU oracle against facts outside the oracle itself.

Every oracle function is checked against something it does not compute:
published known-answer vectors, textbook constants, closed-form solutions,
invariants of the test problems, a library routine (NumPy/SciPy), finite
differences, or brute force on tiny inputs.  Each pin is chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand) fails it.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------- Philox
def test_philox_known_answers(oracle_lib):
    for row in _golden_rows("philox4x32_10_kat.txt"):
        vals = [int(v, 16) for v in row]
        assert oracle.philox(vals[0:4], vals[4:6]) == tuple(vals[6:10])


def test_uniform53_grid_and_range(oracle_lib):
    us = np.array([oracle.uniform(7, 0, oracle.RNG_INIT, n, 0, k) for n in range(2000) for k in range(2)])
    assert np.all(us >= 0.0) and np.all(us < 1.0)
    # every value is an integer multiple of 2^-53
    scaled = us * 2.0 ** 53
    assert np.all(scaled == np.floor(scaled))
    from scipy import stats
    assert stats.kstest(us, "uniform").pvalue > 1e-3


def test_uniform53_bits(oracle_lib):
    # the uniform is built from the high 27 bits of word 0 and high 26 of word 1
    seed, n, epoch = 0x1234_5678_9ABC_DEF0, 5, 3
    w = oracle.philox((n, epoch, oracle.RNG_INIT | (0 << 8), 0), (seed & 0xFFFFFFFF, seed >> 32))
    u0 = oracle.uniform(seed, 0, oracle.RNG_INIT, n, epoch, 0)
    u1 = oracle.uniform(seed, 0, oracle.RNG_INIT, n, epoch, 1)
    assert int(u0 * 2 ** 53) == ((w[0] >> 5) << 26) | (w[1] >> 6)
    assert int(u1 * 2 ** 53) == ((w[2] >> 5) << 26) | (w[3] >> 6)


def test_normals_are_standard(oracle_lib):
    from scipy import stats
    z = np.array([oracle.normal(11, 0, oracle.RNG_THETA, n, 2, k) for n in range(6000) for k in range(4)])
    assert abs(z.mean()) < 4.0 / math.sqrt(len(z))
    assert abs(z.var() - 1.0) < 6.0 * math.sqrt(2.0 / len(z))
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the cosine and sine branches of one Box-Muller pair are uncorrelated
    pairs = z.reshape(-1, 2)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 4.0 / math.sqrt(len(pairs))


def test_streams_differ_by_purpose_epoch_filter(oracle_lib):
    a = oracle.normal(3, 0, oracle.RNG_THETA, 10, 4, 0)
    assert a != oracle.normal(3, 0, oracle.RNG_INNOV, 10, 4, 0)
    assert a != oracle.normal(3, 0, oracle.RNG_THETA, 10, 5, 0)
    assert a != oracle.normal(3, 1, oracle.RNG_THETA, 10, 4, 0)
    assert a != oracle.normal(4, 0, oracle.RNG_THETA, 10, 4, 0)
    assert a == oracle.normal(3, 0, oracle.RNG_THETA, 10, 4, 0)


# ----------------------------------------------------------------- models
def _fd_jac(ode, th, x, eps=1e-6):
    d = len(x)
    J = np.zeros((d, d))
    for j in range(d):
        hstep = eps * max(1.0, abs(x[j]))
        xp, xm = x.copy(), x.copy()
        xp[j] += hstep
        xm[j] -= hstep
        J[:, j] = (oracle.ode_f(ode, th, xp) - oracle.ode_f(ode, th, xm)) / (2 * hstep)
    return J


@pytest.mark.parametrize("ode", [oracle.LINEAR2, oracle.ROBERTSON, oracle.BRUSSELATOR])
def test_jacobian_matches_finite_differences(oracle_lib, ode):
    rng = np.random.default_rng(ode)
    d, p = oracle.ode_dims(ode)
    for _ in range(3):
        if ode == oracle.LINEAR2:
            th, x = np.array([1.3, 800.0]), rng.normal(size=2)
        elif ode == oracle.ROBERTSON:
            th, x = np.array([0.04, 3e7, 1e4]), np.abs(rng.normal(size=3)) * np.array([1, 1e-5, 1])
        else:
            th, x = np.array([1.1, 2.7, 0.025]), 1.0 + 2.0 * rng.random(d)
        J = oracle.ode_jac(ode, th, x)
        Jfd = _fd_jac(ode, th, x, eps=1e-7)
        scale = np.max(np.abs(J))
        assert np.max(np.abs(J - Jfd)) <= 1e-6 * scale


def test_models_against_independent_rhs(oracle_lib):
    """The oracle's right-hand sides equal the input generator's NumPy forms."""
    rng = np.random.default_rng(5)
    th = np.array([0.05, 2e7, 2e4])
    f, jac = W.robertson_rhs(th)
    x = np.abs(rng.normal(size=3))
    assert np.allclose(oracle.ode_f(oracle.ROBERTSON, th, x), f(0, x), rtol=1e-14, atol=0)
    assert np.allclose(oracle.ode_jac(oracle.ROBERTSON, th, x), jac(0, x), rtol=1e-14, atol=0)
    th = np.array([1.2, 3.3, 0.018])
    f, jac = W.brusselator_rhs(th)
    x = 1.0 + rng.random(64)
    assert np.allclose(oracle.ode_f(oracle.BRUSSELATOR, th, x), f(0, x), rtol=1e-12, atol=1e-12)
    assert np.allclose(oracle.ode_jac(oracle.BRUSSELATOR, th, x), jac(0, x), rtol=1e-14, atol=0)


def test_robertson_rhs_conserves_mass(oracle_lib):
    rng = np.random.default_rng(1)
    for _ in range(5):
        x = rng.random(3)
        f = oracle.ode_f(oracle.ROBERTSON, np.array([0.04, 3e7, 1e4]), x)
        assert abs(f.sum()) <= 1e-12 * np.max(np.abs(f))
        J = oracle.ode_jac(oracle.ROBERTSON, np.array([0.04, 3e7, 1e4]), x)
        assert np.max(np.abs(J.sum(axis=0))) <= 1e-12 * np.max(np.abs(J))


def test_linear2_closed_form_against_expm():
    from scipy.linalg import expm
    th, x0 = np.array([1.0, 1000.0]), np.array([1.0, 1.0])
    A = np.array([[-th[0], th[1]], [0.0, -th[1]]])
    for t in [1e-4, 0.003, 0.1, 2.5]:
        assert np.allclose(W.linear2_exact(th, x0, t), expm(A * t) @ x0, rtol=1e-12, atol=1e-300)


# ------------------------------------------------------------- linear solve
def test_lu_solve_against_numpy(oracle_lib):
    rng = np.random.default_rng(2)
    for n in [1, 2, 3, 7, 64]:
        A = rng.normal(size=(n, n)) + n * np.eye(n)
        b = rng.normal(size=n)
        assert np.allclose(oracle.lu_solve(A, b), np.linalg.solve(A, b), rtol=1e-12, atol=1e-14)
    # a pivot is needed: zero leading entry
    A = np.array([[0.0, 2.0], [3.0, 1.0]])
    assert np.allclose(oracle.lu_solve(A, [4.0, 5.0]), np.linalg.solve(A, [4.0, 5.0]))
    with pytest.raises(np.linalg.LinAlgError):
        oracle.lu_solve(np.zeros((2, 2)), [1.0, 1.0])


def test_lu_solve_brusselator_newton_matrix(oracle_lib):
    th = np.array([1.0, 3.0, 0.02])
    x = W.brusselator_x0()
    M = np.eye(64) - (2.0 / 3.0) * (1.0 / 60.0) * oracle.ode_jac(oracle.BRUSSELATOR, th, x)
    b = np.random.default_rng(3).normal(size=64)
    sol = oracle.lu_solve(M, b)
    ref = np.linalg.solve(M, b)
    assert np.max(np.abs(sol - ref)) <= 1e-12 * np.max(np.abs(ref))


# ---------------------------------------------------------- BDF coefficients
def test_bdf2_constant_step_textbook(oracle_lib):
    ref = {r[0]: float(r[1]) for r in _golden_rows("bdf2_constant_step.txt")}
    h = 0.37
    c = oracle.bdf_coefficients(2, h, h, h)
    assert c.rho1 == pytest.approx(ref["rho1"], rel=1e-14)
    assert c.rho2 == pytest.approx(ref["rho2"], rel=1e-14)
    assert c.gamma / h == pytest.approx(ref["gamma_over_h"], rel=1e-14)
    assert (c.pi0, c.pi1, c.pi2) == pytest.approx((ref["pi0"], ref["pi1"], ref["pi2"]), rel=1e-13)
    assert c.mu == pytest.approx(ref["mu"], rel=1e-12)
    c1 = oracle.bdf_coefficients(1, h)
    assert (c1.rho1, c1.rho2, c1.gamma, c1.pi0) == pytest.approx((1.0, 0.0, h, 1.0), rel=1e-15)
    assert c1.mu == pytest.approx(ref["mu_bdf1"], rel=1e-14)


@pytest.mark.parametrize("steps", [(0.1, 0.1, 0.1), (0.2, 0.1, 0.05), (0.05, 0.1, 0.3),
                                   (1.7e-3, 1.6e-3, 1.55e-3), (0.38, 1.0, 1.0)])
def test_bdf2_variable_step_exact_on_quadratics(oracle_lib, steps):
    h0, h1, h2 = steps
    c = oracle.bdf_coefficients(2, h0, h1, h2)
    t1, t0, tm1, tm2 = 0.0, -h0, -h0 - h1, -h0 - h1 - h2
    rng = np.random.default_rng(int(h0 * 1e6))
    for _ in range(4):
        a0, a1, a2 = rng.normal(size=3)
        y = lambda t: a0 + a1 * t + a2 * t * t
        dy = lambda t: a1 + 2 * a2 * t
        # corrector reproduces any quadratic exactly
        assert y(t1) - c.rho1 * y(t0) - c.rho2 * y(tm1) - c.gamma * dy(t1) == pytest.approx(0.0, abs=1e-13)
        # predictor extrapolates any quadratic exactly
        assert c.pi0 * y(t0) + c.pi1 * y(tm1) + c.pi2 * y(tm2) == pytest.approx(y(t1), abs=1e-12)


@pytest.mark.parametrize("steps", [(0.1, 0.1, 0.1), (0.2, 0.1, 0.05), (0.05, 0.1, 0.3), (0.38, 1.0, 1.0)])
def test_milne_estimate_exact_on_cubics(oracle_lib, steps):
    """For x' = g(t) with a cubic solution and exact history, the Milne
    estimate mu (x_corr - x_pred) equals the true local error exactly."""
    h0, h1, h2 = steps
    c = oracle.bdf_coefficients(2, h0, h1, h2)
    t1, t0, tm1, tm2 = 0.0, -h0, -h0 - h1, -h0 - h1 - h2
    rng = np.random.default_rng(17)
    for _ in range(4):
        a = rng.normal(size=4)
        y = lambda t: a[0] + a[1] * t + a[2] * t ** 2 + a[3] * t ** 3
        dy = lambda t: a[1] + 2 * a[2] * t + 3 * a[3] * t ** 2
        x_corr = c.rho1 * y(t0) + c.rho2 * y(tm1) + c.gamma * dy(t1)
        x_pred = c.pi0 * y(t0) + c.pi1 * y(tm1) + c.pi2 * y(tm2)
        true_err = y(t1) - x_corr
        est = c.mu * (x_corr - x_pred)
        assert est == pytest.approx(true_err, rel=1e-9, abs=1e-15)


def test_bdf1_milne_exact_on_quadratics(oracle_lib):
    h = 0.3
    c = oracle.bdf_coefficients(1, h)
    for a in np.random.default_rng(4).normal(size=(4, 3)):
        y = lambda t: a[0] + a[1] * t + a[2] * t * t
        dy = lambda t: a[1] + 2 * a[2] * t
        x_corr = y(-h) + h * dy(0.0)
        x_pred = y(-h) + h * dy(-h)
        assert c.mu * (x_corr - x_pred) == pytest.approx(y(0.0) - x_corr, rel=1e-12, abs=1e-15)


# --------------------------------------------------------------- substep grid
def _cfg(w):
    return oracle.make_config(w)


def test_uniform_grid_and_cold_start(oracle_lib):
    w = W.linear2(N=4, T=3)
    tab, S, depth = oracle.build_substeps(_cfg(w), 0.0, 0.1, 0, 0.0, 0.0)
    assert S == 20 and depth == 2
    kinds = [tab[i].kind for i in range(S)]
    assert kinds[:2] == [1, 1] and all(k == 2 for k in kinds[2:])
    hs = np.array([tab[i].h for i in range(S)])
    assert hs.sum() == pytest.approx(0.1, rel=1e-15)
    assert np.allclose(hs, 0.005, rtol=1e-12)
    # the next interval continues the history: all BDF2
    tab, S, depth = oracle.build_substeps(_cfg(w), 0.1, 0.2, 2, hs[-1], hs[-2])
    assert all(tab[i].kind == 2 for i in range(S))
    # a non-integer substep count is rejected
    with pytest.raises(ValueError):
        oracle.build_substeps(_cfg(w), 0.1, 0.1013, 2, hs[-1], hs[-2])


def test_geometric_grid(oracle_lib):
    w = W.robertson(N=4, T=3)
    t = w.t_obs
    tab, S, depth = oracle.build_substeps(_cfg(w), t[0], t[1], 2, 1e-6, 1e-6)
    hs = np.array([tab[i].h for i in range(S)])
    assert S == 50
    assert hs.sum() == pytest.approx(t[1] - t[0], rel=1e-13)
    ratios = hs[1:] / hs[:-1]
    q = (t[1] / t[0]) ** (1 / 50)
    assert np.allclose(ratios, q, rtol=1e-9)
    # first interval from t = 0 uses q0 and ends exactly at t_1
    tab, S, depth = oracle.build_substeps(_cfg(w), 0.0, t[0], 0, 0.0, 0.0)
    hs0 = np.array([tab[i].h for i in range(S)])
    assert hs0.sum() == pytest.approx(t[0], rel=1e-13)
    assert np.allclose(hs0[1:] / hs0[:-1], w.q0, rtol=1e-9)


def test_large_step_ratio_forces_cold_start(oracle_lib):
    w = W.linear2(N=4, T=3)
    # previous steps of 0.001, new steps of 0.005: ratio 5 >= 2
    tab, S, _ = oracle.build_substeps(_cfg(w), 0.0, 0.1, 2, 0.001, 0.001)
    assert [tab[i].kind for i in range(3)] == [1, 1, 2]


def test_restart_history_mode(oracle_lib):
    w = W.linear2(N=8, T=3).with_(history=W.HIST_RESTART)
    f = oracle.Filter(w)
    f.init()
    f.epoch(w.t_obs[0], w.y_obs[0])
    tab, S = f.substeps(w.t_obs[1])
    assert [tab[i].kind for i in range(3)] == [1, 1, 2]


# ----------------------------------------------------------------- propagation
def _propagate_truth(w, K, substep_scale=1):
    cfg = _cfg(w)
    if w.spacing == W.SPACING_UNIFORM:
        cfg.dt = w.dt / substep_scale
    else:
        cfg.substeps = w.substeps * substep_scale
        cfg.q0 = w.q0 ** (1.0 / substep_scale)
    x = np.array(w.x0, dtype=float)
    h1, h2 = x.copy(), x.copy()
    depth, hp1, hp2, t = 0, 0.0, 0.0, w.t0
    out = []
    for k in range(w.T):
        tab, S, dout = oracle.build_substeps(cfg, t, w.t_obs[k], depth, hp1, hp2)
        x, h1, h2, _ = oracle.propagate(w.ode, K, w.theta_true, tab, S, x, h1, h2)
        hp1, hp2 = tab[S - 1].h, (tab[S - 2].h if S >= 2 else hp1)
        depth, t = dout, w.t_obs[k]
        out.append(x.copy())
    return np.array(out)


def test_bdf2_linear_second_order_convergence(oracle_lib):
    w = W.linear2(N=4, T=10)
    exact = W.linear2_exact(w.theta_true, w.x0, w.t_obs)
    errs = []
    for scale in [1, 2, 4, 8]:
        traj = _propagate_truth(w, 1, scale)
        errs.append(np.max(np.abs(traj[-1] - exact[-1])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - 2.0) < 0.15), (errs, orders)


def test_bdf2_linear_matches_recurrence(oracle_lib):
    """For linear f one Newton step solves (I - gamma A) x_{n+1} = rho1 x_n + rho2 x_{n-1}."""
    th = np.array([1.0, 1000.0])
    A = np.array([[-th[0], th[1]], [0.0, -th[1]]])
    rng = np.random.default_rng(9)
    x, h1, h2 = rng.normal(size=2), rng.normal(size=2), rng.normal(size=2)
    tab = (oracle.Substep * 1)()
    tab[0] = oracle.bdf_coefficients(2, 0.004, 0.005, 0.006)
    c = tab[0]
    xn, _, _, _ = oracle.propagate(oracle.LINEAR2, 1, th, tab, 1, x, h1, h2)
    ref = np.linalg.solve(np.eye(2) - c.gamma * A, c.rho1 * x + c.rho2 * h1)
    assert np.allclose(xn, ref, rtol=1e-13, atol=1e-15)


def test_bdf2_stiff_decay_stays_bounded(oracle_lib):
    # h * theta2 = 5: the stiff mode must be damped, not amplified (A-stability)
    w = W.linear2(N=4, T=50)
    traj = _propagate_truth(w, 1)
    exact = W.linear2_exact(w.theta_true, w.x0, w.t_obs)
    assert np.max(np.abs(traj - exact)) < 1e-3
    assert np.all(np.abs(traj[:, 1]) < 1e-6)


def test_robertson_mass_invariant(oracle_lib):
    w = W.robertson(N=4, T=40)
    traj = _propagate_truth(w, w.newton_iters)
    steps = 40 * 50
    assert np.max(np.abs(traj.sum(axis=1) - 1.0)) <= 1e-14 * steps
    # and the trajectory follows the reference solution
    assert np.max(np.abs(traj - w.x_true)) < 1e-3


@pytest.mark.parametrize("name", ["linear2", "robertson", "brusselator"])
def test_chosen_newton_count_is_converged(oracle_lib, name):
    w = W.get(name, N=4)
    if name == "brusselator":
        w = w.with_(t_obs=w.t_obs[:8], y_obs=w.y_obs[:8], x_true=w.x_true[:8])
    a = _propagate_truth(w, w.newton_iters)
    b = _propagate_truth(w, 10)
    dev = np.max(np.abs(a - b) / np.max(np.abs(b), axis=1, keepdims=True))
    assert dev < 1e-12


def test_milne_error_sum_tracks_true_local_error(oracle_lib):
    """On the linear system the summed squared Milne estimates approximate the
    summed squared true local errors (exact history each step)."""
    th = np.array([1.0, 3.0])
    A = np.array([[-th[0], th[1]], [0.0, -th[1]]])
    from scipy.linalg import expm
    h = 0.01
    x0 = np.array([1.0, 1.0])
    ts = [-2 * h, -h, 0.0]
    hist = [expm(A * (t + 1.0)) @ x0 for t in ts]
    tab = (oracle.Substep * 1)()
    tab[0] = oracle.bdf_coefficients(2, h, h, h)
    _, _, _, E = oracle.propagate(oracle.LINEAR2, 1, th, tab, 1, hist[2], hist[1], hist[0], with_error=True)
    xn, _, _, _ = oracle.propagate(oracle.LINEAR2, 1, th, tab, 1, hist[2], hist[1], hist[0])
    true = expm(A * (h + 1.0)) @ x0 - xn
    assert np.allclose(np.sqrt(E), np.abs(true), rtol=0.2)


# ------------------------------------------------------------------ resampling
def _definition_indices(c, u):
    N = len(c)
    out = []
    for i in range(N):
        tau = (float(i) + u) / float(N) * c[-1]
        ks = [k for k in range(N) if c[k] > tau]
        out.append(ks[0] if ks else next(k for k in range(N) if c[k] == c[-1]))
    return np.array(out)


def test_resample_brute_force(oracle_lib):
    rng = np.random.default_rng(21)
    for N in range(1, 9):
        for _ in range(40):
            g = rng.random(N)
            g[rng.random(N) < 0.3] = 0.0
            if g.sum() == 0:
                g[rng.integers(N)] = 1.0
            c = np.cumsum(g)
            u = rng.random()
            assert np.array_equal(oracle.resample_systematic(c, u), _definition_indices(c, u))
    # u at the extremes of its range
    c = np.cumsum([0.5, 0.0, 0.5])
    for u in [0.0, 1.0 - 2.0 ** -53]:
        assert np.array_equal(oracle.resample_systematic(c, u), _definition_indices(c, u))


def test_resample_equal_weights_identity(oracle_lib):
    for N in [1, 2, 8, 1024]:
        c = np.cumsum(np.ones(N))
        for u in [0.0, 0.3, 0.999]:
            assert np.array_equal(oracle.resample_systematic(c, u), np.arange(N))


def test_resample_offspring_counts(oracle_lib):
    rng = np.random.default_rng(8)
    N = 500
    g = rng.gamma(0.5, size=N)
    g[::7] = 0.0
    c = np.cumsum(g)
    p = g / g.sum()
    mean_counts = np.zeros(N)
    R = 400
    for r in range(R):
        idx = oracle.resample_systematic(c, rng.random())
        counts = np.bincount(idx, minlength=N)
        assert np.all(counts >= np.floor(N * p) - 1) and np.all(counts <= np.ceil(N * p) + 1)
        assert np.all(counts[g == 0] == 0)
        assert np.all(np.diff(idx) >= 0)
        mean_counts += counts / R
    assert np.max(np.abs(mean_counts - N * p)) < 0.1


# ---------------------------------------------------------------- Liu-West
def test_liu_west_shrink_moments(oracle_lib):
    rng = np.random.default_rng(12)
    N, p, a = 400, 3, 0.93
    phi = rng.normal(size=(N, p)) @ np.array([[1.0, 0.2, 0.0], [0.0, 0.5, 0.1], [0.0, 0.0, 2.0]])
    w = rng.random(N)
    w /= w.sum()
    mean = w @ phi
    C = (phi - mean).T @ ((phi - mean) * w[:, None])
    shr = np.array([oracle.liu_west_shrink(a, phi[n], mean) for n in range(N)])
    mean_s = w @ shr
    C_s = (shr - mean_s).T @ ((shr - mean_s) * w[:, None])
    assert np.allclose(mean_s, mean, rtol=1e-13, atol=1e-14)
    assert np.allclose(C_s, a * a * C, rtol=1e-12, atol=1e-14)
    # with the kernel variance s^2 C, s^2 = 1 - a^2, the total covariance is C again
    assert np.allclose(C_s + (1 - a * a) * C, C, rtol=1e-12)


def test_cholesky_psd(oracle_lib):
    rng = np.random.default_rng(13)
    B = rng.normal(size=(3, 3))
    C = B @ B.T + 0.1 * np.eye(3)
    L = oracle.cholesky_psd(C)
    assert np.allclose(L, np.linalg.cholesky(C), rtol=1e-13)
    assert np.allclose(oracle.cholesky_psd(np.zeros((3, 3))), 0.0)
    v = rng.normal(size=3)
    R1 = np.outer(v, v)          # rank one
    L1 = oracle.cholesky_psd(R1)
    assert np.allclose(L1 @ L1.T, R1, atol=1e-12)


# -------------------------------------------------------------- the filter
def test_init_draws_prior(oracle_lib):
    w = W.robertson(N=4000, T=2)
    f = oracle.Filter(w)
    f.init()
    st = f.state()
    lo, hi = np.log(w.prior_lo), np.log(w.prior_hi)
    assert np.all(st["phi"] >= lo) and np.all(st["phi"] <= hi)
    from scipy import stats
    for i in range(3):
        assert stats.kstest((st["phi"][:, i] - lo[i]) / (hi[i] - lo[i]), "uniform").pvalue > 1e-3
    assert np.allclose(st["lw"], -np.log(4000))
    assert np.all(st["x"] == w.x0) and np.all(st["h1"] == w.x0)
    m = f.moments()
    assert np.allclose(m["phibar"], st["phi"].mean(axis=0), rtol=1e-12)
    assert np.allclose(m["C"], np.cov(st["phi"].T, bias=True), rtol=1e-10)
    assert m["ess"] == pytest.approx(4000, rel=1e-12)


def test_uniform_prior_identity_transform(oracle_lib):
    w = W.brusselator(N=300, T=2).with_(transform=W.TRANSFORM_IDENTITY)
    f = oracle.Filter(w)
    f.init()
    phi = f.state()["phi"]
    assert np.all(phi >= np.array(w.prior_lo)) and np.all(phi <= np.array(w.prior_hi))


def test_deterministic_special_case(oracle_lib):
    """a = 1 (no shrink, s = 0), kappa = 0 (no innovation) and a point-mass
    prior: every particle follows the plain BDF2 solution, and xbar equals it."""
    w = W.robertson(N=16, T=6)
    th = w.theta_true
    w = w.with_(a=1.0, kappa=0.0, prior_lo=list(th), prior_hi=list(th))
    f = oracle.Filter(w)
    f.init()
    ref = _propagate_truth(w, w.newton_iters)
    for k in range(w.T):
        assert f.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
        m = f.moments()
        st = f.state()
        assert np.allclose(st["x"], ref[k][None, :], rtol=0, atol=1e-15)
        assert np.allclose(m["xbar"], ref[k], rtol=1e-14, atol=1e-18)
        assert np.allclose(m["C"], 0.0)


def test_single_particle(oracle_lib):
    w = W.linear2(N=1, T=5)
    f = oracle.Filter(w)
    f.init()
    for k in range(w.T):
        assert f.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
        assert np.array_equal(f.work()["idx"], [0])
        assert f.state()["lw"][0] == 0.0


def test_degenerate_epoch_leaves_state_unchanged(oracle_lib):
    w = W.linear2(N=32, T=3)
    f = oracle.Filter(w)
    f.init()
    st = f.state()
    bad = {k: v.copy() for k, v in st.items()}
    bad["x"][:] = np.nan
    f.set_state(**bad)
    assert f.epoch(w.t_obs[0], w.y_obs[0]) == oracle.ERR_DEGENERATE
    after = f.state()
    assert np.all(np.isnan(after["x"])) and np.array_equal(after["phi"], st["phi"])
    assert f.history()["epoch"] == 0
    assert f.epoch(w.t_obs[0], [np.nan]) == oracle.ERR_ARG


def test_zero_weight_particle_never_selected(oracle_lib):
    w = W.linear2(N=64, T=3)
    f = oracle.Filter(w)
    f.init()
    st = f.state()
    st["x"][5] = np.nan           # particle 5 fails: weight zero
    f.set_state(**st)
    assert f.epoch(w.t_obs[0], w.y_obs[0]) == oracle.OK
    assert 5 not in set(f.work()["idx"].tolist())
    assert np.all(np.isfinite(f.moments()["phibar"]))


def test_posterior_concentrates_near_truth(oracle_lib):
    w = W.robertson(N=2048, T=40)
    f = oracle.Filter(w)
    f.init()
    for k in range(w.T):
        assert f.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
    m = f.moments()
    th = np.exp(m["phibar"])
    assert np.all(np.abs(np.log(th / w.theta_true)) < 0.1)


def test_staged_epoch_equals_full_epoch(oracle_lib):
    w = W.robertson(N=256, T=3)
    f1, f2 = oracle.Filter(w), oracle.Filter(w)
    f1.init(); f2.init()
    for k in range(w.T):
        assert f1.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
        tab, S = f2.substeps(w.t_obs[k])
        f2.stage1(tab, S, w.y_obs[k])
        assert f2.cumulative() == oracle.OK
        idx = oracle.resample_systematic(f2.work()["c"], f2.resample_u())
        f2.stage2(tab, S, w.y_obs[k], idx)
        assert f2.commit(w.t_obs[k]) == oracle.OK
    s1, s2 = f1.state(), f2.state()
    for key in s1:
        assert np.array_equal(s1[key], s2[key])
