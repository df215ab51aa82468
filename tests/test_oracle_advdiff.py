"""Oracle pins of the paper's 2D advection-diffusion system (M2, Sec. 4).

Each pin checks the oracle against something other than itself: the
diagonalisation of circulant matrices by the DFT, conservation of total mass
(1^T ell = 0), SciPy's matrix exponential, NumPy's dense solver, and the
exactness of one Newton step on a linear system."""
import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

THETA = np.array(W.AD_THETA)


def _symbol(nt, theta):
    """Eigenvalues of the M2 operator from the DFT of the first column of the
    circulant difference matrix ell, combined as the paper's L."""
    col = np.zeros(nt)
    col[0], col[1] = 1.0, -1.0             # (ell u)_j = u_j - u_{j-1}
    a = np.fft.fft(col)                    # symbol of ell on exp(2 pi i m j / nt)
    ax, ay = a[None, :], a[:, None]
    k1, k2, k3, c1, c2 = theta
    BtB1 = np.conj(ax) * ax
    BtB2 = np.conj(ay) * ay
    cross = np.conj(ax) * ay + np.conj(ay) * ax
    return -(k1 ** 2 * BtB1 + k1 * k3 * cross + (k2 ** 2 + k3 ** 2) * BtB2) + c1 * ax + c2 * ay


@pytest.mark.parametrize("n", [4, 8, 20])
def test_operator_is_diagonalised_by_the_dft(oracle_lib, n):
    nt = n - 1
    rng = np.random.default_rng(n)
    th = THETA * (1.0 + 0.1 * rng.standard_normal(5))
    J = oracle.ode_jac(oracle.ADVDIFF, th, np.zeros(nt * nt))
    lam = _symbol(nt, th)
    for _ in range(3):
        v = rng.standard_normal((nt, nt))
        ref = np.real(np.fft.ifft2(lam * np.fft.fft2(v))).reshape(-1)
        got = J @ v.reshape(-1)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_rhs_is_the_linear_map_of_its_jacobian(oracle_lib):
    rng = np.random.default_rng(1)
    nt = 7
    x = rng.standard_normal(nt * nt)
    J = oracle.ode_jac(oracle.ADVDIFF, THETA, x)
    f = oracle.ode_f(oracle.ADVDIFF, THETA, x)
    assert np.max(np.abs(J @ x - f)) <= 1e-12 * np.max(np.abs(f))


def test_dimension_rules(oracle_lib):
    assert oracle.ode_check_dim(oracle.ADVDIFF, 361)
    assert oracle.ode_check_dim(oracle.ADVDIFF, 1521)
    assert not oracle.ode_check_dim(oracle.ADVDIFF, 400)     # even side
    assert not oracle.ode_check_dim(oracle.ADVDIFF, 360)
    assert not oracle.ode_check_dim(oracle.ADVDIFF, 47 * 47)  # above the largest grid


def test_total_mass_is_conserved(oracle_lib):
    """1^T ell = 0 in both directions, so 1^T L = 0 and every BDF step keeps
    sum(x): the column sums of J vanish and the propagation preserves the
    total to rounding."""
    w = W.advdiff(n=8, N=4, T=2)
    J = oracle.ode_jac(oracle.ADVDIFF, THETA, w.x0)
    assert np.max(np.abs(J.sum(axis=0))) <= 1e-12 * np.max(np.abs(J))
    cfg = oracle.make_config(w)
    tab, S, _ = oracle.build_substeps(cfg, 0.0, 1.0, 0, 0.0, 0.0)
    x, h1, h2 = w.x0.copy(), w.x0.copy(), w.x0.copy()
    x1, _, _, E = oracle.propagate(oracle.ADVDIFF, 1, THETA, tab, S, x, h1, h2, with_error=True)
    assert abs(x1.sum() - w.x0.sum()) <= 1e-12 * np.abs(w.x0).sum()
    assert np.all(np.isfinite(E)) and np.all(E >= 0.0)


def test_bdf2_second_order_against_the_matrix_exponential(oracle_lib):
    """Slow parameters (theta*/10), so that the modes have not decayed to the
    mean by t = 1 and h lambda is in the asymptotic range."""
    from scipy.linalg import expm
    w = W.advdiff(n=8, N=4, T=1)
    th = THETA / 10.0
    J = oracle.ode_jac(oracle.ADVDIFF, th, w.x0)
    exact = expm(J) @ w.x0
    errs = []
    for h in [0.02, 0.01, 0.005]:
        cfg = oracle.make_config(w)
        cfg.dt = h
        tab, S, _ = oracle.build_substeps(cfg, 0.0, 1.0, 0, 0.0, 0.0)
        x, _, _, _ = oracle.propagate(oracle.ADVDIFF, 1, th, tab, S, w.x0, w.x0, w.x0)
        errs.append(np.max(np.abs(x - exact)))
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < r < 2.3 for r in rates), (errs, rates)


def test_workload_truth_is_the_matrix_exponential(oracle_lib):
    from scipy.linalg import expm
    w = W.advdiff(n=8, N=4, T=3)
    J = oracle.ode_jac(oracle.ADVDIFF, THETA, w.x0)
    for k, t in enumerate(w.t_obs):
        ref = expm(J * t) @ w.x0
        assert np.max(np.abs(w.x_true[k] - ref)) <= 1e-10 * np.max(np.abs(ref))


def test_one_newton_iteration_is_exact(oracle_lib):
    """The system is linear, so K = 1 already solves each BDF step: K = 2
    changes the result only by rounding."""
    w = W.advdiff(n=8, N=4, T=1)
    cfg = oracle.make_config(w)
    tab, S, _ = oracle.build_substeps(cfg, 0.0, 1.0, 0, 0.0, 0.0)
    a, _, _, _ = oracle.propagate(oracle.ADVDIFF, 1, THETA, tab, S, w.x0, w.x0, w.x0)
    b, _, _, _ = oracle.propagate(oracle.ADVDIFF, 2, THETA, tab, S, w.x0, w.x0, w.x0)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_lu_factor_apply_matches_numpy(oracle_lib):
    rng = np.random.default_rng(5)
    n = 40
    A = rng.standard_normal((n, n)) + n * np.eye(n) * 0.1
    bs = [rng.standard_normal(n) for _ in range(3)]
    for b, x in zip(bs, oracle.lu_factor_solve(A, bs)):
        ref = np.linalg.solve(A, b)
        assert np.max(np.abs(x - ref)) <= 1e-11 * np.max(np.abs(ref))
    # a row swap in every column: the permutation must be applied before the
    # forward substitution
    P = np.eye(n)[::-1]
    A2 = P @ np.triu(rng.standard_normal((n, n)) + 5 * np.eye(n))
    b = rng.standard_normal(n)
    x = oracle.lu_factor_solve(A2, [b])[0]
    assert np.max(np.abs(A2 @ x - b)) <= 1e-10 * np.max(np.abs(b))


def test_filter_runs_and_concentrates(oracle_lib):
    """A small M2 filter: finite moments every epoch, and the posterior mean
    moves toward theta* relative to the prior centre."""
    w = W.advdiff(n=8, N=256, T=6, seed=3)
    f = oracle.Filter(w)
    assert f.init() == oracle.OK
    for k in range(w.T):
        assert f.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
        mo = f.moments()
        assert np.all(np.isfinite(mo["phibar"])) and np.all(np.isfinite(mo["C"]))
    prior_sd = (np.array(w.prior_hi) - np.array(w.prior_lo)) / np.sqrt(12.0)
    post_sd = np.sqrt(np.diag(f.moments()["C"]))
    assert np.all(post_sd < prior_sd)
