"""Pins of the oracle's BDF3, Adams-Moulton and Adams-Bashforth integrators
(the first three methods of each family, Sec. 3, Tables 1-2) and of the
paper's M1 Michaelis-Menten system (Sec. 2.1), against facts the oracle does
not compute: textbook coefficients and error constants, exactness on
polynomials, convergence orders against a closed form, the stability of each
family on a stiff decay, a steady state, finite differences and an
independent restatement of the right-hand side."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1411_1702_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ADAMS = [oracle.LMM_AM1, oracle.LMM_AM2, oracle.LMM_AM3, oracle.LMM_AB1, oracle.LMM_AB2,
         oracle.LMM_AB3]
ALL_NEW = [oracle.LMM_BDF3] + ADAMS


def _textbook():
    out = {}
    with open(os.path.join(GOLDEN, "lmm_textbook.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, w, c = line.split()
            out[name] = ([float(Fraction(v)) for v in w.split(",")], float(Fraction(c)))
    return out


def test_coefficients_match_textbook(oracle_lib):
    """The oracle derives the weights by integrating (Adams) or differentiating
    (BDF) Lagrange polynomials; they must equal the textbook tables, and
    Milne's factor must follow from the textbook error constants."""
    tb = _textbook()
    h = 0.37
    for q in (1, 2, 3):
        ab, cab = tb[f"AB{q}"]
        am, cam = tb[f"AM{q}"]
        for kind, fam in ((20 + q, "AB"), (10 + q, "AM")):
            s = oracle.lmm_coefficients(kind, h)
            assert np.allclose(list(s.bab)[:q], h * np.array(ab), rtol=1e-14, atol=0)
            assert np.allclose(list(s.beta)[:q], h * np.array(am), rtol=1e-14, atol=0)
            assert s.gamma == pytest.approx(h * am[0], rel=1e-14)
            # Milne's device from the textbook constants
            mu = cam / (cab - cam) if fam == "AM" else cab / (cab - cam)
            assert s.mu == pytest.approx(mu, rel=1e-12), (kind, s.mu, mu)
    w, c = tb["BDF3"]
    s = oracle.lmm_coefficients(3, h)
    assert [s.rho1, s.rho2, s.rho3] == pytest.approx(w[:3], rel=1e-14)
    assert s.gamma == pytest.approx(h * w[3], rel=1e-14)
    # Hermite predictor through x_n, x_{n-1}, x_{n-2} with slope f_n: a cubic;
    # its error constant, by Taylor expansion about t_{n+1}, is 1/4
    assert s.mu == pytest.approx(c / (0.25 - c), rel=1e-12)


def _poly(a):
    y = np.polynomial.Polynomial(a)
    return y, y.deriv()


@pytest.mark.parametrize("q", [1, 2, 3])
def test_adams_exact_on_polynomials_and_milne(oracle_lib, q):
    """On x' = g(t) with a polynomial solution and exact history: AB_q and AM_q
    reproduce every polynomial of degree <= q; on degree q + 1 (constant
    (q+1)-th derivative) Milne's estimate equals the true local error."""
    h = 0.21
    rng = np.random.default_rng(q)
    am = oracle.lmm_coefficients(10 + q, h)
    ab = oracle.lmm_coefficients(20 + q, h)
    for deg in range(q + 2):
        y, dy = _poly(rng.normal(size=deg + 1))
        xn = y(-h)
        x_pred = xn + sum(ab.bab[j] * dy(-(j + 1) * h) for j in range(q))
        x_corr = xn + sum(am.beta[j] * dy(-j * h) for j in range(q))
        if deg <= q:
            assert x_pred == pytest.approx(y(0.0), rel=1e-12, abs=1e-13)
            assert x_corr == pytest.approx(y(0.0), rel=1e-12, abs=1e-13)
        else:
            assert abs(y(0.0) - x_pred) > 1e-6 and abs(y(0.0) - x_corr) > 1e-6
            est_am = am.mu * (x_corr - x_pred)
            est_ab = ab.mu * (x_corr - x_pred)
            assert est_am == pytest.approx(y(0.0) - x_corr, rel=1e-9)
            assert est_ab == pytest.approx(y(0.0) - x_pred, rel=1e-9)


def test_bdf3_exact_on_cubics_and_milne(oracle_lib):
    h = 0.13
    c = oracle.lmm_coefficients(3, h)
    rng = np.random.default_rng(33)
    for deg in range(5):
        y, dy = _poly(rng.normal(size=deg + 1))
        x_corr = c.rho1 * y(-h) + c.rho2 * y(-2 * h) + c.rho3 * y(-3 * h) + c.gamma * dy(0.0)
        x_pred = c.pi0 * y(-h) + c.pi1 * y(-2 * h) + c.pi2 * y(-3 * h) + c.pi3 * dy(-h)
        if deg <= 3:
            assert x_corr == pytest.approx(y(0.0), rel=1e-12, abs=1e-13)
            assert x_pred == pytest.approx(y(0.0), rel=1e-12, abs=1e-13)
        else:
            assert c.mu * (x_corr - x_pred) == pytest.approx(y(0.0) - x_corr, rel=1e-9)


def test_order_ramp_after_cold_start(oracle_lib):
    w = W.linear2(N=4, T=3)
    cases = {oracle.LMM_BDF3: [1, 1, 3, 3], oracle.LMM_AM3: [11, 12, 13, 13],
             oracle.LMM_AM2: [11, 12, 12, 12], oracle.LMM_AB3: [21, 22, 23, 23],
             oracle.LMM_AB1: [21, 21, 21, 21]}
    for lmm, kinds in cases.items():
        cfg = oracle.make_config(w.with_(lmm=lmm))
        tab, S, depth = oracle.build_substeps(cfg, 0.0, 0.1, 0, 0.0, 0.0)
        assert [tab[i].kind for i in range(4)] == kinds
        assert depth == 2
        # a carried history runs at full order from the first substep
        tab, S, _ = oracle.build_substeps(cfg, 0.1, 0.2, 2, 0.005, 0.005)
        assert {tab[i].kind for i in range(S)} == {kinds[-1]}
        assert tab[0].tn == 0.1 and tab[S - 1].t == 0.2
    # the higher-order families are built for uniform steps only
    cfg = oracle.make_config(W.robertson(N=4, T=2).with_(lmm=oracle.LMM_AM2))
    with pytest.raises(ValueError):
        oracle.build_substeps(cfg, 1e-4, 2e-4, 2, 1e-6, 1e-6)


def _run_linear(lmm, theta, h, t_end, K=1):
    """Propagate x' = A x from exact history at t = 0, -h, -2h to t_end."""
    from scipy.linalg import expm
    A = np.array([[-theta[0], theta[1]], [0.0, -theta[1]]])
    x0 = np.array([1.0, 1.0])
    w = W.linear2(N=4, T=1).with_(lmm=lmm, dt=h)
    cfg = oracle.make_config(w)
    tab, S, _ = oracle.build_substeps(cfg, 0.0, t_end, 2, h, h)
    x, h1, h2 = x0, expm(-h * A) @ x0, expm(-2 * h * A) @ x0
    x, _, _, _ = oracle.propagate(oracle.LINEAR2, K, np.asarray(theta, float), tab, S, x, h1, h2)
    return x, expm(t_end * A) @ x0


@pytest.mark.parametrize("lmm,q", [(oracle.LMM_BDF3, 3), (oracle.LMM_AM1, 1), (oracle.LMM_AM2, 2),
                                   (oracle.LMM_AM3, 3), (oracle.LMM_AB1, 1), (oracle.LMM_AB2, 2),
                                   (oracle.LMM_AB3, 3)])
def test_convergence_order_on_linear_closed_form(oracle_lib, lmm, q):
    errs = []
    for h in (0.04, 0.02, 0.01, 0.005):
        x, ex = _run_linear(lmm, (1.0, 2.5), h, 1.0)
        errs.append(np.max(np.abs(x - ex)))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - q) < 0.2), (errs, orders)


def test_stiff_decay_stability(oracle_lib):
    """h theta2 = 5 on the stiff linear system: every Adams-Bashforth method
    amplifies the stiff mode (its stability region misses -5), while BDF1-3,
    AM1 (backward Euler) and AM2 (trapezoid, A-stable) damp it."""
    for lmm in (oracle.LMM_AB1, oracle.LMM_AB2, oracle.LMM_AB3):
        x, _ = _run_linear(lmm, (1.0, 1000.0), 0.005, 1.0)
        assert not np.all(np.abs(x) < 1e3)
    for lmm in (oracle.LMM_BDF1, oracle.LMM_BDF2, oracle.LMM_BDF3, oracle.LMM_AM1, oracle.LMM_AM2):
        x, ex = _run_linear(lmm, (1.0, 1000.0), 0.005, 1.0)
        assert np.max(np.abs(x - ex)) < 5e-3, (lmm, x, ex)


@pytest.mark.parametrize("lmm", ALL_NEW)
def test_carried_history_equals_one_interval(oracle_lib, lmm):
    """Splitting an interval in two with the history carried gives the same
    states: the derivative history of the Adams methods is rebuilt from the
    stored states exactly as it was carried (same theta, autonomous f)."""
    th = np.array([1.0, 2.5])
    w = W.linear2(N=4, T=1).with_(lmm=lmm, dt=0.01)
    cfg = oracle.make_config(w)
    x0 = np.array([1.0, 0.5])
    tab, S, d1 = oracle.build_substeps(cfg, 0.0, 0.4, 0, 0.0, 0.0)
    xa, _, _, Ea = oracle.propagate(oracle.LINEAR2, 1, th, tab, S, x0, x0, x0, with_error=True)
    tab, S, d1 = oracle.build_substeps(cfg, 0.0, 0.2, 0, 0.0, 0.0)
    x, h1, h2, E1 = oracle.propagate(oracle.LINEAR2, 1, th, tab, S, x0, x0, x0, with_error=True)
    tab, S, _ = oracle.build_substeps(cfg, 0.2, 0.4, d1, tab[S - 1].h, tab[S - 2].h)
    xb, _, _, E2 = oracle.propagate(oracle.LINEAR2, 1, th, tab, S, x, h1, h2, with_error=True)
    assert np.allclose(xb, xa, rtol=1e-14, atol=1e-16)
    assert np.allclose(E1 + E2, Ea, rtol=1e-12, atol=1e-30)


def test_adams_linear_step_solves_recurrence(oracle_lib):
    """For linear f one Newton iteration of AM_q solves
    (I - gamma A) x_{n+1} = x_n + sum_{j>=1} beta_j A x_{n+1-j} exactly."""
    th = np.array([1.0, 1000.0])
    A = np.array([[-th[0], th[1]], [0.0, -th[1]]])
    rng = np.random.default_rng(12)
    x, h1, h2 = rng.normal(size=2), rng.normal(size=2), rng.normal(size=2)
    tab = (oracle.Substep * 1)()
    tab[0] = oracle.lmm_coefficients(13, 0.004)
    c = tab[0]
    xn, _, _, _ = oracle.propagate(oracle.LINEAR2, 1, th, tab, 1, x, h1, h2)
    rhs = x + c.beta[1] * (A @ x) + c.beta[2] * (A @ h1)
    assert np.allclose(xn, np.linalg.solve(np.eye(2) - c.gamma * A, rhs), rtol=1e-13, atol=1e-15)
    tab[0] = oracle.lmm_coefficients(23, 0.004)
    c = tab[0]
    xn, _, _, _ = oracle.propagate(oracle.LINEAR2, 1, th, tab, 1, x, h1, h2)
    ref = x + c.bab[0] * (A @ x) + c.bab[1] * (A @ h1) + c.bab[2] * (A @ h2)
    assert np.allclose(xn, ref, rtol=1e-13, atol=1e-15)


# ------------------------------------------------------------------------ M1
def test_mm_input_and_constants(oracle_lib):
    k = oracle.mm_constants()
    assert k == W.MM_KNOWN
    assert oracle.mm_input(0.0) == k["A0"] and oracle.mm_input(k["t0"]) == k["A0"]
    for t in (0.7, 3.0, 4.5, 20.0):
        s = t - k["t0"]
        assert oracle.mm_input(t) == pytest.approx(k["A0"] + k["A"] * s * np.exp(-s / k["tau"]),
                                                   rel=1e-15)
    # the pulse peaks at t0 + tau with height A tau / e
    ts = np.linspace(0.6, 20.0, 2001)
    v = [oracle.mm_input(t) for t in ts]
    assert ts[int(np.argmax(v))] == pytest.approx(k["t0"] + k["tau"], abs=0.02)


def test_mm_rhs_and_jacobian(oracle_lib):
    rng = np.random.default_rng(8)
    for _ in range(4):
        th = np.exp(rng.uniform(np.log(np.array(W.MM_THETA) / 10), np.log(np.array(W.MM_THETA) * 10)))
        x = rng.uniform(0.05, 3.0, size=3)
        t = rng.uniform(0.0, 25.0)
        f, jac = W.michaelis_rhs(th)
        assert np.allclose(oracle.ode_f(oracle.MICHAELIS, th, x, t), f(t, x), rtol=1e-14, atol=1e-15)
        J = oracle.ode_jac(oracle.MICHAELIS, th, x)
        assert np.allclose(J, jac(t, x), rtol=1e-14, atol=0)
        Jfd = np.zeros((3, 3))
        for j in range(3):
            e = np.zeros(3)
            e[j] = 1e-7 * max(1.0, abs(x[j]))
            Jfd[:, j] = (oracle.ode_f(oracle.MICHAELIS, th, x + e, t) -
                         oracle.ode_f(oracle.MICHAELIS, th, x - e, t)) / (2 * e[j])
        assert np.max(np.abs(J - Jfd)) <= 1e-6 * np.max(np.abs(J))
        # the fluxes cancel in the sum except input and outflow
        assert np.sum(oracle.ode_f(oracle.MICHAELIS, th, x, t)) == pytest.approx(
            oracle.mm_input(t) - W.MM_KNOWN["lam"] * (x[2] - W.MM_KNOWN["c0"]), rel=1e-12)


@pytest.mark.parametrize("lmm", [oracle.LMM_BDF1, oracle.LMM_BDF2, oracle.LMM_BDF3, oracle.LMM_AM1,
                                 oracle.LMM_AM2, oracle.LMM_AM3, oracle.LMM_AB1, oracle.LMM_AB2,
                                 oracle.LMM_AB3])
def test_mm_steady_state_is_kept(oracle_lib, lmm):
    """Under the constant input A0 (t <= t0) the initial state is an
    equilibrium of the true system; every method keeps it (f = 0 exactly
    up to rounding, and all the formulas are consistent)."""
    w = W.michaelis(N=4, T=1, lmm=lmm)
    th = np.array(W.MM_THETA)
    assert np.max(np.abs(oracle.ode_f(oracle.MICHAELIS, th, w.x0, 0.2))) < 1e-15
    cfg = oracle.make_config(w)
    x = np.array(w.x0)
    tab, S, _ = oracle.build_substeps(cfg, 0.0, 0.5, 0, 0.0, 0.0)
    xe, _, _, E = oracle.propagate(oracle.MICHAELIS, w.newton_iters, th, tab, S, x, x, x,
                                   with_error=True)
    assert np.allclose(xe, w.x0, rtol=1e-14, atol=0)
    assert np.all(E < 1e-28)


@pytest.mark.parametrize("lmm,q", [(oracle.LMM_BDF2, 2), (oracle.LMM_BDF3, 3), (oracle.LMM_AM2, 2),
                                   (oracle.LMM_AM3, 3), (oracle.LMM_AB2, 2), (oracle.LMM_AB3, 3)])
def test_mm_converges_to_reference_trajectory(oracle_lib, lmm, q):
    """Against the Radau reference of the input generator: started at t = 1
    (after the input's kink at t0) from exact history, the error at t = 3
    falls with h at the method's order."""
    w = W.michaelis(N=4, T=1, lmm=lmm)
    th = np.array(W.MM_THETA)
    errs = []
    for h in (0.05, 0.025, 0.0125):
        ts = np.array([1.0 - 2 * h, 1.0 - h, 1.0, 3.0])
        ref = W.michaelis_truth(th, w.x0, ts, rtol=1e-12)
        cfg = oracle.make_config(w.with_(dt=h))
        tab, S, _ = oracle.build_substeps(cfg, 1.0, 3.0, 2, h, h)
        x, _, _, _ = oracle.propagate(oracle.MICHAELIS, 8, th, tab, S, ref[2], ref[1], ref[0])
        errs.append(np.max(np.abs(x - ref[3])))
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(orders - q) < 0.3), (errs, orders)


def test_mm_newton_count_is_converged(oracle_lib):
    """K = 4 agrees with fully converged Newton (K = 12) to 1e-12 along the
    reference trajectory for every implicit method."""
    for lmm in (oracle.LMM_BDF1, oracle.LMM_BDF2, oracle.LMM_BDF3, oracle.LMM_AM1, oracle.LMM_AM2,
                oracle.LMM_AM3):
        w = W.michaelis(N=4, T=50, lmm=lmm)
        cfg = oracle.make_config(w)
        res = []
        for K in (w.newton_iters, 12):
            x = np.array(w.x0)
            h1, h2 = x.copy(), x.copy()
            depth, hp1, hp2, t = 0, 0.0, 0.0, 0.0
            out = []
            for k in range(w.T):
                tab, S, dout = oracle.build_substeps(cfg, t, w.t_obs[k], depth, hp1, hp2)
                x, h1, h2, _ = oracle.propagate(w.ode, K, w.theta_true, tab, S, x, h1, h2)
                hp1, hp2, depth, t = tab[S - 1].h, tab[S - 2].h, dout, w.t_obs[k]
                out.append(x.copy())
            res.append(np.array(out))
        assert np.max(np.abs(res[0] - res[1]) / np.abs(res[1])) < 1e-12


@pytest.mark.parametrize("lmm", [oracle.LMM_BDF3, oracle.LMM_AM2, oracle.LMM_AB2])
def test_mm_deterministic_special_case(oracle_lib, lmm):
    """a = 1, kappa = 0, point-mass prior: every particle follows the plain
    solve of the method, and the weighted mean equals it."""
    w = W.michaelis(N=8, T=6, lmm=lmm)
    th = w.theta_true
    w = w.with_(a=1.0, kappa=0.0, prior_lo=list(th), prior_hi=list(th))
    f = oracle.Filter(w)
    f.init()
    cfg = oracle.make_config(w)
    x = np.array(w.x0)
    h1, h2 = x.copy(), x.copy()
    depth, hp1, hp2, t = 0, 0.0, 0.0, 0.0
    for k in range(w.T):
        assert f.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
        tab, S, dout = oracle.build_substeps(cfg, t, w.t_obs[k], depth, hp1, hp2)
        x, h1, h2, _ = oracle.propagate(w.ode, w.newton_iters, th, tab, S, x, h1, h2)
        hp1, hp2, depth, t = tab[S - 1].h, tab[S - 2].h, dout, w.t_obs[k]
        assert np.allclose(f.moments()["xbar"], x, rtol=1e-14, atol=0)
        assert np.allclose(f.state()["x"], x[None, :], rtol=0, atol=1e-15)


def test_mm_posterior_concentrates(oracle_lib):
    """A full run of each family on M1: the weighted mean of theta moves
    from the prior's centre toward theta*, and the state follows the truth."""
    for lmm in (oracle.LMM_BDF2, oracle.LMM_AM3, oracle.LMM_AB3):
        w = W.michaelis(N=3000, T=50, lmm=lmm)
        f = oracle.Filter(w)
        f.init()
        for k in range(w.T):
            assert f.epoch(w.t_obs[k], w.y_obs[k]) == oracle.OK
        m = f.moments()
        # V1/k1 and V2/k2 (the identifiable ratios at these concentrations)
        ratio = np.exp(m["phibar"][[0, 1]] - m["phibar"][[2, 3]])
        true = np.array(W.MM_THETA)[[0, 1]] / np.array(W.MM_THETA)[[2, 3]]
        assert np.all(np.abs(np.log(ratio / true)) < 0.4), (lmm, ratio, true)
        assert np.allclose(m["xbar"], w.x_true[-1], rtol=0.05)
