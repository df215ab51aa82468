"""The stage kernels take a Newton correction's pivot reciprocal unrefined in
every iteration but the last (an inexact Newton step, Sec. 2.1's implicit
LMM solve otherwise).  The argument: the next iteration evaluates the exact
residual, so the first step's error delta * e0 is corrected and only a
second-order term reaches the result.

This checks that argument on the CPU for the Robertson system in FP64: the
kernel's elimination (Gaussian elimination specialised to the sparsity of
I - gamma J) is restated here with the first iteration's reciprocal of the
pivot scaled by (1 + delta), |delta| up to 2^-16 (a wide margin over the
hardware approximation), from predictors 0.1-1 % off the solution, over
the prior's parameter range and the substep sizes of the workload.  After
K = 2 iterations the result must match the same iteration with delta = 0 to
1e-12 of its infinity norm (a hundredfold inside the parity bound of 1e-10)
and every component to 1e-9 of itself, while the same perturbation put in
the last iteration instead must move some component at least a hundred
times more: the early error is absorbed, the last one is not.
"""
import numpy as np


def _f(k, y):
    k1, k2, k3 = k
    a, b, c = k1 * y[0], k3 * y[1] * y[2], k2 * y[1] * y[1]
    return np.array([b - a, a - b - c, c])


def _newton(k, g, r, y, K, delta_first):
    # the kernel's elimination, with the first iteration's pivot reciprocal
    # scaled by (1 + delta_first)
    k1, k2, k3 = k
    gk1, gk2, gk3 = g * k1, g * k2, g * k3
    opk1 = 1.0 + gk1
    im = 1.0 / opk1
    l = gk1 * im
    y = y.copy()
    for it in range(K):
        q, p, t = gk3 * y[1], gk3 * y[2], gk2 * y[1]
        w = t + t
        G1 = opk1 * y[0] - r[0] - q * y[2]
        G2 = y[1] - r[1] + t * y[1] + q * y[2] - gk1 * y[0]
        G3 = y[2] - r[2] - t * y[1]
        den = 1.0 + w + im * (q * w + p)
        num = q * im * G3 - (l * G1 + G2)
        rden = 1.0 / den
        if it == 0:
            rden *= 1.0 + delta_first
        d2 = num * rden
        d3 = w * d2 - G3
        d1 = im * (q * d3 + p * d2 - G1)
        y += np.array([d1, d2, d3])
    return y


def _solution_point(rng, k):
    # a state near the slow manifold: y2 from k1 y1 = k2 y2^2 + k3 y2 y3
    k1, k2, k3 = k
    y1 = rng.uniform(0.3, 1.0)
    y3 = 1.0 - y1
    y2 = (-k3 * y3 + np.sqrt((k3 * y3) ** 2 + 4.0 * k2 * k1 * y1)) / (2.0 * k2)
    return np.array([y1, y2, 1.0 - y1 - y2])


def test_exact_newton_step_matches_residual():
    # the restated elimination is exact Newton: with delta = 0 one iteration
    # from y0 equals y0 - (I - g J(y0))^-1 G(y0) solved by numpy
    rng = np.random.default_rng(5)
    for _ in range(200):
        k = np.array([0.04, 3e7, 1e4]) * 10.0 ** rng.uniform(-1, 1, 3)
        g = 10.0 ** rng.uniform(-6, 0)
        ys = _solution_point(rng, k)
        r = ys - g * _f(k, ys)
        y0 = ys * (1.0 + rng.uniform(-1e-2, 1e-2, 3))
        k1, k2, k3 = k
        J = np.array([[-k1, k3 * y0[2], k3 * y0[1]],
                      [k1, -k3 * y0[2] - 2 * k2 * y0[1], -k3 * y0[1]],
                      [0.0, 2 * k2 * y0[1], 0.0]])
        G = y0 - r - g * _f(k, y0)
        want = y0 - np.linalg.solve(np.eye(3) - g * J, G)
        got = _newton(k, g, r, y0, 1, 0.0)
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def _sample(rng):
    k = np.array([0.04, 3e7, 1e4]) * 10.0 ** rng.uniform(-1, 1, 3)
    g = 10.0 ** rng.uniform(-6, 0)
    ys = _solution_point(rng, k)
    r = ys - g * _f(k, ys)
    y0 = ys * (1.0 + rng.uniform(-1e-2, 1e-2, 3) * 10.0 ** rng.uniform(-1, 0))
    return k, g, r, y0


def test_unrefined_first_reciprocal_is_absorbed_but_last_is_not():
    # per component (y2 is ~1e-5 of y1, so the infinity norm alone would
    # hide it): perturbing the first iteration's reciprocal moves the K = 2
    # result at second order, perturbing the last one's at first order
    rng = np.random.default_rng(1411)
    first_norm = first_comp = last_comp = 0.0
    for _ in range(4000):
        k, g, r, y0 = _sample(rng)
        base = _newton(k, g, r, y0, 2, 0.0)
        y1 = _newton(k, g, r, y0, 1, 0.0)
        for delta in (2.0 ** -16, -(2.0 ** -16)):
            got = _newton(k, g, r, y0, 2, delta)
            first_norm = max(first_norm, np.max(np.abs(got - base)) / np.max(np.abs(base)))
            first_comp = max(first_comp, np.max(np.abs(got - base) / np.abs(base)))
            last = _newton(k, g, r, y1, 1, delta)
            last_comp = max(last_comp, np.max(np.abs(last - base) / np.abs(base)))
    assert first_norm <= 1e-12, first_norm      # the parity metric
    assert first_comp <= 1e-9, first_comp       # every component
    assert last_comp >= 100.0 * first_comp, (last_comp, first_comp)
