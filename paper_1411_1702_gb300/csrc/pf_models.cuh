// pf_models.cuh -- the test problems as per-particle device models.
//
// Each model solves the implicit substep equation of the LMM (the paper's
// Sec. 2.1: implicit methods need a Newton-type solve every step)
//     G(y) = y - r - gamma f(y) = 0,
// with r the method's explicit part (rho1 x_n + rho2 x_{n-1} for BDF2); a
// time-dependent input (kForced, added to component 0) is folded into r by
// the caller, so newton() and gf() see only the autonomous part of f.
// by K full Newton iterations (I - gamma J(y)) dy = -G(y) with the analytic
// Jacobian re-evaluated at every iterate.  State, Jacobian and elimination
// live in registers, one particle per thread.  Each elimination below is exact
// Gaussian elimination specialised to the sparsity of I - gamma J; its result
// equals dense partial-pivoting elimination up to rounding.
#pragma once
#include "pf_common.cuh"

namespace pfg {

// x' = A x, A = [[-th1, th2], [0, -th2]].
struct Linear2 {
  static constexpr int D = 2, P = 2, ODE = PF_ODE_LINEAR2;
  static constexpr bool kForced = false;
  struct Th {
    double t1, t2;
  };
  __device__ __forceinline__ static Th theta(const double* t) { return Th{t[0], t[1]}; }

  // gamma f(x)
  __device__ __forceinline__ static void gf(const Th& T, double g, const double* x, double* out) {
    out[0] = g * fma(-T.t1, x[0], T.t2 * x[1]);
    out[1] = -g * T.t2 * x[1];
  }

  // I - gamma A = [[1 + g t1, -g t2], [0, 1 + g t2]] is constant: its two
  // pivots are inverted once per substep (J does not depend on y).
  __device__ __forceinline__ static void newton(const Th& T, double g, const double* r, double* y,
                                                int K) {
    const double gt1 = g * T.t1, gt2 = g * T.t2;
    const double o1 = 1.0 + gt1, o2 = 1.0 + gt2;
    // two refinement steps: with K = 1 no later iteration absorbs the
    // reciprocal's error
    const double i1 = rcp_nr2(o1), i2 = rcp_nr2(o2);
    for (int it = 0; it < K; ++it) {
      // G = (I - g A) y - r, each row one FMA chain on the pivots
      const double G0 = fma(-gt2, y[1], fma(o1, y[0], -r[0]));
      const double G1 = fma(o2, y[1], -r[1]);
      const double d1 = -G1 * i2;
      const double d0 = fma(gt2, d1, -G0) * i1;
      y[0] += d0;
      y[1] += d1;
    }
  }
};

// Robertson: y1' = -k1 y1 + k3 y2 y3, y2' = k1 y1 - k3 y2 y3 - k2 y2^2,
// y3' = k2 y2^2.  With q = g k3 y2, p = g k3 y3, w = 2 g k2 y2,
//   M = I - gamma J = [[m11, -p, -q], [-g k1, 1 + p + w, q], [0, -w, 1]],
// m11 = 1 + g k1 >= 1 is the same for every Newton iteration of a substep, so
// it is the elimination pivot of column 1 (no row swap is ever needed):
// with im = 1/m11 and l = g k1 im = 1 - im, row 2 + l row 1 and row 3
// (d3 = w d2 - G3) give
//   (1 + w + im (p + q w)) d2 = -(G2 + l G1) + im q G3,
//   d1 = im (q d3 + p d2 - G1).
// Each correction is formed from quantities on its own scale (y2 and y3 can be
// 1e-9 of y1), and G1 enters y2's equation only through l, as in the exact
// inverse.
struct Robertson {
  static constexpr int D = 3, P = 3, ODE = PF_ODE_ROBERTSON;
  static constexpr bool kForced = false;
  struct Th {
    double k1, k2, k3;
  };
  __device__ __forceinline__ static Th theta(const double* t) { return Th{t[0], t[1], t[2]}; }

  __device__ __forceinline__ static void gf(const Th& T, double g, const double* x, double* out) {
    const double a = g * T.k1 * x[0];
    const double b = g * T.k3 * x[1] * x[2];
    const double c = g * T.k2 * x[1] * x[1];
    out[0] = b - a;
    out[1] = (a - b) - c;
    out[2] = c;
  }

  __device__ __forceinline__ static void newton(const Th& T, double g, const double* r, double* y,
                                                int K) {
    const double gk1 = g * T.k1, gk2 = g * T.k2, gk3 = g * T.k3;
    const double opk1 = 1.0 + gk1;
    const double im = rcp_nr(opk1);
    const double l = gk1 * im;
    // one iteration; the pivot's reciprocal is refined only in the last
    auto step = [&](const bool last) {
      const double q = gk3 * y[1];  // g k3 y2
      const double p = gk3 * y[2];  // g k3 y3
      const double t = gk2 * y[1];  // g k2 y2
      const double w = t + t;       // 2 g k2 y2
      // G = y - r - gamma f(y), the products g k3 y2 y3 = q y3 and
      // g k2 y2^2 = t y2 fused into the sums; the first row's y1 + g k1 y1
      // is one product with the pivot 1 + g k1
      const double G1 = fma(-q, y[2], fma(opk1, y[0], -r[0]));
      const double G2 = fma(-gk1, y[0], fma(q, y[2], fma(t, y[1], y[1] - r[1])));
      const double G3 = fma(-t, y[1], y[2] - r[2]);
      const double den = fma(im, fma(q, w, p), 1.0 + w);
      const double num = fma(q * im, G3, -fma(l, G1, G2));
      const double d2 = num * rcp_newton(den, last);
      const double d3 = fma(w, d2, -G3);
      const double d1 = im * fma(q, d3, fma(p, d2, -G1));
      y[0] += d1;
      y[1] += d2;
      y[2] += d3;
    };
    for (int it = 0; it + 1 < K; ++it) step(false);
    if (K > 0) step(true);
  }
};

// M1 of Sec. 2.1, three compartments with Michaelis-Menten fluxes:
//   x1' = Phi(t) - V1 x1/(x1+k1), x2' = V1 x1/(x1+k1) - V2 x2/(x2+k2),
//   x3' = V2 x2/(x2+k2) - lambda (x3 - c0),  theta = (V1, V2, k1, k2).
// The input Phi(t) is the same for every particle and comes per substep from
// the host (kForced).  lambda and c0 are the known constants of the problem
// (the paper names them without values; lambda = 0.5, c0 = 2 is the reading
// the library is built with).  J is lower triangular,
//   I - gamma J = [[1 + g a, 0, 0], [-g a, 1 + g b, 0], [0, -g b, 1 + g lambda]],
// a = V1 k1/(x1+k1)^2, b = V2 k2/(x2+k2)^2, so each Newton step is a forward
// substitution with one reciprocal per row.
struct Michaelis {
  static constexpr int D = 3, P = 4, ODE = PF_ODE_MICHAELIS3;
  static constexpr bool kForced = true;
  static constexpr double kLambda = 0.5, kC0 = 2.0;
  struct Th {
    double v1, v2, k1, k2;
  };
  __device__ __forceinline__ static Th theta(const double* t) { return Th{t[0], t[1], t[2], t[3]}; }

  // gamma times the autonomous part of f (everything but the input)
  __device__ __forceinline__ static void gf(const Th& T, double g, const double* x, double* out) {
    const double j1 = T.v1 * x[0] * rcp_nr2(x[0] + T.k1);
    const double j2 = T.v2 * x[1] * rcp_nr2(x[1] + T.k2);
    out[0] = -g * j1;
    out[1] = g * (j1 - j2);
    out[2] = g * fma(-kLambda, x[2] - kC0, j2);
  }

  __device__ __forceinline__ static void newton(const Th& T, double g, const double* r, double* y,
                                                int K) {
    const double opl = fma(g, kLambda, 1.0);
    const double gl = rcp_nr2(opl);
    // the fluxes with q = 1/(x + k): g j = g V x q = g V - u, u = (g V k) q,
    // and g a = (g V k) q^2 = u q.  The residual's constant parts, once per
    // substep:
    //   G0 = (y[0] + [g V1 - r[0]]) - u1
    //   G1 = ((y[1] + [g V2 - g V1 - r[1]]) + u1) - u2
    //   G2 = (1 + g lambda) y[2] - [r[2] + g lambda c0 + g V2] + u2
    const double gv1 = g * T.v1, gv2 = g * T.v2;
    const double gv1k1 = gv1 * T.k1, gv2k2 = gv2 * T.k2;
    const double c0 = gv1 - r[0];
    const double c1 = (gv2 - gv1) - r[1];
    const double c2 = -(fma(g * kLambda, kC0, r[2]) + gv2);
    // one iteration; the pivots' reciprocals are refined only in the last.
    // The flux reciprocals enter the residual: the last iteration refines
    // them twice (its residual is the final one), the earlier ones once,
    // since the next iteration's exact residual corrects their step
    auto step = [&](const bool last) {
      const double s1 = y[0] + T.k1, s2 = y[1] + T.k2;
      const double q1 = last ? rcp_nr2(s1) : rcp_nr(s1), q2 = last ? rcp_nr2(s2) : rcp_nr(s2);
      const double u1 = gv1k1 * q1, u2 = gv2k2 * q2;
      const double ga = u1 * q1, gb = u2 * q2;
      // G = y - r - gamma f_aut(y)
      const double G0 = (y[0] + c0) - u1;
      const double G1 = ((y[1] + c1) + u1) - u2;
      const double G2 = fma(opl, y[2], c2) + u2;
      const double d0 = -G0 * rcp_newton(1.0 + ga, last);
      const double d1 = fma(ga, d0, -G1) * rcp_newton(1.0 + gb, last);
      const double d2 = fma(gb, d1, -G2) * gl;
      y[0] += d0;
      y[1] += d1;
      y[2] += d2;
    };
    for (int it = 0; it + 1 < K; ++it) step(false);
    if (K > 0) step(true);
  }
};

}  // namespace pfg
