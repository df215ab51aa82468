// pf_grid.cu -- host-side substep grid and LMM coefficients of one observation
// interval (the fixed, shared step sequence of the paper's Sec. 3.1: every
// particle takes the same steps, so every particle costs the same).
//
// Variable-step BDF2 with ratio w = h_n / h_{n-1} (closed form):
//   x_{n+1} - (1+w)^2/(1+2w) x_n + w^2/(1+2w) x_{n-1} = h_n (1+w)/(1+2w) f_{n+1}.
// Predictor: the quadratic through x_n, x_{n-1}, x_{n-2} evaluated at t_{n+1};
// with a = h_n, b = a + h_{n-1}, c = b + h_{n-2} (distances back from t_{n+1}):
//   pi0 = b c / (h_{n-1} (h_{n-1} + h_{n-2})), pi1 = -a c / (h_{n-1} h_{n-2}),
//   pi2 = a b / ((h_{n-1} + h_{n-2}) h_{n-2}).
// Leading local errors for a solution with constant x''': predictor
// Ep = a b c / 6, corrector Ec = -a^3 (1+w)^2 / (6 w (1+2w)); Milne's device
// estimates the corrector's error as Ec / (Ep - Ec) (x_corr - x_pred)
// (= -2/11 (x_corr - x_pred) at constant step).
// BDF1 (backward Euler, cold starts): gamma = h, estimate -1/2 (x_corr - x_EE)
// against the explicit-Euler predictor x_EE = x_n + h f(x_n).
#include <cmath>

#include "pf_kernels.h"

namespace pfg {

static void bdf2_coefficients(double h0, double h1, double h2, StepCoef& c) {
  const double w = h0 / h1;
  const double den = 1.0 + 2.0 * w;
  c.kind = 2;
  c.h = h0;
  c.rho1 = (1.0 + w) * (1.0 + w) / den;
  c.rho2 = -(w * w) / den;
  c.gamma = h0 * (1.0 + w) / den;
  const double a = h0, b = h0 + h1, cc = h0 + h1 + h2;
  c.pi0 = b * cc / (h1 * (h1 + h2));
  c.pi1 = -(a * cc) / (h1 * h2);
  c.pi2 = a * b / ((h1 + h2) * h2);
  const double ec = -(a * a * a) * (1.0 + w) * (1.0 + w) / (6.0 * w * den);
  const double ep = a * b * cc / 6.0;
  c.mu = ec / (ep - ec);
}

static void bdf1_coefficients(double h0, StepCoef& c) {
  c.kind = 1;
  c.h = h0;
  c.gamma = h0;
  c.rho1 = 1.0;
  c.rho2 = 0.0;
  c.pi0 = 1.0;
  c.pi1 = 0.0;
  c.pi2 = 0.0;
  c.mu = -0.5;
}

// Substep times: uniform, t_prev + i (t_next - t_prev)/S with S = (t_next -
// t_prev)/dt an integer to 1e-9; geometric, t_prev q^i with q =
// (t_next/t_prev)^(1/S), or from t_prev = 0, t_next (q0^i - 1)/(q0^S - 1).  The
// last time is t_next exactly.  depth = stored past points (0..2); BDF2 needs 2;
// a step ratio >= 2 restarts the history (zero-stability of variable BDF2).
int build_substeps(int lmm, int spacing, double dt, int substeps, double q0, double t_prev,
                   double t_next, int depth, double hprev1, double hprev2, StepCoef* tab,
                   int max_steps, int* depth_out) {
  if (!(t_next > t_prev) || !std::isfinite(t_next) || !std::isfinite(t_prev)) return -1;
  if (max_steps > kSMax) max_steps = kSMax;
  double times[kSMax + 1];
  int S;
  if (spacing == PF_SPACING_UNIFORM) {
    if (!(dt > 0.0)) return -1;
    const double ratio = (t_next - t_prev) / dt;
    const double Sr = std::floor(ratio + 0.5);
    if (Sr < 1.0 || std::fabs(ratio - Sr) > 1e-9 * Sr || Sr > (double)max_steps) return -1;
    S = (int)Sr;
    const double h = (t_next - t_prev) / (double)S;
    for (int i = 0; i < S; ++i) times[i] = t_prev + (double)i * h;
  } else if (spacing == PF_SPACING_GEOMETRIC) {
    S = substeps;
    if (S < 1 || S > max_steps) return -1;
    if (t_prev > 0.0) {
      const double q = std::pow(t_next / t_prev, 1.0 / (double)S);
      for (int i = 0; i < S; ++i) times[i] = t_prev * std::pow(q, (double)i);
    } else {
      if (!(q0 > 1.0)) return -1;
      const double den = std::pow(q0, (double)S) - 1.0;
      for (int i = 0; i < S; ++i) times[i] = t_next * ((std::pow(q0, (double)i) - 1.0) / den);
    }
  } else {
    return -1;
  }
  times[S] = t_next;
  if (lmm == PF_LMM_BDF1) depth = 0;
  for (int i = 0; i < S; ++i) {
    const double h0 = times[i + 1] - times[i];
    if (!(h0 > 0.0)) return -1;
    if (depth >= 1 && h0 / hprev1 >= 2.0) depth = 0;
    if (lmm == PF_LMM_BDF2 && depth >= 2) bdf2_coefficients(h0, hprev1, hprev2, tab[i]);
    else bdf1_coefficients(h0, tab[i]);
    tab[i].pad = 0;
    hprev2 = hprev1;
    hprev1 = h0;
    depth = depth < 2 ? depth + 1 : 2;
  }
  if (lmm == PF_LMM_BDF1) depth = 0;
  if (depth_out) *depth_out = depth;
  return S;
}

}  // namespace pfg

extern "C" int pf_substep_table(int lmm, int spacing, double dt, int substeps, double q0,
                                double t_prev, double t_next, int depth, double hprev1,
                                double hprev2, double* coef, int max_steps, int* depth_out) {
  if (!coef || max_steps < 1) return -1;
  static thread_local pfg::StepCoef tab[pfg::kSMax];
  const int S = pfg::build_substeps(lmm, spacing, dt, substeps, q0, t_prev, t_next, depth, hprev1,
                                    hprev2, tab, max_steps, depth_out);
  for (int i = 0; i < S; ++i) {
    const pfg::StepCoef& c = tab[i];
    double* row = coef + 9 * i;
    row[0] = c.kind;
    row[1] = c.h;
    row[2] = c.gamma;
    row[3] = c.rho1;
    row[4] = c.rho2;
    row[5] = c.pi0;
    row[6] = c.pi1;
    row[7] = c.pi2;
    row[8] = c.mu;
  }
  return S;
}
