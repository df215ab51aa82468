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
//
// BDF3 and the Adams methods (the first three of each family, Tables 1-2)
// run at a constant step h with the textbook weights:
//   BDF3  x_{n+1} = (18 x_n - 9 x_{n-1} + 2 x_{n-2})/11 + (6/11) h f_{n+1},
//         error constant -3/22; predictor: the cubic through x_n, x_{n-1},
//         x_{n-2} with slope f_n, -3/2 x_n + 3 x_{n-1} - 1/2 x_{n-2} + 3 h f_n,
//         error constant 1/4; Milne factor (-3/22)/(1/4 + 3/22) = -6/17.
//   AB_q  h (1), h (3/2, -1/2), h (23, -16, 5)/12 on f_n, f_{n-1}, f_{n-2};
//         error constants 1/2, 5/12, 3/8.
//   AM_q  h (1), h (1/2, 1/2), h (5, 8, -1)/12 on f_{n+1}, f_n, f_{n-1};
//         error constants -1/2, -1/12, -1/24.
// AM_q is corrected against AB_q (factor Cc/(Cp - Cc)); an AB_q step is
// itself the predictor and is measured against AM_q evaluated once at the new
// point (factor Cp/(Cp - Cc)).
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

static void bdf3_coefficients(double h, StepCoef& c) {
  c.kind = 3;
  c.h = h;
  c.gamma = 6.0 * h / 11.0;
  c.rho1 = 18.0 / 11.0;
  c.rho2 = -9.0 / 11.0;
  c.rho3 = 2.0 / 11.0;
  c.pi0 = -1.5;
  c.pi1 = 3.0;
  c.pi2 = -0.5;
  c.pi3 = 3.0 * h;
  c.mu = -6.0 / 17.0;
}

// family 1 = Adams-Moulton, 2 = Adams-Bashforth; q = order
static void adams_coefficients(int family, int q, double h, StepCoef& c) {
  static const double ab[3][3] = {{1.0, 0.0, 0.0}, {1.5, -0.5, 0.0}, {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0}};
  static const double am[3][3] = {{1.0, 0.0, 0.0}, {0.5, 0.5, 0.0}, {5.0 / 12.0, 8.0 / 12.0, -1.0 / 12.0}};
  static const double cp[3] = {0.5, 5.0 / 12.0, 3.0 / 8.0};
  static const double cc[3] = {-0.5, -1.0 / 12.0, -1.0 / 24.0};
  const int i = q - 1;
  c.kind = 10 * family + q;
  c.h = h;
  c.pi0 = h * ab[i][0];
  c.pi1 = h * ab[i][1];
  c.pi2 = h * ab[i][2];
  c.gamma = h * am[i][0];
  c.rho1 = h * am[i][1];
  c.rho2 = h * am[i][2];
  c.mu = family == 1 ? cc[i] / (cp[i] - cc[i]) : cp[i] / (cp[i] - cc[i]);
}

bool lmm_known(int lmm) {
  return lmm == PF_LMM_BDF1 || lmm == PF_LMM_BDF2 || lmm == PF_LMM_BDF3 ||
         (lmm >= PF_LMM_AM1 && lmm <= PF_LMM_AM3) || (lmm >= PF_LMM_AB1 && lmm <= PF_LMM_AB3);
}

bool lmm_needs_uniform(int lmm) { return lmm != PF_LMM_BDF1 && lmm != PF_LMM_BDF2; }

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
// last time is t_next exactly.  depth = stored past points (0..2); BDF2 and
// BDF3 need 2, an Adams method of order q runs at order min(q, depth + 1); a
// step ratio >= 2 restarts the history (zero-stability of variable BDF2).
// times_out (optional) receives the S + 1 substep times.
int build_substeps(int lmm, int spacing, double dt, int substeps, double q0, double t_prev,
                   double t_next, int depth, double hprev1, double hprev2, StepCoef* tab,
                   int max_steps, int* depth_out, double* times_out) {
  if (!(t_next > t_prev) || !std::isfinite(t_next) || !std::isfinite(t_prev)) return -1;
  if (!lmm_known(lmm)) return -1;
  if (lmm_needs_uniform(lmm) && spacing != PF_SPACING_UNIFORM) return -1;
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
    StepCoef& c = tab[i];
    c = StepCoef{};
    if (lmm == PF_LMM_BDF2 && depth >= 2) bdf2_coefficients(h0, hprev1, hprev2, c);
    else if (lmm == PF_LMM_BDF3 && depth >= 2) bdf3_coefficients(h0, c);
    else if (lmm / 10 == 1 || lmm / 10 == 2) {
      const int q = lmm % 10;
      adams_coefficients(lmm / 10, depth + 1 < q ? depth + 1 : q, h0, c);
    } else bdf1_coefficients(h0, c);
    hprev2 = hprev1;
    hprev1 = h0;
    depth = depth < 2 ? depth + 1 : 2;
  }
  if (lmm == PF_LMM_BDF1) depth = 0;
  if (depth_out) *depth_out = depth;
  if (times_out)
    for (int i = 0; i <= S; ++i) times_out[i] = times[i];
  return S;
}

}  // namespace pfg

extern "C" int pf_substep_table(int lmm, int spacing, double dt, int substeps, double q0,
                                double t_prev, double t_next, int depth, double hprev1,
                                double hprev2, double* coef, int max_steps, int* depth_out) {
  if (!coef || max_steps < 1) return -1;
  static thread_local pfg::StepCoef tab[pfg::kSMax];
  const int S = pfg::build_substeps(lmm, spacing, dt, substeps, q0, t_prev, t_next, depth, hprev1,
                                    hprev2, tab, max_steps, depth_out, nullptr);
  for (int i = 0; i < S; ++i) {
    const pfg::StepCoef& c = tab[i];
    double* row = coef + PF_SUBSTEP_ROW * i;
    row[0] = c.kind;
    row[1] = c.h;
    row[2] = c.gamma;
    row[3] = c.rho1;
    row[4] = c.rho2;
    row[5] = c.pi0;
    row[6] = c.pi1;
    row[7] = c.pi2;
    row[8] = c.mu;
    row[9] = c.rho3;
    row[10] = c.pi3;
  }
  return S;
}

namespace pfg {
// M1's input (Sec. 2.1), Phi(t) = A0 + A (t - t0)_+ exp(-(t - t0)/tau), with
// the constants the library fixes for the problem (A0 = 1, A = 0.5, t0 = 0.5,
// tau = 4); the same for every particle, so it is tabulated per substep here.
double mm_input(double t) {
  const double A0 = 1.0, A = 0.5, t0 = 0.5, tau = 4.0;
  const double s = t - t0;
  if (!(s > 0.0)) return A0;
  const double pulse = A * s;
  return A0 + pulse * std::exp(-s / tau);
}
}  // namespace pfg
