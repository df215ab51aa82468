/*
 * pf_oracle.c -- plain FP64 CPU oracle of the LMM PF-SMC sampler.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark.  It shares no code with the CUDA library.
 *
 * Paper: Arnold, Calvetti, Somersalo, "Vectorized and Parallel Particle Filter
 * SMC Parameter Estimation for Stiff ODEs" (arXiv 1411.1702), Algorithm 1
 * ("LMM PF-SMC Sampler", Sec. 2) and the remarks on implicit LMMs with a
 * Newton-type solve (Sec. 2.1) and on fixed steps for load balance (Sec. 3.1).
 *
 * Everything is written for clarity: one particle at a time, dense Gaussian
 * elimination for every Newton system, sequential sums.  The particle loops
 * carry an OpenMP pragma only so that the CPU baseline can use all host cores;
 * each particle is independent, so the result does not depend on the thread
 * count.  Build with -ffp-contract=off so that no multiply-add is fused.
 */
#include "pf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Round: two 32x32->64 products of counter words */
/* 0 and 2 with the round multipliers; the new words are                    */
/* (hi1^c1^k0, lo1, hi0^c3^k1, lo0); the key is bumped by the Weyl constants */
/* between rounds.                                                          */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout (reading of the random-number scheme): word 0 = particle
 * slot n, word 1 = epoch, word 2 = purpose | (block << 8), word 3 = filter id.
 * Key = the 64-bit seed split in two 32-bit halves. */
static void draw_block(uint64_t seed, uint32_t stream, int purpose, uint32_t n, uint32_t epoch,
                       uint32_t block, uint32_t out[4]) {
  uint32_t ctr[4] = {n, epoch, (uint32_t)purpose | (block << 8), stream};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* 53-bit uniform in [0,1) from two 32-bit words: 27 high bits of the first
 * and 26 high bits of the second, scaled by 2^-53 (exact in FP64). */
static double uniform53(uint32_t a, uint32_t b) {
  double hi = (double)(a >> 5);
  double lo = (double)(b >> 6);
  return (hi * 67108864.0 + lo) / 9007199254740992.0;
}

/* k-th uniform of a (purpose, n, epoch) stream: block k/2, word pair k%2. */
double or_uniform(uint64_t seed, uint32_t stream, int purpose, uint32_t n, uint32_t epoch, int k) {
  uint32_t w[4];
  draw_block(seed, stream, purpose, n, epoch, (uint32_t)(k / 2), w);
  if (k % 2 == 0) return uniform53(w[0], w[1]);
  return uniform53(w[2], w[3]);
}

/* k-th standard normal: Box-Muller (Box & Muller 1958) on the two uniforms
 * of block k/2; even k takes the cosine branch, odd k the sine branch. */
double or_normal(uint64_t seed, uint32_t stream, int purpose, uint32_t n, uint32_t epoch, int k) {
  uint32_t w[4];
  draw_block(seed, stream, purpose, n, epoch, (uint32_t)(k / 2), w);
  double u1 = uniform53(w[0], w[1]);
  double u2 = uniform53(w[2], w[3]);
  double r = sqrt(-2.0 * log(1.0 - u1));
  double angle = 2.0 * M_PI * u2;
  if (k % 2 == 0) return r * cos(angle);
  return r * sin(angle);
}

/* ------------------------------------------------------------------------ */
/* Test problems x' = f(t, x; theta).                                         */
/*  LINEAR2:    x' = A x, A = [[-th1, th2], [0, -th2]] (eigenvalues -th1, -th2). */
/*  ROBERTSON:  y1' = -k1 y1 + k3 y2 y3, y2' = k1 y1 - k3 y2 y3 - k2 y2^2,      */
/*              y3' = k2 y2^2, theta = (k1, k2, k3).                           */
/*  BRUSSELATOR: 1D reaction-diffusion on 32 interior points xi_i = i/33,      */
/*              Dirichlet u = 1, v = 3 at both ends, theta = (A, B, alpha),    */
/*              u_i' = A + u_i^2 v_i - (B+1) u_i + alpha 33^2 (u_{i-1}-2u_i+u_{i+1}), */
/*              v_i' = B u_i - u_i^2 v_i + alpha 33^2 (v_{i-1}-2v_i+v_{i+1}),  */
/*              state interleaved (u_0, v_0, u_1, v_1, ...).                  */
/*  MICHAELIS:  M1 of Sec. 2.1, three compartments with Michaelis-Menten      */
/*              fluxes and the input Phi(t) = A0 + A (t - t0)_+ e^{-(t-t0)/tau}: */
/*              x1' = Phi(t) - V1 x1/(x1+k1),                                  */
/*              x2' = V1 x1/(x1+k1) - V2 x2/(x2+k2),                           */
/*              x3' = V2 x2/(x2+k2) - lambda (x3 - c0),                        */
/*              theta = (V1, V2, k1, k2).  The paper calls lambda, c0, A0, A,  */
/*              t0, tau known but prints no values; the reading takes          */
/*              lambda = 0.5, c0 = 2, A0 = 1, A = 0.5, t0 = 0.5, tau = 4.      */
/* ------------------------------------------------------------------------ */
#define MM_LAMBDA 0.5
#define MM_C0 2.0
#define MM_A0 1.0
#define MM_A 0.5
#define MM_T0 0.5
#define MM_TAU 4.0
#define BR_POINTS 32
#define BR_UB 1.0
#define BR_VB 3.0

int or_ode_dims(int ode, int* d, int* p) {
  switch (ode) {
    case OR_LINEAR2: *d = 2; *p = 2; return 0;
    case OR_ROBERTSON: *d = 3; *p = 3; return 0;
    case OR_BRUSSELATOR: *d = 2 * BR_POINTS; *p = 3; return 0;
    case OR_ADVDIFF: *d = 0; *p = 5; return 0;
    case OR_MICHAELIS: *d = 3; *p = 4; return 0;
  }
  return -1;
}

void or_mm_constants(double* out6) {
  out6[0] = MM_LAMBDA; out6[1] = MM_C0; out6[2] = MM_A0;
  out6[3] = MM_A; out6[4] = MM_T0; out6[5] = MM_TAU;
}

/* the input function of M1: Phi(t) = A0 + A (t - t0)_+ exp(-(t - t0)/tau) */
double or_mm_input(double t) {
  double s = t - MM_T0;
  if (!(s > 0.0)) return MM_A0;
  return MM_A0 + MM_A * s * exp(-s / MM_TAU);
}

/* side of the M2 grid for state dimension d, or 0 if d is not an odd square */
static int ad_side(int d) {
  for (int nt = 3; nt <= 45; nt += 2)
    if (nt * nt == d) return nt;
  return 0;
}

int or_ode_check_dim(int ode, int d) {
  int dd, p;
  if (or_ode_dims(ode, &dd, &p) != 0) return -1;
  if (ode == OR_ADVDIFF) return ad_side(d) ? 0 : -1;
  return d == dd ? 0 : -1;
}

/* M2 (Sec. 4): the forward difference matrix ell of the paper, (ell u)_j =
 * u_j - u_{j-1} with periodic wrap, and its transpose (ell^T u)_j = u_j -
 * u_{j+1}, applied along one axis of the nt x nt grid stored as
 * U[iy * nt + ix] (x fastest): axis 0 is B1 = I (x) ell (the x direction),
 * axis 1 is B2 = ell (x) I (the y direction). */
static void ad_ell(int nt, int axis, int transpose, const double* u, double* out) {
  for (int iy = 0; iy < nt; ++iy) {
    for (int ix = 0; ix < nt; ++ix) {
      int jx = ix, jy = iy;
      int step = transpose ? 1 : nt - 1; /* +1 or -1 modulo nt */
      if (axis == 0) jx = (ix + step) % nt;
      else jy = (iy + step) % nt;
      out[iy * nt + ix] = u[iy * nt + ix] - u[jy * nt + jx];
    }
  }
}

/* M2 right-hand side f = L U,
 *   L = -{k1^2 B1^T B1 + k1 k3 (B1^T B2 + B2^T B1) + (k2^2 + k3^2) B2^T B2}
 *       + c1 B1 + c2 B2,
 * with theta = (k1, k2, k3, c1, c2) (Sec. 4), each product applied as a
 * composition of the difference operators. */
static void ad_rhs(int d, const double* th, const double* x, double* f) {
  const int nt = ad_side(d);
  const double k1 = th[0], k2 = th[1], k3 = th[2], c1 = th[3], c2 = th[4];
  double* b1 = (double*)malloc(sizeof(double) * (size_t)d * 4);
  double* b2 = b1 + d;
  double* t1 = b2 + d;
  double* t2 = t1 + d;
  ad_ell(nt, 0, 0, x, b1); /* B1 x */
  ad_ell(nt, 1, 0, x, b2); /* B2 x */
  for (int i = 0; i < d; ++i) f[i] = c1 * b1[i] + c2 * b2[i];
  ad_ell(nt, 0, 1, b1, t1); /* B1^T B1 x */
  for (int i = 0; i < d; ++i) f[i] -= k1 * k1 * t1[i];
  ad_ell(nt, 0, 1, b2, t1); /* B1^T B2 x */
  ad_ell(nt, 1, 1, b1, t2); /* B2^T B1 x */
  for (int i = 0; i < d; ++i) f[i] -= k1 * k3 * (t1[i] + t2[i]);
  ad_ell(nt, 1, 1, b2, t1); /* B2^T B2 x */
  for (int i = 0; i < d; ++i) f[i] -= (k2 * k2 + k3 * k3) * t1[i];
  free(b1);
}

void or_ode_f(int ode, int d, const double* th, double t, const double* x, double* f) {
  if (ode == OR_MICHAELIS) {
    double V1 = th[0], V2 = th[1], k1 = th[2], k2 = th[3];
    double flux1 = V1 * x[0] / (x[0] + k1);
    double flux2 = V2 * x[1] / (x[1] + k2);
    f[0] = or_mm_input(t) - flux1;
    f[1] = flux1 - flux2;
    f[2] = flux2 - MM_LAMBDA * (x[2] - MM_C0);
  } else if (ode == OR_ADVDIFF) {
    ad_rhs(d, th, x, f);
  } else if (ode == OR_LINEAR2) {
    f[0] = -th[0] * x[0] + th[1] * x[1];
    f[1] = -th[1] * x[1];
  } else if (ode == OR_ROBERTSON) {
    double k1 = th[0], k2 = th[1], k3 = th[2];
    f[0] = -k1 * x[0] + k3 * x[1] * x[2];
    f[1] = k1 * x[0] - k3 * x[1] * x[2] - k2 * x[1] * x[1];
    f[2] = k2 * x[1] * x[1];
  } else if (ode == OR_BRUSSELATOR) {
    double A = th[0], B = th[1], D = th[2] * 33.0 * 33.0;
    for (int i = 0; i < BR_POINTS; ++i) {
      double u = x[2 * i], v = x[2 * i + 1];
      double ul = (i == 0) ? BR_UB : x[2 * (i - 1)];
      double ur = (i == BR_POINTS - 1) ? BR_UB : x[2 * (i + 1)];
      double vl = (i == 0) ? BR_VB : x[2 * (i - 1) + 1];
      double vr = (i == BR_POINTS - 1) ? BR_VB : x[2 * (i + 1) + 1];
      f[2 * i] = A + u * u * v - (B + 1.0) * u + D * (ul - 2.0 * u + ur);
      f[2 * i + 1] = B * u - u * u * v + D * (vl - 2.0 * v + vr);
    }
  }
}

/* Analytic Jacobian df/dx, row-major d x d.  M2 is linear, J = L: column j
 * is L applied to the j-th unit vector. */
void or_ode_jac(int ode, int d, const double* th, const double* x, double* J) {
  for (int i = 0; i < d * d; ++i) J[i] = 0.0;
  if (ode == OR_MICHAELIS) {
    /* d/dx [V x/(x+k)] = V k/(x+k)^2; the input does not depend on x */
    double V1 = th[0], V2 = th[1], k1 = th[2], k2 = th[3];
    double a = V1 * k1 / ((x[0] + k1) * (x[0] + k1));
    double b = V2 * k2 / ((x[1] + k2) * (x[1] + k2));
    J[0] = -a;
    J[3] = a;  J[4] = -b;
    J[7] = b;  J[8] = -MM_LAMBDA;
  } else if (ode == OR_ADVDIFF) {
    double* e = (double*)calloc((size_t)d * 2, sizeof(double));
    double* col = e + d;
    for (int j = 0; j < d; ++j) {
      e[j] = 1.0;
      ad_rhs(d, th, e, col);
      for (int i = 0; i < d; ++i) J[(size_t)i * d + j] = col[i];
      e[j] = 0.0;
    }
    free(e);
    (void)x;
  } else if (ode == OR_LINEAR2) {
    J[0] = -th[0]; J[1] = th[1];
    J[2] = 0.0;    J[3] = -th[1];
  } else if (ode == OR_ROBERTSON) {
    double k1 = th[0], k2 = th[1], k3 = th[2];
    J[0] = -k1; J[1] = k3 * x[2];                      J[2] = k3 * x[1];
    J[3] = k1;  J[4] = -k3 * x[2] - 2.0 * k2 * x[1];   J[5] = -k3 * x[1];
    J[6] = 0.0; J[7] = 2.0 * k2 * x[1];                J[8] = 0.0;
  } else if (ode == OR_BRUSSELATOR) {
    double B = th[1], D = th[2] * 33.0 * 33.0;
    for (int i = 0; i < BR_POINTS; ++i) {
      double u = x[2 * i], v = x[2 * i + 1];
      int ru = 2 * i, rv = 2 * i + 1;
      J[ru * d + ru] = 2.0 * u * v - (B + 1.0) - 2.0 * D;
      J[ru * d + rv] = u * u;
      J[rv * d + ru] = B - 2.0 * u * v;
      J[rv * d + rv] = -u * u - 2.0 * D;
      if (i > 0) {
        J[ru * d + ru - 2] = D;
        J[rv * d + rv - 2] = D;
      }
      if (i < BR_POINTS - 1) {
        J[ru * d + ru + 2] = D;
        J[rv * d + rv + 2] = D;
      }
    }
  }
}

/* Dense Gaussian elimination with partial pivoting: solve A x = b.
 * Returns 0, or -1 on an exactly singular pivot. */
int or_lu_solve(int n, const double* Ain, const double* bin, double* x) {
  double* A = (double*)malloc(sizeof(double) * ((size_t)n * n + n));
  double* b = A + (size_t)n * n;
  memcpy(A, Ain, sizeof(double) * n * n);
  memcpy(b, bin, sizeof(double) * n);
  for (int k = 0; k < n; ++k) {
    int piv = k;
    double best = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      if (fabs(A[i * n + k]) > best) {
        best = fabs(A[i * n + k]);
        piv = i;
      }
    }
    if (best == 0.0) {
      free(A);
      return -1;
    }
    if (piv != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[k * n + j];
        A[k * n + j] = A[piv * n + j];
        A[piv * n + j] = t;
      }
      double t = b[k]; b[k] = b[piv]; b[piv] = t;
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[i * n + k] / A[k * n + k];
      if (l == 0.0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
      b[i] -= l * b[k];
    }
  }
  for (int i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * x[j];
    x[i] = s / A[i * n + i];
  }
  free(A);
  return 0;
}

/* The same elimination split in two: or_lu_factor overwrites A with the
 * multipliers (below the diagonal) and U, recording the row swap of every
 * column in piv; or_lu_apply then solves for any right-hand side.  Used where
 * one Newton matrix serves many solves (the linear M2 system). */
int or_lu_factor(int n, double* A, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[(size_t)k * n + k]);
    for (int i = k + 1; i < n; ++i) {
      if (fabs(A[(size_t)i * n + k]) > best) {
        best = fabs(A[(size_t)i * n + k]);
        p = i;
      }
    }
    if (best == 0.0) return -1;
    piv[k] = p;
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double t = A[(size_t)k * n + j];
        A[(size_t)k * n + j] = A[(size_t)p * n + j];
        A[(size_t)p * n + j] = t;
      }
    }
    for (int i = k + 1; i < n; ++i) {
      double l = A[(size_t)i * n + k] / A[(size_t)k * n + k];
      A[(size_t)i * n + k] = l;
      if (l == 0.0) continue;
      for (int j = k + 1; j < n; ++j) A[(size_t)i * n + j] -= l * A[(size_t)k * n + j];
    }
  }
  return 0;
}

void or_lu_apply(int n, const double* LU, const int* piv, const double* b, double* x) {
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(y, b, sizeof(double) * n);
  /* the rows were swapped whole (multipliers included), so P b first, then
   * forward substitution with the unit lower factor */
  for (int k = 0; k < n; ++k) {
    if (piv[k] != k) {
      double t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t;
    }
  }
  for (int k = 0; k < n; ++k)
    for (int i = k + 1; i < n; ++i) y[i] -= LU[(size_t)i * n + k] * y[k];
  for (int i = n - 1; i >= 0; --i) {
    double s = y[i];
    for (int j = i + 1; j < n; ++j) s -= LU[(size_t)i * n + j] * x[j];
    x[i] = s / LU[(size_t)i * n + i];
  }
  free(y);
}

/* ------------------------------------------------------------------------ */
/* LMM coefficients on a variable grid (Sec. 2.1: implicit BDF methods).      */
/* Nodes are measured from t_{n+1}: s_0 = 0, s_1 = -h0, s_2 = -(h0 + h1),     */
/* s_3 = -(h0 + h1 + h2), with h0 = t_{n+1} - t_n and h1, h2 the previous      */
/* steps.  BDF(k) is "the derivative at t_{n+1} of the polynomial through     */
/* x_{n+1}, ..., x_{n+1-k} equals f(x_{n+1})".                                 */
/* ------------------------------------------------------------------------ */

/* derivative at 0 of the j-th Lagrange basis polynomial on nodes s[0..m-1] */
static double lagrange_dbasis_at0(const double* s, int m, int j) {
  double total = 0.0;
  for (int q = 0; q < m; ++q) {
    if (q == j) continue;
    double term = 1.0 / (s[j] - s[q]);
    for (int k = 0; k < m; ++k) {
      if (k == j || k == q) continue;
      term *= (0.0 - s[k]) / (s[j] - s[k]);
    }
    total += term;
  }
  return total;
}

/* value at z of the j-th Lagrange basis polynomial on nodes s[0..m-1] */
static double lagrange_basis_at(const double* s, int m, int j, double z) {
  double v = 1.0;
  for (int k = 0; k < m; ++k) {
    if (k == j) continue;
    v *= (z - s[k]) / (s[j] - s[k]);
  }
  return v;
}

static double lagrange_basis_at0(const double* s, int m, int j) {
  return lagrange_basis_at(s, m, j, 0.0);
}

/* Coefficients of one substep.
 *  kind 1 (BDF1, backward Euler): x_{n+1} - x_n = h0 f(x_{n+1}); Newton starts
 *    at x_n; the local error is estimated from the explicit-Euler predictor
 *    x_n + h0 f(x_n) by Milne's device.
 *  kind 2 (BDF2): coefficients from the quadratic through (s_0, s_1, s_2); the
 *    predictor is the quadratic through x_n, x_{n-1}, x_{n-2} evaluated at s_0.
 * Milne's device: for a solution whose leading error derivative is constant,
 *    x_exact - x_corr = Cc * D and x_exact - x_pred = Cp * D, so the local error
 *    of the corrector is Cc/(Cp - Cc) * (x_corr - x_pred).  Cc and Cp are the
 *    residuals of each formula on y(s) = s^3/6 (BDF2) or s^2/2 (BDF1). */
int or_bdf_coefficients(int kind, double h0, double h1, double h2, or_substep* out) {
  memset(out, 0, sizeof(*out));
  out->kind = kind;
  out->h = h0;
  if (kind == 1) {
    double s[2] = {0.0, -h0};
    double l0 = lagrange_dbasis_at0(s, 2, 0);
    double l1 = lagrange_dbasis_at0(s, 2, 1);
    out->gamma = 1.0 / l0;
    out->rho1 = -l1 / l0;
    out->rho2 = 0.0;
    out->pi0 = 1.0;  /* Newton starts at x_n */
    /* residuals on y(s) = s^2/2, y'(s) = s */
    double Cc = 0.0 - out->rho1 * (s[1] * s[1] / 2.0) - out->gamma * 0.0;
    double Cp = 0.0 - (s[1] * s[1] / 2.0) - h0 * s[1]; /* x_n + h0 f(x_n) */
    out->mu = Cc / (Cp - Cc);
    return 0;
  }
  if (kind == 2) {
    double s[4] = {0.0, -h0, -(h0 + h1), -(h0 + h1 + h2)};
    double l0 = lagrange_dbasis_at0(s, 3, 0);
    double l1 = lagrange_dbasis_at0(s, 3, 1);
    double l2 = lagrange_dbasis_at0(s, 3, 2);
    out->gamma = 1.0 / l0;
    out->rho1 = -l1 / l0;
    out->rho2 = -l2 / l0;
    const double sp[3] = {s[1], s[2], s[3]};
    out->pi0 = lagrange_basis_at0(sp, 3, 0);
    out->pi1 = lagrange_basis_at0(sp, 3, 1);
    out->pi2 = lagrange_basis_at0(sp, 3, 2);
    /* residuals on y(s) = s^3/6, y'(0) = 0 */
    double c1 = s[1] * s[1] * s[1] / 6.0, c2 = s[2] * s[2] * s[2] / 6.0, c3 = s[3] * s[3] * s[3] / 6.0;
    double Cc = 0.0 - out->rho1 * c1 - out->rho2 * c2;
    double Cp = 0.0 - (out->pi0 * c1 + out->pi1 * c2 + out->pi2 * c3);
    out->mu = Cc / (Cp - Cc);
    return 0;
  }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* BDF3 and the Adams families at constant step h (the first three methods  */
/* of each family, Sec. 3, Tables 1-2).  Nodes are measured from t_{n+1}.   */
/*  AB_q: x_{n+1} = x_n + integral over [t_n, t_{n+1}] of the polynomial     */
/*        through f_n, ..., f_{n-q+1} (nodes -h, ..., -qh).                  */
/*  AM_q: the same with the polynomial through f_{n+1}, ..., f_{n-q+2}       */
/*        (nodes 0, ..., -(q-1)h); implicit in f_{n+1}.                     */
/*  BDF3: the derivative at t_{n+1} of the cubic through x_{n+1}, ...,      */
/*        x_{n-2} equals f_{n+1}.  Its predictor (reading) is the cubic     */
/*        through x_n, x_{n-1}, x_{n-2} with slope f(t_n, x_n) at t_n, which */
/*        needs no more stored history than BDF2.                           */
/* Milne's device pairs each corrector with a predictor of the same order q */
/* (AM_q with AB_q; BDF3 with the cubic above): with Cc, Cp the residuals   */
/* of the two formulas on y(s) = s^{q+1}/(q+1)!, the corrector's local      */
/* error is Cc/(Cp - Cc) (x_corr - x_pred).  An AB_q step is the predictor  */
/* itself, so its error is Cp/(Cp - Cc) (x_corr - x_pred), with AM_q        */
/* evaluated once at the new point.                                        */
/* ------------------------------------------------------------------------ */

/* s^k / k! */
static double mono(double s, int k) {
  double v = 1.0;
  for (int i = 1; i <= k; ++i) v *= s / (double)i;
  return v;
}

/* integral over [-h, 0] of the j-th Lagrange basis polynomial on nodes
 * s[0..m-1]; Simpson's rule is exact for the degrees used here (m - 1 <= 2) */
static double lagrange_basis_integral(const double* s, int m, int j, double h) {
  return (h / 6.0) * (lagrange_basis_at(s, m, j, -h) + 4.0 * lagrange_basis_at(s, m, j, -0.5 * h) +
                      lagrange_basis_at(s, m, j, 0.0));
}

/* AB_q weights of f_n, ..., f_{n-q+1} and AM_q weights of f_{n+1}, ..., f_{n-q+2} */
static void adams_weights(int q, double h, double* bab, double* beta) {
  double sb[3], sm[3];
  for (int j = 0; j < q; ++j) {
    sb[j] = -(double)(j + 1) * h;
    sm[j] = -(double)j * h;
  }
  for (int j = 0; j < 3; ++j) {
    bab[j] = j < q ? lagrange_basis_integral(sb, q, j, h) : 0.0;
    beta[j] = j < q ? lagrange_basis_integral(sm, q, j, h) : 0.0;
  }
}

/* residuals on y = s^{q+1}/(q+1)! of AB_q (Cp) and AM_q (Cc) */
static void adams_error_constants(int q, double h, const double* bab, const double* beta,
                                  double* Cp, double* Cc) {
  double p = mono(0.0, q + 1) - mono(-h, q + 1);
  double c = p;
  for (int j = 0; j < q; ++j) {
    p -= bab[j] * mono(-(double)(j + 1) * h, q);
    c -= beta[j] * mono(-(double)j * h, q);
  }
  *Cp = p;
  *Cc = c;
}

int or_lmm_coefficients(int kind, double h, or_substep* out) {
  memset(out, 0, sizeof(*out));
  out->kind = kind;
  out->h = h;
  if (!(h > 0.0)) return -1;
  if (kind == 3) {
    /* corrector: derivative at 0 of the cubic through nodes 0, -h, -2h, -3h */
    double s[4] = {0.0, -h, -2.0 * h, -3.0 * h};
    double l[4];
    for (int j = 0; j < 4; ++j) l[j] = lagrange_dbasis_at0(s, 4, j);
    out->gamma = 1.0 / l[0];
    out->rho1 = -l[1] / l[0];
    out->rho2 = -l[2] / l[0];
    out->rho3 = -l[3] / l[0];
    /* predictor: weights of x(-h), x(-2h), x(-3h), x'(-h) reproducing the
     * value at 0 of every cubic (a 4 x 4 linear system, row k = monomial s^k) */
    double A[16], e[4] = {1.0, 0.0, 0.0, 0.0}, w[4];
    for (int k = 0; k < 4; ++k) {
      A[k * 4 + 0] = pow(-h, k);
      A[k * 4 + 1] = pow(-2.0 * h, k);
      A[k * 4 + 2] = pow(-3.0 * h, k);
      A[k * 4 + 3] = k == 0 ? 0.0 : (double)k * pow(-h, k - 1);
    }
    if (or_lu_solve(4, A, e, w) != 0) return -1;
    out->pi0 = w[0];
    out->pi1 = w[1];
    out->pi2 = w[2];
    out->pi3 = w[3];
    double Cc = mono(0.0, 4) - (out->rho1 * mono(-h, 4) + out->rho2 * mono(-2.0 * h, 4) +
                                out->rho3 * mono(-3.0 * h, 4) + out->gamma * mono(0.0, 3));
    double Cp = mono(0.0, 4) - (out->pi0 * mono(-h, 4) + out->pi1 * mono(-2.0 * h, 4) +
                                out->pi2 * mono(-3.0 * h, 4) + out->pi3 * mono(-h, 3));
    out->mu = Cc / (Cp - Cc);
    return 0;
  }
  int q = kind % 10;
  if ((kind / 10 != 1 && kind / 10 != 2) || q < 1 || q > 3) return -1;
  adams_weights(q, h, out->bab, out->beta);
  out->gamma = out->beta[0];
  double Cp, Cc;
  adams_error_constants(q, h, out->bab, out->beta, &Cp, &Cc);
  out->mu = (kind / 10 == 1) ? Cc / (Cp - Cc) : Cp / (Cp - Cc);
  return 0;
}

static int or_lmm_valid(int lmm) {
  return lmm == OR_LMM_BDF1 || lmm == OR_LMM_BDF2 || lmm == OR_LMM_BDF3 ||
         (lmm >= OR_LMM_AM1 && lmm <= OR_LMM_AM3) || (lmm >= OR_LMM_AB1 && lmm <= OR_LMM_AB3);
}

/* Substep grid of one observation interval (t_prev, t_next] and the BDF kind
 * of every substep (Sec. 3.1: the same fixed steps for every particle).
 *  UNIFORM:   S = round((t_next - t_prev)/dt), which must be an integer to
 *             1e-9 relative; substep times t_prev + i (t_next - t_prev)/S.
 *  GEOMETRIC: S = cfg->substeps; times t_prev q^i with q = (t_next/t_prev)^(1/S),
 *             or, from t_prev = 0, t_next (q0^i - 1)/(q0^S - 1).
 *  The last substep time is t_next exactly; h_i is the difference of times.
 * History depth = number of stored past points beyond x_n (0, 1 or 2).  A BDF2
 * or BDF3 step needs depth 2; otherwise the step is BDF1.  An Adams method of
 * order q runs at order min(q, depth + 1).  A step ratio h_n/h_{n-1} >= 2
 * forces a cold start (depth 0), keeping variable-step BDF2 zero-stable.
 * BDF3 and the Adams families need uniform spacing (constant step). */
int or_build_substeps(const or_config* cfg, double t_prev, double t_next, int depth,
                      double hprev1, double hprev2, or_substep* tab, int max_steps,
                      int* depth_out) {
  if (!(t_next > t_prev)) return -1;
  if (!or_lmm_valid(cfg->lmm)) return -1;
  if (cfg->lmm != OR_LMM_BDF1 && cfg->lmm != OR_LMM_BDF2 && cfg->spacing != OR_SPACING_UNIFORM)
    return -1; /* the higher-order families are built for a constant step */
  int S;
  double times[OR_SMAX + 1];
  if (cfg->spacing == OR_SPACING_UNIFORM) {
    double ratio = (t_next - t_prev) / cfg->dt;
    double Sr = floor(ratio + 0.5);
    if (Sr < 1.0 || fabs(ratio - Sr) > 1e-9 * Sr) return -1;
    S = (int)Sr;
    if (S > max_steps || S > OR_SMAX) return -1;
    for (int i = 0; i < S; ++i) times[i] = t_prev + (double)i * ((t_next - t_prev) / (double)S);
  } else {
    S = cfg->substeps;
    if (S < 1 || S > max_steps || S > OR_SMAX) return -1;
    if (t_prev > 0.0) {
      double q = pow(t_next / t_prev, 1.0 / (double)S);
      for (int i = 0; i < S; ++i) times[i] = t_prev * pow(q, (double)i);
    } else {
      double q = cfg->q0;
      if (!(q > 1.0)) return -1;
      double denom = pow(q, (double)S) - 1.0;
      for (int i = 0; i < S; ++i) times[i] = t_next * ((pow(q, (double)i) - 1.0) / denom);
    }
  }
  times[S] = t_next;
  const int lmm = cfg->lmm;
  if (lmm == OR_LMM_BDF1) depth = 0;
  for (int i = 0; i < S; ++i) {
    double h0 = times[i + 1] - times[i];
    if (depth >= 1 && h0 / hprev1 >= 2.0) depth = 0;
    if (lmm == OR_LMM_BDF1 || lmm == OR_LMM_BDF2) {
      int kind = (lmm == OR_LMM_BDF2 && depth >= 2) ? 2 : 1;
      or_bdf_coefficients(kind, h0, hprev1, hprev2, &tab[i]);
    } else if (lmm == OR_LMM_BDF3) {
      /* BDF3 and its predictor need x_n, x_{n-1}, x_{n-2}; BDF1 until then */
      if (depth >= 2) or_lmm_coefficients(3, h0, &tab[i]);
      else or_bdf_coefficients(1, h0, 0.0, 0.0, &tab[i]);
    } else {
      /* Adams order q needs f_n, ..., f_{n-q+1}: the order grows by one per
       * step after a cold start */
      int q = lmm % 10, order = depth + 1 < q ? depth + 1 : q;
      or_lmm_coefficients((lmm / 10) * 10 + order, h0, &tab[i]);
    }
    tab[i].tn = times[i];
    tab[i].t = times[i + 1];
    hprev2 = hprev1;
    hprev1 = h0;
    depth = depth < 2 ? depth + 1 : 2;
  }
  if (lmm == OR_LMM_BDF1) depth = 0;
  if (depth_out) *depth_out = depth;
  return S;
}

/* Psi of Algorithm 1 (Steps 2 and 4d) for one particle: S substeps, each with
 * K full Newton iterations (I - gamma J(x)) dx = -G(x),
 * G(x) = x - rho1 x_n - rho2 x_{n-1} - gamma f(x), J re-evaluated every
 * iteration.  (x, h1, h2) = (x_n, x_{n-1}, x_{n-2}) on entry and exit.  If E is
 * not NULL, the squared Milne local-error estimates are summed into E (Step 4b
 * reading: Gamma = kappa diag(sum_s e_s^2)).  Returns 0, or -1 if the Newton
 * matrix became singular. */
static int propagate_adams(int ode, int d, int K, const double* th, const or_substep* tab, int S,
                           double* x, double* h1, double* h2, double* E);

int or_propagate(int ode, int d, int K, const double* th, const or_substep* tab, int S,
                 double* x, double* h1, double* h2, double* E) {
  if (S >= 1 && tab[0].kind > 10) return propagate_adams(ode, d, K, th, tab, S, x, h1, h2, E);
  const int linear = (ode == OR_ADVDIFF);
  double* xi = (double*)malloc(sizeof(double) * (size_t)d * 6);
  double *xp = xi + d, *r = xp + d, *G = r + d, *f = G + d, *dx = f + d;
  double* J = (double*)malloc(sizeof(double) * (size_t)d * d);
  double* M = (double*)malloc(sizeof(double) * (size_t)d * d);
  int* piv = (int*)malloc(sizeof(int) * (size_t)d);
  /* M2 is linear: J = L for every iterate, so its Newton matrix I - gamma L
   * is factored once per step size and reused */
  int have_J = 0, have_lu = 0, rc = 0;
  double lu_gamma = 0.0;
  for (int s = 0; s < S && rc == 0; ++s) {
    const or_substep* c = &tab[s];
    if (c->kind == 3) or_ode_f(ode, d, th, c->tn, x, f); /* BDF3 predictor slope */
    for (int i = 0; i < d; ++i) {
      if (c->kind == 2) {
        xp[i] = c->pi0 * x[i] + c->pi1 * h1[i] + c->pi2 * h2[i];
      } else if (c->kind == 3) {
        xp[i] = c->pi0 * x[i] + c->pi1 * h1[i] + c->pi2 * h2[i] + c->pi3 * f[i];
      } else {
        xp[i] = x[i];
      }
      r[i] = c->rho1 * x[i] + c->rho2 * h1[i];
      if (c->kind == 3) r[i] += c->rho3 * h2[i];
      xi[i] = xp[i];
    }
    if (c->kind == 1) {
      /* explicit-Euler predictor, used only by the error estimate */
      or_ode_f(ode, d, th, c->tn, x, f);
      for (int i = 0; i < d; ++i) xp[i] = x[i] + c->h * f[i];
    }
    for (int it = 0; it < K; ++it) {
      or_ode_f(ode, d, th, c->t, xi, f);
      if (!linear || !have_J) {
        or_ode_jac(ode, d, th, xi, J);
        have_J = 1;
      }
      for (int i = 0; i < d; ++i) G[i] = -(xi[i] - r[i] - c->gamma * f[i]);
      if (!linear || !have_lu || lu_gamma != c->gamma) {
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j)
            M[(size_t)i * d + j] = (i == j ? 1.0 : 0.0) - c->gamma * J[(size_t)i * d + j];
      }
      if (linear) {
        if (!have_lu || lu_gamma != c->gamma) {
          if (or_lu_factor(d, M, piv) != 0) {
            rc = -1;
            break;
          }
          have_lu = 1;
          lu_gamma = c->gamma;
        }
        or_lu_apply(d, M, piv, G, dx);
      } else if (or_lu_solve(d, M, G, dx) != 0) {
        rc = -1;
        break;
      }
      for (int i = 0; i < d; ++i) xi[i] += dx[i];
    }
    if (rc != 0) break;
    if (E) {
      for (int i = 0; i < d; ++i) {
        double e = c->mu * (xi[i] - xp[i]);
        E[i] += e * e;
      }
    }
    for (int i = 0; i < d; ++i) {
      h2[i] = h1[i];
      h1[i] = x[i];
      x[i] = xi[i];
    }
  }
  free(xi);
  free(J);
  free(M);
  free(piv);
  return rc;
}

/* Psi by an Adams method (Sec. 3, Tables 1-2): the stored history is the
 * states x_n, x_{n-1}, x_{n-2} (as for BDF), and the derivative history
 * f_n, f_{n-1}, f_{n-2} is evaluated from them with the particle's current
 * theta at the interval's start, at times t_n, t_n - h, t_n - 2h (constant
 * step).  Each substep:
 *   predictor (AB_q)  x_p = x_n + sum_j bab_j f_{n-j};
 *   AM_q: K Newton iterations on x - (x_n + sum_{j>=1} beta_j f_{n+1-j})
 *         - gamma f(t_{n+1}, x) = 0 from x_p; error mu (x_{n+1} - x_p);
 *   AB_q: x_{n+1} = x_p; error mu (x_c - x_p) with the AM_q value
 *         x_c = x_n + gamma f_{n+1} + sum_{j>=1} beta_j f_{n+1-j};
 * then f_{n+1} = f(t_{n+1}, x_{n+1}) joins the derivative history. */
static int propagate_adams(int ode, int d, int K, const double* th, const or_substep* tab, int S,
                           double* x, double* h1, double* h2, double* E) {
  double* F = (double*)malloc(sizeof(double) * (size_t)d * 10);
  double *F0 = F, *F1 = F + d, *F2 = F + 2 * d; /* f_n, f_{n-1}, f_{n-2} */
  double *xp = F + 3 * d, *r = F + 4 * d, *xi = F + 5 * d, *G = F + 6 * d, *fn = F + 7 * d;
  double *dx = F + 8 * d, *xc = F + 9 * d;
  double* J = (double*)malloc(sizeof(double) * (size_t)d * d);
  double* M = (double*)malloc(sizeof(double) * (size_t)d * d);
  int rc = 0;
  const int q0 = tab[0].kind % 10;
  or_ode_f(ode, d, th, tab[0].tn, x, F0);
  if (q0 >= 2) or_ode_f(ode, d, th, tab[0].tn - tab[0].h, h1, F1);
  if (q0 >= 3) or_ode_f(ode, d, th, tab[0].tn - 2.0 * tab[0].h, h2, F2);
  for (int s = 0; s < S && rc == 0; ++s) {
    const or_substep* c = &tab[s];
    const int q = c->kind % 10, implicit = c->kind < 20;
    const double* Fh[3] = {F0, F1, F2};
    for (int i = 0; i < d; ++i) {
      double v = x[i];
      for (int j = 0; j < q; ++j) v += c->bab[j] * Fh[j][i];
      xp[i] = v;
      double w = x[i];
      for (int j = 1; j < q; ++j) w += c->beta[j] * Fh[j - 1][i];
      r[i] = w;
      xi[i] = xp[i];
    }
    if (implicit) {
      for (int it = 0; it < K; ++it) {
        or_ode_f(ode, d, th, c->t, xi, fn);
        or_ode_jac(ode, d, th, xi, J);
        for (int i = 0; i < d; ++i) G[i] = -(xi[i] - r[i] - c->gamma * fn[i]);
        for (int i = 0; i < d; ++i)
          for (int j = 0; j < d; ++j)
            M[(size_t)i * d + j] = (i == j ? 1.0 : 0.0) - c->gamma * J[(size_t)i * d + j];
        if (or_lu_solve(d, M, G, dx) != 0) {
          rc = -1;
          break;
        }
        for (int i = 0; i < d; ++i) xi[i] += dx[i];
      }
      if (rc != 0) break;
    }
    or_ode_f(ode, d, th, c->t, xi, fn); /* f_{n+1} */
    if (E) {
      for (int i = 0; i < d; ++i) {
        double e;
        if (implicit) {
          e = c->mu * (xi[i] - xp[i]);
        } else {
          xc[i] = r[i] + c->gamma * fn[i];
          e = c->mu * (xc[i] - xp[i]);
        }
        E[i] += e * e;
      }
    }
    /* rotate the histories: x_{n+1} becomes x_n, f_{n+1} becomes f_n */
    double* t = F2;
    F2 = F1;
    F1 = F0;
    F0 = t;
    for (int i = 0; i < d; ++i) {
      F0[i] = fn[i];
      h2[i] = h1[i];
      h1[i] = x[i];
      x[i] = xi[i];
    }
  }
  free(F);
  free(J);
  free(M);
  return rc;
}

/* Gaussian observation model pi(y | x): log-likelihood without the constant
 * -sum log sigma_i - (m/2) log 2 pi, which cancels in every normalisation of
 * Steps 3a and 5.  RELATIVE noise reads "1% multiplicative" as
 * sigma_i = sigma * |y_i| (floored at 1e-300). */
double or_loglik(const or_config* cfg, const double* y, const double* x) {
  double s = 0.0;
  for (int i = 0; i < cfg->m; ++i) {
    double sig = cfg->sigma[i];
    if (cfg->noise == OR_NOISE_RELATIVE) sig = cfg->sigma[i] * fmax(fabs(y[i]), 1e-300);
    double z = (y[i] - x[cfg->obs_idx[i]]) / sig;
    s += z * z;
  }
  return -0.5 * s;
}

/* Step 3b, read as systematic resampling: tau_i = ((i + u)/N) c_{N-1};
 * l_i = min{k : c_k > tau_i}; if none, the first k with c_k = c_{N-1}. */
void or_resample_systematic(int64_t N, const double* c, double u, int32_t* idx) {
  double total = c[N - 1];
  int64_t first_full = 0;
  while (c[first_full] < total) ++first_full;
  int64_t k = 0;
  for (int64_t i = 0; i < N; ++i) {
    double tau = ((double)i + u) / (double)N * total;
    while (k < N && !(c[k] > tau)) ++k;
    idx[i] = (int32_t)(k < N ? k : first_full);
  }
}

/* Cholesky factor of a symmetric positive semi-definite p x p matrix
 * (lower, row-major).  A non-positive pivot gives a zero column, so C = 0 gives
 * L = 0 (reading: no jitter). */
void or_cholesky_psd(int p, const double* C, double* L) {
  for (int i = 0; i < p * p; ++i) L[i] = 0.0;
  for (int j = 0; j < p; ++j) {
    double dsum = C[j * p + j];
    for (int k = 0; k < j; ++k) dsum -= L[j * p + k] * L[j * p + k];
    if (!(dsum > 0.0)) continue;
    double ljj = sqrt(dsum);
    L[j * p + j] = ljj;
    for (int i = j + 1; i < p; ++i) {
      double s = C[i * p + j];
      for (int k = 0; k < j; ++k) s -= L[i * p + k] * L[j * p + k];
      L[i * p + j] = s / ljj;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* The filter                                                               */
/* ------------------------------------------------------------------------ */
struct or_filter {
  or_config cfg;
  int d, p;
  int64_t N;
  double *x, *h1, *h2, *phi, *lw;            /* committed ensemble         */
  double *nx, *nh1, *nh2, *nphi, *nlw;       /* epoch under construction   */
  double *ll1, *lg, *c;
  int32_t* idx;
  double phibar[OR_PMAX], C[OR_PMAX * OR_PMAX], xbar[OR_DMAX], ess;
  int epoch, depth;
  double t_prev, hprev1, hprev2;
  int pend_depth;                 /* history after the pending interval */
  double pend_h1, pend_h2;
};

static double* alloc_d(int64_t n) { return (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

or_filter* or_create(const or_config* cfg) {
  int d, p;
  if (or_ode_dims(cfg->ode, &d, &p) != 0) return NULL;
  d = cfg->d;
  if (or_ode_check_dim(cfg->ode, d) != 0 || d > OR_DMAX) return NULL;
  if (p != cfg->p || cfg->N < 1 || cfg->m < 0 || cfg->m > OR_MMAX) return NULL;
  if (!or_lmm_valid(cfg->lmm)) return NULL;
  if (cfg->lmm != OR_LMM_BDF1 && cfg->lmm != OR_LMM_BDF2 && cfg->spacing != OR_SPACING_UNIFORM)
    return NULL;
  or_filter* f = (or_filter*)calloc(1, sizeof(or_filter));
  f->cfg = *cfg;
  f->d = d; f->p = p; f->N = cfg->N;
  int64_t N = cfg->N;
  f->x = alloc_d(N * d); f->h1 = alloc_d(N * d); f->h2 = alloc_d(N * d);
  f->phi = alloc_d(N * p); f->lw = alloc_d(N);
  f->nx = alloc_d(N * d); f->nh1 = alloc_d(N * d); f->nh2 = alloc_d(N * d);
  f->nphi = alloc_d(N * p); f->nlw = alloc_d(N);
  f->ll1 = alloc_d(N); f->lg = alloc_d(N); f->c = alloc_d(N);
  f->idx = (int32_t*)calloc((size_t)N, sizeof(int32_t));
  return f;
}

void or_destroy(or_filter* f) {
  if (!f) return;
  free(f->x); free(f->h1); free(f->h2); free(f->phi); free(f->lw);
  free(f->nx); free(f->nh1); free(f->nh2); free(f->nphi); free(f->nlw);
  free(f->ll1); free(f->lg); free(f->c); free(f->idx);
  free(f);
}

/* Step 2, Liu-West shrinkage: phibar^n = a phi^n + (1 - a) phibar. */
void or_liu_west_shrink(int p, double a, const double* phi, const double* phibar, double* out) {
  for (int i = 0; i < p; ++i) out[i] = a * phi[i] + (1.0 - a) * phibar[i];
}

/* parameter in model space: theta = exp(phi) (LOG transform) or phi */
static void to_theta(const or_filter* f, const double* phi, double* th) {
  for (int i = 0; i < f->p; ++i) th[i] = (f->cfg.transform == OR_TRANSFORM_LOG) ? exp(phi[i]) : phi[i];
}

/* Weighted moments of the committed ensemble (Step 1 and Step 6):
 * w_n = exp(lw_n), phibar = sum w phi, C = sum w (phi - phibar)(phi - phibar)^T,
 * xbar = sum w x, ess = 1 / sum w^2.  Particles of weight exactly zero are
 * skipped (their state may be non-finite after a failed Newton solve). */
static void moments(or_filter* f) {
  int p = f->p, d = f->d;
  double mean[OR_PMAX] = {0}, xm[OR_DMAX] = {0}, w2 = 0.0;
  for (int64_t n = 0; n < f->N; ++n) {
    double w = exp(f->lw[n]);
    if (w == 0.0) continue; /* a zero-weight particle contributes nothing */
    for (int i = 0; i < p; ++i) mean[i] += w * f->phi[n * p + i];
    for (int i = 0; i < d; ++i) xm[i] += w * f->x[n * d + i];
    w2 += w * w;
  }
  double cov[OR_PMAX * OR_PMAX] = {0};
  for (int64_t n = 0; n < f->N; ++n) {
    double w = exp(f->lw[n]);
    if (w == 0.0) continue;
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j)
        cov[i * p + j] += w * (f->phi[n * p + i] - mean[i]) * (f->phi[n * p + j] - mean[j]);
  }
  memcpy(f->phibar, mean, sizeof(double) * p);
  memcpy(f->C, cov, sizeof(double) * p * p);
  memcpy(f->xbar, xm, sizeof(double) * d);
  f->ess = 1.0 / w2;
}

/* Step 1: theta^n drawn from the prior (uniform or log-uniform per component,
 * mapped to phi), x^n = x0 (known initial state; the history slots hold x0 as
 * well), w^n = 1/N; then the weighted mean and covariance. */
int or_init(or_filter* f) {
  const or_config* cfg = &f->cfg;
  int p = f->p, d = f->d;
  for (int64_t n = 0; n < f->N; ++n) {
    for (int i = 0; i < p; ++i) {
      double u = or_uniform(cfg->seed, cfg->stream, OR_RNG_INIT, (uint32_t)n + cfg->slot0, 0u, i);
      double th;
      if (cfg->prior_kind[i] == OR_LOGUNIFORM) {
        double lo = log(cfg->prior_lo[i]), hi = log(cfg->prior_hi[i]);
        double lphi = lo + u * (hi - lo);
        th = exp(lphi);
        f->phi[n * p + i] = (cfg->transform == OR_TRANSFORM_LOG) ? lphi : th;
      } else {
        th = cfg->prior_lo[i] + u * (cfg->prior_hi[i] - cfg->prior_lo[i]);
        f->phi[n * p + i] = (cfg->transform == OR_TRANSFORM_LOG) ? log(th) : th;
      }
    }
    for (int i = 0; i < d; ++i) {
      f->x[n * d + i] = cfg->x0[i];
      f->h1[n * d + i] = cfg->x0[i];
      f->h2[n * d + i] = cfg->x0[i];
    }
    f->lw[n] = -log((double)f->N);
  }
  f->epoch = 0;
  f->depth = 0;
  f->t_prev = cfg->t0;
  f->hprev1 = 0.0;
  f->hprev2 = 0.0;
  moments(f);
  return OR_OK;
}

int or_epoch_substeps(or_filter* f, double t_next, or_substep* tab, int max_steps) {
  int depth = (f->cfg.history == OR_HIST_RESTART) ? 0 : f->depth;
  int depth_out = 0;
  int S = or_build_substeps(&f->cfg, f->t_prev, t_next, depth, f->hprev1, f->hprev2, tab,
                            max_steps, &depth_out);
  if (S >= 1) {
    f->pend_depth = depth_out;
    f->pend_h1 = tab[S - 1].h;
    f->pend_h2 = (S >= 2) ? tab[S - 2].h : f->hprev1;
  }
  return S;
}

static int is_finite_d(double v) { return isfinite(v) ? 1 : 0; }

/* Steps 2 and 3a: shrink phi toward phibar (phibar^n = a phi^n + (1-a) phibar),
 * propagate x by Psi with theta(phibar^n), then log g = log w + log pi(y|xbar). */
int or_stage1(or_filter* f, const or_substep* tab, int S, const double* y) {
  const or_config* cfg = &f->cfg;
  int p = f->p, d = f->d;
  double a = cfg->a;
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < f->N; ++n) {
    double ph[OR_PMAX], th[OR_PMAX], x[OR_DMAX], h1[OR_DMAX], h2[OR_DMAX];
    or_liu_west_shrink(p, a, &f->phi[n * p], f->phibar, ph);
    to_theta(f, ph, th);
    memcpy(x, &f->x[n * d], sizeof(double) * d);
    memcpy(h1, &f->h1[n * d], sizeof(double) * d);
    memcpy(h2, &f->h2[n * d], sizeof(double) * d);
    int bad = or_propagate(cfg->ode, d, cfg->newton_iters, th, tab, S, x, h1, h2, NULL);
    double ll = bad ? NAN : or_loglik(cfg, y, x);
    f->ll1[n] = ll;
    double lg = f->lw[n] + ll;
    f->lg[n] = is_finite_d(lg) ? lg : -INFINITY;
  }
  return OR_OK;
}

/* Step 3a normalisation in the log domain: g_n = exp(lg_n - max lg), and the
 * cumulative sums c_k = g_0 + ... + g_k used by Step 3b. */
int or_cumulative(or_filter* f) {
  double M = -INFINITY;
  for (int64_t n = 0; n < f->N; ++n)
    if (f->lg[n] > M) M = f->lg[n];
  if (!(M > -INFINITY)) return OR_ERR_DEGENERATE;
  double acc = 0.0;
  for (int64_t n = 0; n < f->N; ++n) {
    acc += exp(f->lg[n] - M);
    f->c[n] = acc;
  }
  return OR_OK;
}

double or_resample_u(const or_filter* f) {
  return or_uniform(f->cfg.seed, f->cfg.stream, OR_RNG_RESAMPLE, 0u, (uint32_t)f->epoch, 0);
}

/* Steps 3c, 4 and 5 for every slot n, given the indices l_n:
 *  4a  phi_{j+1}^n = phibar^{l_n} + s L z,  s^2 = 1 - a^2,  L L^T = C_j;
 *  4b  Gamma = kappa diag(sum of squared Milne estimates along the
 *      repropagation from x_j^{l_n} with theta_{j+1}^n);
 *  4c  v = sqrt(Gamma) z';
 *  4d  x_{j+1} = Psi(x_j^{l_n}, theta_{j+1}^n) + v (stored history shifted by v);
 *  5   log w = log pi(y|x_{j+1}) - log pi(y|xbar^{l_n}) (unnormalised). */
int or_stage2(or_filter* f, const or_substep* tab, int S, const double* y, const int32_t* idx) {
  const or_config* cfg = &f->cfg;
  int p = f->p, d = f->d;
  double a = cfg->a, s = sqrt(1.0 - a * a);
  double L[OR_PMAX * OR_PMAX];
  or_cholesky_psd(p, f->C, L);
  uint32_t epoch = (uint32_t)f->epoch;
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < f->N; ++n) {
    int64_t l = idx[n];
    double ph[OR_PMAX], th[OR_PMAX], z[OR_PMAX], x[OR_DMAX], h1[OR_DMAX], h2[OR_DMAX];
    double E[OR_DMAX];
    const uint32_t slot = (uint32_t)n + cfg->slot0;
    for (int i = 0; i < p; ++i) z[i] = or_normal(cfg->seed, cfg->stream, OR_RNG_THETA, slot, epoch, i);
    double shrunk[OR_PMAX];
    or_liu_west_shrink(p, a, &f->phi[l * p], f->phibar, shrunk);
    for (int i = 0; i < p; ++i) {
      double lz = 0.0;
      for (int k = 0; k <= i; ++k) lz += L[i * p + k] * z[k];
      ph[i] = shrunk[i] + s * lz;
    }
    to_theta(f, ph, th);
    memcpy(x, &f->x[l * d], sizeof(double) * d);
    memcpy(h1, &f->h1[l * d], sizeof(double) * d);
    memcpy(h2, &f->h2[l * d], sizeof(double) * d);
    for (int i = 0; i < d; ++i) E[i] = 0.0;
    int bad = or_propagate(cfg->ode, d, cfg->newton_iters, th, tab, S, x, h1, h2, E);
    for (int i = 0; i < d; ++i) {
      double zi = or_normal(cfg->seed, cfg->stream, OR_RNG_INNOV, slot, epoch, i);
      double v = sqrt(cfg->kappa * E[i]) * zi;
      x[i] += v;
      h1[i] += v;
      h2[i] += v;
    }
    double ll2 = bad ? NAN : or_loglik(cfg, y, x);
    double lw = ll2 - f->ll1[l];
    f->nlw[n] = is_finite_d(lw) ? lw : -INFINITY;
    memcpy(&f->nx[n * d], x, sizeof(double) * d);
    memcpy(&f->nh1[n * d], h1, sizeof(double) * d);
    memcpy(&f->nh2[n * d], h2, sizeof(double) * d);
    memcpy(&f->nphi[n * p], ph, sizeof(double) * p);
  }
  return OR_OK;
}

/* Step 5 normalisation (log-sum-exp), Step 6 moments, and the history update.
 * Nothing changes if every new weight is zero (degenerate epoch). */
int or_commit(or_filter* f, double t_next) {
  double M = -INFINITY;
  for (int64_t n = 0; n < f->N; ++n)
    if (f->nlw[n] > M) M = f->nlw[n];
  if (!(M > -INFINITY)) return OR_ERR_DEGENERATE;
  double sum = 0.0;
  for (int64_t n = 0; n < f->N; ++n) sum += exp(f->nlw[n] - M);
  double lse = M + log(sum);
  for (int64_t n = 0; n < f->N; ++n) f->nlw[n] = f->nlw[n] - lse;
  double* t;
  t = f->x; f->x = f->nx; f->nx = t;
  t = f->h1; f->h1 = f->nh1; f->nh1 = t;
  t = f->h2; f->h2 = f->nh2; f->nh2 = t;
  t = f->phi; f->phi = f->nphi; f->nphi = t;
  t = f->lw; f->lw = f->nlw; f->nlw = t;
  moments(f);
  /* history bookkeeping for the next interval (set by or_epoch_substeps) */
  f->depth = f->pend_depth;
  f->hprev1 = f->pend_h1;
  f->hprev2 = f->pend_h2;
  f->t_prev = t_next;
  f->epoch += 1;
  return OR_OK;
}

/* One epoch j -> j+1 of Algorithm 1 (Steps 2-6). */
int or_epoch(or_filter* f, double t_next, const double* y) {
  or_substep* tab = (or_substep*)malloc(sizeof(or_substep) * OR_SMAX);
  int S = or_epoch_substeps(f, t_next, tab, OR_SMAX);
  if (S < 1) { free(tab); return OR_ERR_ARG; }
  for (int i = 0; i < f->cfg.m; ++i)
    if (!isfinite(y[i])) { free(tab); return OR_ERR_ARG; }
  or_stage1(f, tab, S, y);
  int st = or_cumulative(f);
  if (st != OR_OK) { free(tab); return st; }
  or_resample_systematic(f->N, f->c, or_resample_u(f), f->idx);
  or_stage2(f, tab, S, y, f->idx);
  st = or_commit(f, t_next);
  free(tab);
  return st;
}

void or_get_state(const or_filter* f, double* x, double* h1, double* h2, double* phi, double* lw) {
  int64_t N = f->N;
  if (x) memcpy(x, f->x, sizeof(double) * N * f->d);
  if (h1) memcpy(h1, f->h1, sizeof(double) * N * f->d);
  if (h2) memcpy(h2, f->h2, sizeof(double) * N * f->d);
  if (phi) memcpy(phi, f->phi, sizeof(double) * N * f->p);
  if (lw) memcpy(lw, f->lw, sizeof(double) * N);
}

void or_set_state(or_filter* f, const double* x, const double* h1, const double* h2,
                  const double* phi, const double* lw) {
  int64_t N = f->N;
  if (x) memcpy(f->x, x, sizeof(double) * N * f->d);
  if (h1) memcpy(f->h1, h1, sizeof(double) * N * f->d);
  if (h2) memcpy(f->h2, h2, sizeof(double) * N * f->d);
  if (phi) memcpy(f->phi, phi, sizeof(double) * N * f->p);
  if (lw) memcpy(f->lw, lw, sizeof(double) * N);
}

void or_get_moments(const or_filter* f, double* phibar, double* C, double* xbar, double* ess) {
  if (phibar) memcpy(phibar, f->phibar, sizeof(double) * f->p);
  if (C) memcpy(C, f->C, sizeof(double) * f->p * f->p);
  if (xbar) memcpy(xbar, f->xbar, sizeof(double) * f->d);
  if (ess) *ess = f->ess;
}

void or_set_moments(or_filter* f, const double* phibar, const double* C) {
  memcpy(f->phibar, phibar, sizeof(double) * f->p);
  memcpy(f->C, C, sizeof(double) * f->p * f->p);
}

void or_get_work(const or_filter* f, double* ll1, double* lg, double* c, int32_t* idx) {
  int64_t N = f->N;
  if (ll1) memcpy(ll1, f->ll1, sizeof(double) * N);
  if (lg) memcpy(lg, f->lg, sizeof(double) * N);
  if (c) memcpy(c, f->c, sizeof(double) * N);
  if (idx) memcpy(idx, f->idx, sizeof(int32_t) * N);
}

void or_get_history(const or_filter* f, int* epoch, int* depth, double* t_prev, double* hprev1,
                    double* hprev2) {
  *epoch = f->epoch; *depth = f->depth; *t_prev = f->t_prev;
  *hprev1 = f->hprev1; *hprev2 = f->hprev2;
}

void or_set_history(or_filter* f, int epoch, int depth, double t_prev, double hprev1, double hprev2) {
  f->epoch = epoch; f->depth = depth; f->t_prev = t_prev;
  f->hprev1 = hprev1; f->hprev2 = hprev2;
}

/* ------------------------------------------------------------------------ */
/* A shard of a particle-sharded filter                                     */
/* ------------------------------------------------------------------------ */
int or_shard_init(or_filter* f) {
  int st = or_init(f);
  for (int64_t n = 0; n < f->N; ++n) f->lw[n] = 0.0;
  /* the sums of every shard are taken about one common shift: zero for
   * Step 1 (the committed mean afterwards) */
  for (int i = 0; i < f->p; ++i) f->phibar[i] = 0.0;
  for (int i = 0; i < f->p * f->p; ++i) f->C[i] = 0.0;
  return st;
}

void or_get_pending_lw(const or_filter* f, double* lw) { memcpy(lw, f->nlw, sizeof(double) * f->N); }

void or_set_ll1(or_filter* f, const double* ll1) { memcpy(f->ll1, ll1, sizeof(double) * f->N); }

int or_shard_nsums(const or_filter* f) { return 2 + f->p + f->p * (f->p + 1) / 2 + f->d; }

/* Step 6's weighted sums of one shard, about the committed mean phibar */
void or_shard_sums(const or_filter* f, int pending, double M, double* sums) {
  const int p = f->p, d = f->d;
  const double* lw = pending ? f->nlw : f->lw;
  const double* phi = pending ? f->nphi : f->phi;
  const double* x = pending ? f->nx : f->x;
  const int ns = or_shard_nsums(f);
  for (int k = 0; k < ns; ++k) sums[k] = 0.0;
  double* S1 = sums + 2;
  double* S2 = S1 + p;
  double* Sx = S2 + p * (p + 1) / 2;
  for (int64_t n = 0; n < f->N; ++n) {
    double e = exp(lw[n] - M);
    if (e == 0.0) continue; /* a zero-weight particle contributes nothing */
    sums[0] += e;
    sums[1] += e * e;
    double dp[OR_PMAX];
    for (int i = 0; i < p; ++i) {
      dp[i] = phi[n * p + i] - f->phibar[i];
      S1[i] += e * dp[i];
    }
    int q = 0;
    for (int i = 0; i < p; ++i)
      for (int j = i; j < p; ++j) S2[q++] += e * dp[i] * dp[j];
    for (int i = 0; i < d; ++i) Sx[i] += e * x[n * d + i];
  }
}

int or_shard_commit(or_filter* f, int pending, double M, const double* sums, double t_next) {
  const int p = f->p, d = f->d;
  const double S0 = sums[0];
  if (!(S0 > 0.0)) return OR_ERR_DEGENERATE;
  const double* S1 = sums + 2;
  const double* S2 = S1 + p;
  const double* Sx = S2 + p * (p + 1) / 2;
  double m[OR_PMAX];
  for (int i = 0; i < p; ++i) m[i] = S1[i] / S0;
  int q = 0;
  for (int i = 0; i < p; ++i)
    for (int j = i; j < p; ++j) {
      double v = S2[q++] / S0 - m[i] * m[j];
      f->C[i * p + j] = v;
      f->C[j * p + i] = v;
    }
  for (int i = 0; i < p; ++i) f->phibar[i] += m[i];
  for (int i = 0; i < d; ++i) f->xbar[i] = Sx[i] / S0;
  f->ess = S0 * S0 / sums[1];
  const double lse = M + log(S0);
  if (pending) {
    double* t;
    t = f->x; f->x = f->nx; f->nx = t;
    t = f->h1; f->h1 = f->nh1; f->nh1 = t;
    t = f->h2; f->h2 = f->nh2; f->nh2 = t;
    t = f->phi; f->phi = f->nphi; f->nphi = t;
    t = f->lw; f->lw = f->nlw; f->nlw = t;
    f->depth = f->pend_depth;
    f->hprev1 = f->pend_h1;
    f->hprev2 = f->pend_h2;
    f->t_prev = t_next;
    f->epoch += 1;
  }
  for (int64_t n = 0; n < f->N; ++n) f->lw[n] = f->lw[n] - lse;
  return OR_OK;
}

int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* threads of the particle loops from now on (CPU-baseline timing only; the
 * result does not depend on it) */
void or_set_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
