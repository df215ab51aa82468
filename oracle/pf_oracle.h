/*
 * pf_oracle.h -- CPU oracle of the LMM PF-SMC sampler (Algorithm 1 of
 * Arnold, Calvetti, Somersalo, "Vectorized and Parallel Particle Filter SMC
 * Parameter Estimation for Stiff ODEs").
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, FP64 restatement of the
 * method that the CUDA library is checked against.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header, table or constant generator with the CUDA library.
 *
 * Every function cites the section, step or equation of the paper it follows,
 * or names the reading taken where the paper is silent (the readings are
 * listed in the repository's design notes).
 *
 * Parity pins: every function here is pinned by a CPU test against a closed
 * form, an invariant, a published known-answer vector or brute force; none is
 * "parity unpinned".
 */
#ifndef PF_ORACLE_H
#define PF_ORACLE_H
#include <stdint.h>

#define OR_DMAX 2025   /* the largest M2 grid, 45 x 45 */
#define OR_PMAX 8
#define OR_MMAX 32
#define OR_SMAX 4096

/* problem ids; OR_ADVDIFF is the paper's 2D advection-diffusion system (M2,
 * Sec. 4) on an nt x nt periodic grid, d = nt^2 with nt odd, 3 <= nt <= 45;
 * OR_MICHAELIS is the paper's three-compartment Michaelis-Menten system (M1,
 * Sec. 2.1), d = 3, theta = (V1, V2, k1, k2), with the known constants taken
 * as stated in or_mm_constants */
enum { OR_LINEAR2 = 1, OR_ROBERTSON = 2, OR_BRUSSELATOR = 3, OR_ADVDIFF = 4, OR_MICHAELIS = 5 };
/* LMMs (Sec. 3, Tables 1-2): the first three methods of each family */
enum {
  OR_LMM_BDF1 = 1, OR_LMM_BDF2 = 2, OR_LMM_BDF3 = 3,
  OR_LMM_AM1 = 11, OR_LMM_AM2 = 12, OR_LMM_AM3 = 13,
  OR_LMM_AB1 = 21, OR_LMM_AB2 = 22, OR_LMM_AB3 = 23
};
/* random-stream purposes (counter word 2, low byte) */
enum { OR_RNG_INIT = 1, OR_RNG_THETA = 2, OR_RNG_INNOV = 3, OR_RNG_RESAMPLE = 4 };
enum { OR_UNIFORM = 0, OR_LOGUNIFORM = 1 };          /* prior kinds          */
enum { OR_SPACING_UNIFORM = 0, OR_SPACING_GEOMETRIC = 1 };
enum { OR_HIST_CARRY = 0, OR_HIST_RESTART = 1 };
enum { OR_TRANSFORM_LOG = 0, OR_TRANSFORM_IDENTITY = 1 };
enum { OR_NOISE_ADDITIVE = 0, OR_NOISE_RELATIVE = 1 };
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_DEGENERATE = 5 };

typedef struct {
  int ode, d, p, m;
  int64_t N;
  int lmm;          /* OR_LMM_*: BDF1, BDF2 (BDF1 on cold starts), BDF3,
                       AM1-3, AB1-3 (lower orders of the family on cold
                       starts); all but BDF1/BDF2 need uniform spacing     */
  int newton_iters; /* fixed Newton count K                                 */
  int spacing;      /* OR_SPACING_*                                          */
  double dt;        /* uniform substep length                               */
  int substeps;     /* geometric: substeps per interval                     */
  double q0;        /* geometric: ratio used on an interval starting at t=0 */
  int history;      /* OR_HIST_*                                             */
  int transform;    /* OR_TRANSFORM_*                                        */
  int obs_idx[OR_MMAX];
  int noise;        /* OR_NOISE_*                                            */
  double sigma[OR_MMAX];
  double a;         /* Liu-West shrinkage factor, 0<a<1 (Step 2)            */
  double kappa;     /* scale of the innovation covariance                   */
  uint64_t seed;
  uint32_t stream;  /* filter id, fourth counter word                       */
  int prior_kind[OR_PMAX];
  double prior_lo[OR_PMAX], prior_hi[OR_PMAX];
  double x0[OR_DMAX];
  double t0;        /* time of the initial state                            */
  uint32_t slot0;   /* first global slot of a shard (its random streams are
                       keyed by the global slot); 0 for a whole filter       */
} or_config;

/* One substep of the LMM on the shared grid.
 * BDF kinds 1, 2: x_{n+1} - rho1 x_n - rho2 x_{n-1} = gamma f(t_{n+1}, x_{n+1}),
 *   predictor pi0 x_n + pi1 x_{n-1} + pi2 x_{n-2} (kind 2) or the explicit
 *   Euler step (kind 1), local error mu (x_{n+1} - x_p).
 * BDF kind 3: x_{n+1} - rho1 x_n - rho2 x_{n-1} - rho3 x_{n-2} = gamma f_{n+1},
 *   predictor pi0 x_n + pi1 x_{n-1} + pi2 x_{n-2} + pi3 f(t_n, x_n).
 * Adams-Moulton kinds 10 + q: x_{n+1} = x_n + beta0 f_{n+1} + beta1 f_n +
 *   beta2 f_{n-1} (gamma = beta0), predictor AB_q.
 * Adams-Bashforth kinds 20 + q: x_{n+1} = x_n + bab0 f_n + bab1 f_{n-1} +
 *   bab2 f_{n-2}; its error is measured against AM_q evaluated at x_{n+1}.
 * Adams weights are scaled by h; f_j = f(t_j, x_j). */
typedef struct {
  int kind;         /* 1, 2, 3 (BDF); 11-13 (AM order q); 21-23 (AB order q) */
  double h;         /* step length                                          */
  double gamma;     /* weight of f(t_{n+1}, x_{n+1}) in the implicit equation */
  double rho1, rho2;
  double pi0, pi1, pi2;
  double mu;        /* local error = mu (x_corr - x_pred)                    */
  double rho3, pi3;
  double beta[3];   /* AM_q weights of f_{n+1}, f_n, f_{n-1}                 */
  double bab[3];    /* AB_q weights of f_n, f_{n-1}, f_{n-2}                 */
  double tn, t;     /* t_n and t_{n+1}                                       */
} or_substep;

typedef struct or_filter or_filter;

/* --- building blocks (each pinned on its own) --------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double or_uniform(uint64_t seed, uint32_t stream, int purpose, uint32_t n, uint32_t epoch, int k);
double or_normal(uint64_t seed, uint32_t stream, int purpose, uint32_t n, uint32_t epoch, int k);
/* f(t, x; theta); only OR_MICHAELIS depends on t (its input function) */
void or_ode_f(int ode, int d, const double* theta, double t, const double* x, double* f);
void or_ode_jac(int ode, int d, const double* theta, const double* x, double* J);
/* M1's known constants (lambda, c0, A0, A, t0, tau) and its input Phi(t) */
void or_mm_constants(double* out6);
double or_mm_input(double t);
/* parameter count and the fixed state dimension (0 when the dimension is a
 * choice of the problem, as for OR_ADVDIFF) */
int or_ode_dims(int ode, int* d, int* p);
/* 0 if d is a valid state dimension of the problem */
int or_ode_check_dim(int ode, int d);
int or_lu_solve(int n, const double* A, const double* b, double* x);
/* LU with partial pivoting, factor once and solve many right-hand sides */
int or_lu_factor(int n, double* A, int* piv);
void or_lu_apply(int n, const double* LU, const int* piv, const double* b, double* x);
int or_bdf_coefficients(int kind, double h0, double h1, double h2, or_substep* out);
/* constant-step coefficients of BDF3 (kind 3), AM_q (10 + q), AB_q (20 + q) */
int or_lmm_coefficients(int kind, double h, or_substep* out);
int or_build_substeps(const or_config* cfg, double t_prev, double t_next, int depth,
                      double hprev1, double hprev2, or_substep* tab, int max_steps,
                      int* depth_out);
int or_propagate(int ode, int d, int K, const double* theta, const or_substep* tab, int S,
                 double* x, double* h1, double* h2, double* E);
double or_loglik(const or_config* cfg, const double* y, const double* x);
void or_resample_systematic(int64_t N, const double* c, double u, int32_t* idx);
void or_cholesky_psd(int p, const double* C, double* L);
void or_liu_west_shrink(int p, double a, const double* phi, const double* phibar, double* out);

/* --- the filter (Algorithm 1) -------------------------------------------- */
or_filter* or_create(const or_config* cfg);
void or_destroy(or_filter* f);
int or_init(or_filter* f);                                   /* Step 1      */
int or_epoch(or_filter* f, double t_next, const double* y);  /* Steps 2-6   */
/* stage entry points for parity injection */
int or_epoch_substeps(or_filter* f, double t_next, or_substep* tab, int max_steps);
int or_stage1(or_filter* f, const or_substep* tab, int S, const double* y);
int or_cumulative(or_filter* f);
double or_resample_u(const or_filter* f);
int or_stage2(or_filter* f, const or_substep* tab, int S, const double* y, const int32_t* idx);
int or_commit(or_filter* f, double t_next);
/* state access, arrays are particle-major: x[n*d + i], phi[n*p + i] */
void or_get_state(const or_filter* f, double* x, double* h1, double* h2, double* phi,
                  double* lw);
void or_set_state(or_filter* f, const double* x, const double* h1, const double* h2,
                  const double* phi, const double* lw);
void or_get_moments(const or_filter* f, double* phibar, double* C, double* xbar, double* ess);
void or_set_moments(or_filter* f, const double* phibar, const double* C);
void or_get_work(const or_filter* f, double* ll1, double* lg, double* c, int32_t* idx);
void or_get_history(const or_filter* f, int* epoch, int* depth, double* t_prev,
                    double* hprev1, double* hprev2);
void or_set_history(or_filter* f, int epoch, int depth, double t_prev, double hprev1,
                    double hprev2);
/* --- a shard of a particle-sharded filter (Sec. 3.1's particle loops split
 * over processes): Step 5's normalisation and Step 6's moments taken from
 * sums over every shard.  Test infrastructure for the sharded protocol. */
/* Step 1's draws for the shard's slots; raw log weight 0; the moments are
 * zero (the common shift of Step 1's sums) until or_shard_commit */
int or_shard_init(or_filter* f);
/* raw log weights of the last or_stage2 (before any normalisation) */
void or_get_pending_lw(const or_filter* f, double* lw);
/* first-stage log-likelihoods (as received with the parents) */
void or_set_ll1(or_filter* f, const double* ll1);
/* number of Step 6 sums: 2 + p + p(p+1)/2 + d */
int or_shard_nsums(const or_filter* f);
/* Step 6's sums over the shard's new ensemble (pending = 1) or its committed
 * one (pending = 0, Step 1), with weights e_n = exp(lw_n - M): sum e, sum e^2,
 * sum e (phi - phibar), sum e (phi_i - phibar_i)(phi_j - phibar_j) (i <= j),
 * sum e x, phibar the committed mean */
void or_shard_sums(const or_filter* f, int pending, double M, double* sums);
/* commit with the sums over every shard: phibar += S1 / S0,
 * C = S2 / S0 - (S1 / S0)(S1 / S0)^T, xbar = Sx / S0, ess = S0^2 / W2, and the
 * log weights normalised by M + log S0; pending = 1 takes the new ensemble
 * and advances the history (or_commit's bookkeeping) */
int or_shard_commit(or_filter* f, int pending, double M, const double* sums, double t_next);
int or_threads(void);
void or_set_threads(int n);
#endif
