/*
 * Host-side memory and undefined-behaviour check of the CPU oracle: built by
 * tests/test_oracle_sanitizers.py together with oracle/pf_oracle.c under
 * AddressSanitizer and UndefinedBehaviorSanitizer, it runs the oracle's
 * filter (Algorithm 1) for a few epochs on every problem and every LMM, and
 * its building blocks on edge cases (N = 1, cold starts, degenerate epochs).
 * Synthetic inputs only; exit status 0 means every call returned the
 * expected status and the sanitizers found nothing.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "../oracle/pf_oracle.h"

static int fails = 0;
#define EXPECT(c)                                                  \
  do {                                                             \
    if (!(c)) {                                                    \
      fprintf(stderr, "%s:%d: expected %s\n", __FILE__, __LINE__, #c); \
      ++fails;                                                     \
    }                                                              \
  } while (0)

static void base(or_config* c, int ode, int d, int p, int64_t N, int lmm) {
  memset(c, 0, sizeof(*c));
  c->ode = ode; c->d = d; c->p = p; c->N = N; c->lmm = lmm;
  c->newton_iters = 2; c->spacing = OR_SPACING_UNIFORM; c->dt = 0.01;
  c->history = OR_HIST_CARRY; c->transform = OR_TRANSFORM_LOG;
  c->m = 1; c->obs_idx[0] = 0; c->noise = OR_NOISE_ADDITIVE; c->sigma[0] = 0.05;
  c->a = 0.98; c->kappa = 1.0; c->seed = 11; c->stream = 3;
  for (int i = 0; i < p; ++i) {
    c->prior_kind[i] = OR_LOGUNIFORM;
    c->prior_lo[i] = 0.5;
    c->prior_hi[i] = 2.0;
  }
  for (int i = 0; i < d; ++i) c->x0[i] = 1.0 + 0.01 * i;
}

static void run(const or_config* c, int epochs, double dt_obs) {
  or_filter* f = or_create(c);
  EXPECT(f != NULL);
  if (!f) return;
  EXPECT(or_init(f) == OR_OK);
  double y[OR_MMAX];
  for (int k = 1; k <= epochs; ++k) {
    for (int i = 0; i < c->m; ++i) y[i] = c->x0[c->obs_idx[i]] * exp(-0.1 * k);
    int st = or_epoch(f, c->t0 + k * dt_obs, y);
    EXPECT(st == OR_OK || st == OR_ERR_DEGENERATE);
  }
  double phibar[OR_PMAX], C[OR_PMAX * OR_PMAX], ess;
  double* xbar = (double*)malloc(sizeof(double) * (size_t)c->d);
  or_get_moments(f, phibar, C, xbar, &ess);
  EXPECT(ess >= 1.0 - 1e-9 && ess <= (double)c->N + 1e-9);
  free(xbar);
  or_destroy(f);
}

int main(void) {
  static const int lmms[] = {OR_LMM_BDF1, OR_LMM_BDF2, OR_LMM_BDF3, OR_LMM_AM1, OR_LMM_AM2,
                             OR_LMM_AM3, OR_LMM_AB1, OR_LMM_AB2, OR_LMM_AB3};
  or_config c;
  for (int li = 0; li < 9; ++li) {
    base(&c, OR_LINEAR2, 2, 2, 37, lmms[li]);
    run(&c, 4, 0.1);
    base(&c, OR_ROBERTSON, 3, 3, 19, lmms[li]);
    c.dt = 1e-5;
    run(&c, 3, 1e-4);
    base(&c, OR_MICHAELIS, 3, 4, 23, lmms[li]);
    c.newton_iters = 4; c.dt = 0.05; c.m = 3; c.obs_idx[1] = 1; c.obs_idx[2] = 2;
    c.sigma[1] = c.sigma[2] = 0.05;
    run(&c, 4, 0.5);
  }
  /* the larger problems with BDF2, and geometric spacing */
  base(&c, OR_BRUSSELATOR, 64, 3, 5, OR_LMM_BDF2);
  c.dt = 1.0 / 60.0; c.newton_iters = 3;
  run(&c, 2, 1.0 / 3.0);
  base(&c, OR_ADVDIFF, 25, 5, 4, OR_LMM_BDF2);
  c.transform = OR_TRANSFORM_IDENTITY; c.newton_iters = 1; c.dt = 0.1;
  for (int i = 0; i < 5; ++i) { c.prior_kind[i] = OR_UNIFORM; c.prior_lo[i] = 0.5; c.prior_hi[i] = 1.5; }
  run(&c, 2, 1.0);
  base(&c, OR_ROBERTSON, 3, 3, 7, OR_LMM_BDF2);
  c.spacing = OR_SPACING_GEOMETRIC; c.substeps = 20; c.q0 = 1.1; c.t0 = 1e-4;
  run(&c, 3, 1e-4);
  /* N = 1 and the restart history */
  base(&c, OR_LINEAR2, 2, 2, 1, OR_LMM_AM3);
  c.history = OR_HIST_RESTART;
  run(&c, 3, 0.1);
  /* a degenerate epoch: the observation is not finite -> argument error */
  base(&c, OR_LINEAR2, 2, 2, 8, OR_LMM_BDF2);
  {
    or_filter* f = or_create(&c);
    EXPECT(or_init(f) == OR_OK);
    double y = NAN;
    EXPECT(or_epoch(f, 0.1, &y) == OR_ERR_ARG);
    or_destroy(f);
  }
  /* rejected configurations */
  base(&c, OR_LINEAR2, 2, 2, 8, 4);
  EXPECT(or_create(&c) == NULL);
  base(&c, OR_ROBERTSON, 3, 3, 8, OR_LMM_AB2);
  c.spacing = OR_SPACING_GEOMETRIC; c.substeps = 10; c.q0 = 1.1;
  EXPECT(or_create(&c) == NULL);
  /* building blocks on small inputs */
  {
    double cum[5] = {0.0, 1.0, 1.0, 2.5, 4.0};
    int32_t idx[5];
    or_resample_systematic(5, cum, 0.3, idx);
    for (int i = 0; i < 5; ++i) EXPECT(idx[i] >= 0 && idx[i] < 5 && idx[i] != 0);
    double Cm[4] = {0.0, 0.0, 0.0, 0.0}, L[4];
    or_cholesky_psd(2, Cm, L);
    EXPECT(L[0] == 0.0 && L[3] == 0.0);
    or_substep s;
    for (int k = 0; k < 7; ++k) {
      static const int kinds[] = {3, 11, 12, 13, 21, 22, 23};
      EXPECT(or_lmm_coefficients(kinds[k], 0.1, &s) == 0);
    }
    EXPECT(or_lmm_coefficients(14, 0.1, &s) != 0);
  }
  if (fails) fprintf(stderr, "%d failed expectations\n", fails);
  else printf("oracle sanitizer driver: ok\n");
  return fails ? 1 : 0;
}
