/*
 * pf.h -- C ABI of the GB300 (sm_103a) LMM PF-SMC sampler.
 *
 * The library runs the per-observation epoch of Algorithm 1 ("LMM PF-SMC
 * Sampler") of Arnold, Calvetti, Somersalo, "Vectorized and Parallel Particle
 * Filter SMC Parameter Estimation for Stiff ODEs": a Liu-West auxiliary
 * particle filter over (x, theta) whose particles are propagated by a linear
 * multistep method (BDF1-3, Adams-Moulton 1-3 with a full Newton solve per
 * particle and per substep, or Adams-Bashforth 1-3), and whose innovation
 * variance comes from the LMM's local error estimate (Step 4b).  All arithmetic is FP64 and runs in
 * hand-written CUDA kernels; nothing falls back to the CPU.
 *
 * Conventions
 *  - Every entry point returns a pf_status.  No C++ exception crosses the ABI.
 *  - Host pointers are owned by the caller and only read or written during the
 *    call; the library copies what it keeps.  Device memory of a filter is
 *    owned by the filter (allocated in pf_create, freed in pf_destroy).
 *  - One filter must not be used from two host threads at once.
 *  - Epochs are transactional: a failed epoch (degenerate weights, CUDA error)
 *    leaves the committed ensemble, moments and history unchanged.
 *  - Indices are 0-based.  Matrices are row-major.  Host ensemble arrays are
 *    particle-major: x[n*d + i], phi[n*p + i].
 *  - Parameters live in a working space phi: phi = log(theta) with
 *    PF_TRANSFORM_LOG (default), phi = theta with PF_TRANSFORM_IDENTITY.
 *    Means and covariances are reported in phi space.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_filter pf_filter; /* opaque, library-owned */

typedef enum {
  PF_OK = 0,
  PF_ERR_INVALID_ARG = 1, /* argument out of range or inconsistent          */
  PF_ERR_OOM = 2,         /* device or pinned-host allocation failed        */
  PF_ERR_BUDGET = 3,      /* request exceeds a stated size limit            */
  PF_ERR_CUDA = 4,        /* a CUDA runtime call failed                     */
  PF_ERR_DEGENERATE = 5,  /* every weight of the epoch is zero or not finite */
  PF_ERR_NUMERIC = 6,     /* a non-finite moment                            */
  PF_ERR_TIMEOUT = 7,     /* reserved: a bounded device wait gave up        */
  PF_ERR_STATE = 8        /* call out of order (e.g. no observation loaded) */
} pf_status;

/* Problems x' = f(t, x; theta).  Three textbook stiff systems, and the paper's
 * own two (Sec. 2.1's M1, whose unprinted constants are a stated reading, and
 * Sec. 4's system as given):
 *  PF_ODE_LINEAR2        d=2, p=2: x' = A x, A = [[-th1, th2], [0, -th2]].
 *  PF_ODE_ROBERTSON      d=3, p=3: Robertson kinetics, theta = (k1, k2, k3).
 *  PF_ODE_BRUSSELATOR1D  d=64, p=3: 1D Brusselator on 32 interior points,
 *                        Dirichlet u=1, v=3, theta = (A, B, alpha), state
 *                        interleaved (u_0, v_0, u_1, v_1, ...).
 *  PF_ODE_ADVDIFF2D      d=nt^2 (nt odd, 3 <= nt <= 45), p=5: the 2D
 *                        advection-diffusion system of Sec. 4 on the periodic
 *                        nt x nt grid, U' = L U with
 *                        L = -{k1^2 B1'B1 + k1 k3 (B1'B2 + B2'B1)
 *                              + (k2^2 + k3^2) B2'B2} + c1 B1 + c2 B2,
 *                        B1 = I (x) ell, B2 = ell (x) I, (ell u)_j = u_j - u_{j-1}
 *                        (periodic), theta = (k1, k2, k3, c1, c2), state
 *                        U[iy*nt + ix] (x fastest).  Linear: one Newton
 *                        iteration solves each step.
 *  PF_ODE_MICHAELIS3     d=3, p=4: the three-compartment Michaelis-Menten
 *                        system of Sec. 2.1 (M1),
 *                          x1' = Phi(t) - V1 x1/(x1+k1),
 *                          x2' = V1 x1/(x1+k1) - V2 x2/(x2+k2),
 *                          x3' = V2 x2/(x2+k2) - lambda (x3 - c0),
 *                        Phi(t) = A0 + A (t - t0)_+ exp(-(t - t0)/tau),
 *                        theta = (V1, V2, k1, k2).  The paper calls lambda,
 *                        c0, A0, A, t0, tau known but prints no values; this
 *                        library fixes lambda = 0.5, c0 = 2, A0 = 1, A = 0.5,
 *                        t0 = 0.5, tau = 4. */
typedef enum {
  PF_ODE_LINEAR2 = 1,
  PF_ODE_ROBERTSON = 2,
  PF_ODE_BRUSSELATOR1D = 3,
  PF_ODE_ADVDIFF2D = 4,
  PF_ODE_MICHAELIS3 = 5
} pf_ode;

/* LMM of Psi (Sec. 2.1, Sec. 3 and Tables 1-2: the first three methods of
 * each family, numbered by order).
 *  BDF1 = backward Euler; BDF2 = variable-step BDF2 (BDF1 on the first two
 *  substeps after a cold start); BDF3 (BDF1 until two past states exist).
 *  AM1-AM3: Adams-Moulton of order 1-3 (AM1 is backward Euler, AM2 the
 *  trapezoidal rule), Newton-solved like BDF.  AB1-AB3: explicit
 *  Adams-Bashforth of order 1-3 (no Newton solve; not suited to stiff
 *  problems).  Adams methods start at order 1 and gain one order per step.
 *  Local errors by Milne's device against a same-order predictor (AB_q for
 *  AM_q, AM_q evaluated once for AB_q, a cubic through three states and one
 *  slope for BDF3).  BDF3 and the Adams methods need PF_SPACING_UNIFORM and
 *  one of PF_ODE_LINEAR2, PF_ODE_ROBERTSON, PF_ODE_MICHAELIS3. */
typedef enum {
  PF_LMM_BDF1 = 1,
  PF_LMM_BDF2 = 2,
  PF_LMM_BDF3 = 3,
  PF_LMM_AM1 = 11,
  PF_LMM_AM2 = 12,
  PF_LMM_AM3 = 13,
  PF_LMM_AB1 = 21,
  PF_LMM_AB2 = 22,
  PF_LMM_AB3 = 23
} pf_lmm;

enum { PF_PRIOR_UNIFORM = 0, PF_PRIOR_LOGUNIFORM = 1 };
enum { PF_SPACING_UNIFORM = 0, PF_SPACING_GEOMETRIC = 1 };
enum { PF_HISTORY_CARRY = 0, PF_HISTORY_RESTART = 1 };
enum { PF_TRANSFORM_LOG = 0, PF_TRANSFORM_IDENTITY = 1 };
enum { PF_NOISE_ADDITIVE = 0, PF_NOISE_RELATIVE = 1 };

/* Size limits of this build. */
#define PF_MAX_OBS 32         /* m                                    */
#define PF_MAX_SUBSTEPS 640   /* substeps per observation interval    */
#define PF_MAX_PARTICLES (1LL << 30)

/* Prior pi_0(x_0, theta) of Step 1: x_0 is known (a point mass at x0), and
 * theta_i is uniform or log-uniform on [lo_i, hi_i], independently. */
typedef struct {
  int p;              /* number of parameters, must match the ODE        */
  const int* kind;    /* p entries, PF_PRIOR_*                           */
  const double* lo;   /* p entries, 0 < lo <= hi for log-uniform         */
  const double* hi;   /* p entries                                       */
  int d;              /* state dimension, must match the ODE             */
  const double* x0;   /* d entries: the initial state                    */
  double t0;          /* its time                                        */
} pf_prior;

/* Sampler settings.  Zero-initialise, then set what you need. */
typedef struct {
  double a;           /* Liu-West shrinkage, 0 < a <= 1 (Step 2)          */
  int newton_iters;   /* fixed Newton count K >= 1 per substep            */
  int spacing;        /* PF_SPACING_*                                     */
  int substeps;       /* geometric spacing: substeps per interval         */
  double q0;          /* geometric spacing: step ratio on an interval that
                         starts at t = 0 (> 1)                           */
  int history;        /* PF_HISTORY_CARRY: LMM history carried across
                         observations (translated by the innovation);
                         PF_HISTORY_RESTART: cold start every interval    */
  int transform;      /* PF_TRANSFORM_*                                   */
  int m;              /* observed components per epoch, 0 < m <= 32      */
  const int* obs_idx; /* m state indices                                  */
  int noise;          /* PF_NOISE_ADDITIVE: sd sigma_i; PF_NOISE_RELATIVE:
                         sd sigma_i * |y_i| (floored at 1e-300)          */
  const double* sigma;/* m entries                                       */
  double kappa;       /* Gamma = kappa * diag(sum of squared local errors) */
  uint64_t seed;      /* Philox4x32-10 key                                */
  uint32_t filter_id; /* fourth Philox counter word                       */
  void* stream;       /* cudaStream_t to run on; NULL = a stream the filter
                         creates and owns                                  */
  int timing;         /* 0: no timing events; 1: CUDA events around every
                         kernel of every epoch; 2: around stage 2 only, the
                         dominant kernel (the other kernels keep their
                         programmatic launch overlap).  Read them with
                         pf_kernel_times.  Other values: INVALID_ARG.      */
} pf_options;

/* Create a filter and run Step 1 of Algorithm 1 (prior draws, w = 1/N,
 * weighted mean and covariance).  dt is the uniform substep length (the
 * interval length must be an integer multiple of it to 1e-9 relative); it is
 * ignored with geometric spacing.  BDF3 and the Adams methods need uniform
 * spacing and a problem of dimension <= 3 (INVALID_ARG otherwise).  Allocates about
 * 8 * N * (2 * (3d + p + 1) + 4) bytes of device memory.  Errors:
 * INVALID_ARG (dimensions do not match the ODE, N < 1 or > PF_MAX_PARTICLES,
 * bad prior or options), OOM, CUDA.  *out is NULL on error. */
pf_status pf_create(pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                    const pf_prior* prior, const pf_options* opt, pf_filter** out);

/* Device bytes a filter of this shape lays out: its ensembles (two
 * ping-pong copies of x, h1, h2, phi, w), work arrays and control block in one
 * block.  Host-only.  Errors: INVALID_ARG (NULL bytes, unsupported ode, d < 1,
 * p outside 1..5, N < 1). */
pf_status pf_device_bytes(pf_ode ode, int d, int p, int64_t N, size_t* bytes);
/* pf_create in caller-owned device memory: the filter lays all its device
 * arrays out in device_mem (at least pf_device_bytes(ode, d, p, N) bytes,
 * 256-byte aligned, on the current device) and never frees it; the caller
 * keeps it alive and unused elsewhere until pf_destroy returns.  Everything
 * else is as pf_create.  Errors: as pf_create, and INVALID_ARG for a NULL,
 * misaligned or too small device_mem, or one that is not device (or managed)
 * memory of the current device (checked before any device work). */
pf_status pf_create_with_buffers(pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                                 const pf_prior* prior, const pf_options* opt, void* device_mem,
                                 size_t device_bytes, pf_filter** out);

/* Assimilate one observation y_k (m host doubles) at time t_k > the previous
 * observation time: Steps 2-6 of Algorithm 1 (shrink, propagate, first-stage
 * weights, systematic resampling, proliferation, repropagation with the
 * local-error innovation, reweighting, moments).  Synchronous: returns after
 * the epoch is committed.  With timing off, the upload, the epoch's kernels and
 * the read-back run as one CUDA graph launch on the filter's stream (a graph is
 * captured the first time a substep count is seen; a few are kept).  Errors:
 * INVALID_ARG (non-finite y, bad t_k, substep count out of range), DEGENERATE
 * (all first- or second-stage weights zero; nothing committed), CUDA. */
pf_status pf_assimilate(pf_filter* f, double t_k, const double* y_k);

/* Weighted estimates of the committed ensemble (Step 6): theta_bar (p, in phi
 * space), C (p*p, phi space, weights summing to one, no Bessel factor) and the
 * weighted mean state x_bar (d).  Any pointer may be NULL.  Synchronous. */
pf_status pf_estimates(const pf_filter* f, double* theta_bar, double* C, double* x_bar);

typedef struct {
  int64_t epochs;        /* committed epochs                               */
  double ess;            /* 1 / sum w^2 of the committed weights           */
  double log_weight_sum; /* log sum of the unnormalised Step-5 weights     */
  int64_t unique_parents;/* distinct indices of the last resampling        */
  int64_t nonfinite;     /* particles given zero weight in the last epoch  */
  double theta_mean[8];  /* weighted mean of theta (model space)           */
  double last_epoch_ms;  /* device time of the last synchronous epoch (of
                            pf_assimilate: with its parameter upload and
                            read-back when timing is off and the epoch runs
                            as one graph)                                   */
  int64_t h2d_bytes;     /* host-to-device bytes copied since creation     */
  int64_t d2h_bytes;     /* device-to-host bytes copied since creation     */
  double ess_stage1;     /* (sum g)^2 / sum g^2 of the last epoch's first-stage
                            weights g (Step 3a), 0 before the first epoch   */
} pf_stats_t;
pf_status pf_stats(const pf_filter* f, pf_stats_t* out);

/* Per-kernel device time of the epochs run since the last call (requires
 * pf_options.timing).  Slot k of ms[] and launches[] (n entries, n >= 6):
 * 0 stage 1 (shrink, propagate, first-stage weights), 1 scan tiles, 2 scan
 * offsets (0: resampling applies the tile offsets as it reads the cumulative
 * weights, so this slot has no launch), 3 systematic resampling (with the
 * corner pass above one wave of merge tiles), 4 stage 2 (proliferate,
 * repropagate, innovation, reweight), 5 moments and commit (and the 2D
 * system's state mean).  With timing 2 only slot 4 is measured (the others
 * read 0 with 0 launches).  Waits for the filter's stream, then resets the
 * accumulators.  Errors: INVALID_ARG (n < 6), STATE (timing off), CUDA. */
#define PF_KERNEL_SLOTS 6
pf_status pf_kernel_times(pf_filter* f, double* ms, int64_t* launches, int n);

/* Text of the last error on this filter (or on this thread when f is NULL).
 * The pointer stays valid until the next call on the same filter/thread. */
const char* pf_last_error(const pf_filter* f);

/* Free the filter's device and host memory.  NULL is a no-op.  A filter that
 * is a member of a batch is destroyed only after its batch (pf_batch_destroy). */
void pf_destroy(pf_filter* f);

/* ---- device-resident observation series ---------------------------------
 * Upload T observations (times t[T], data y[T*m], row k = observation k) and
 * precompute every interval's substep table, so that pf_run can advance the
 * filter without any host-to-device traffic.  The series continues from the
 * filter's current time.  Errors: INVALID_ARG, OOM, CUDA. */
pf_status pf_load_observations(pf_filter* f, int T, const double* t, const double* y);

/* Enqueue epochs k0..k1-1 of the loaded series on the filter's stream and
 * return without waiting.  Epoch k0 must be the next unassimilated one.  A
 * failing epoch stops the rest (they become no-ops on the device).  Errors:
 * STATE (no series, or k0 out of order), INVALID_ARG, CUDA. */
pf_status pf_run(pf_filter* f, int k0, int k1);

/* Wait for enqueued work.  Returns the status of the first failed epoch (the
 * filter then rolls back to the last committed epoch), else PF_OK. */
pf_status pf_synchronize(pf_filter* f);

/* Redo Step 1 into the existing buffers (no allocation); the loaded series
 * restarts at observation 0. */
pf_status pf_reset(pf_filter* f);

/* ---- checkpoint and inspection ------------------------------------------
 * Copy the committed ensemble to or from host memory: x, h1, h2 (N*d each:
 * x_n and the two previous LMM substep states), phi (N*p) and the normalised
 * log weights logw (N).  Any pointer may be NULL (not copied).  Setting the
 * ensemble does not recompute the moments; use pf_set_moments. */
pf_status pf_get_ensemble(const pf_filter* f, double* x, double* h1, double* h2, double* phi,
                          double* logw);
pf_status pf_set_ensemble(pf_filter* f, const double* x, const double* h1, const double* h2,
                          const double* phi, const double* logw);
pf_status pf_set_moments(pf_filter* f, const double* phibar, const double* C);

/* Checkpoint and resume.  pf_save copies the committed state of f -- the
 * ensemble (states, LMM history, parameters, log weights), the moments and
 * their Cholesky factor, the weighted mean state, the epoch count and the LMM
 * history bookkeeping -- into a caller-owned host buffer of at least
 * pf_checkpoint_size bytes (about 8 * N * (3d + p + 1) bytes).  It waits for
 * the filter's stream first.  pf_load restores such a blob into a filter
 * created with the same problem, d, p, N, LMM, seed and filter id (checked:
 * INVALID_ARG otherwise) and discards any loaded observation series.  The
 * random streams are counter-based (seed, epoch, particle), so a resumed filter
 * continues bit-identically to one that was never interrupted.  The blob is
 * in this library's own layout and native byte order.  Errors: INVALID_ARG
 * (NULL, short or foreign buffer, mismatched filter), STATE (pf_save with a
 * failed epoch pending, pf_load into a batch member), CUDA. */
pf_status pf_checkpoint_size(const pf_filter* f, size_t* bytes);
pf_status pf_save(const pf_filter* f, void* buf, size_t bytes);
pf_status pf_load(pf_filter* f, const void* buf, size_t bytes);

/* Work arrays of the last epoch (N each): first-stage log-likelihoods, log
 * fitness weights, cumulative fitness weights c_k and resampled indices. */
pf_status pf_get_work(const pf_filter* f, double* loglik1, double* log_g, double* cumulative,
                      int32_t* idx);

/* LMM history bookkeeping: committed epoch count, history depth (0-2 stored
 * past points), time of the last observation and the last two step lengths.
 * (For the Adams methods the stored states also rebuild the derivative
 * history f_{n-1}, f_{n-2}, at t_n - h and t_n - 2h.) */
pf_status pf_get_history(const pf_filter* f, int64_t* epochs, int* depth, double* t_prev,
                         double* hprev1, double* hprev2);
pf_status pf_set_history(pf_filter* f, int64_t epochs, int depth, double t_prev, double hprev1,
                         double hprev2);

/* ---- host-only helper (no GPU needed) -----------------------------------
 * Substep table of one interval (t_prev, t_next] for the given history state,
 * as the filter builds it.  Per substep i, row i of coef (PF_SUBSTEP_ROW = 11
 * doubles): kind, h, gamma, rho1, rho2, pi0, pi1, pi2, mu, rho3, pi3.
 *  BDF kinds 1-3: x_{n+1} - rho1 x_n - rho2 x_{n-1} - rho3 x_{n-2}
 *    = gamma f(x_{n+1}); predictor pi0 x_n + pi1 x_{n-1} + pi2 x_{n-2}
 *    + pi3 f(x_n) (kind 1: Newton starts at x_n, predictor x_n + h f(x_n)).
 *  Adams kinds 10 + q (Moulton) and 20 + q (Bashforth), order q: predictor
 *    x_n + pi0 f_n + pi1 f_{n-1} + pi2 f_{n-2}; corrector x_n + gamma f_{n+1}
 *    + rho1 f_n + rho2 f_{n-1}.
 *  mu is Milne's factor: local error = mu (x_corr - x_pred).
 * Returns the substep count S (> 0) or -1; *depth_out gets the history depth
 * after the interval.  lmm, spacing, dt, substeps, q0 as in pf_create. */
#define PF_SUBSTEP_ROW 11
int pf_substep_table(int lmm, int spacing, double dt, int substeps, double q0, double t_prev,
                     double t_next, int depth, double hprev1, double hprev2, double* coef,
                     int max_steps, int* depth_out);

/* ---- batches of filters ---------------------------------------------------
 * A batch advances many independent filters (any mix of problems, LMMs and
 * sizes, except PF_ODE_ADVDIFF2D, whose one-block-per-particle kernels do not
 * batch: INVALID_ARG) by one epoch each with a handful of tile-scheduled
 * launches -- one per phase of Algorithm 1's epoch, split by problem and LMM
 * family where the kernels differ -- captured
 * in a CUDA graph that is reused while the set of active filters stays the
 * same.  On its first epoch the batch autotunes the launch shape (tile order,
 * concurrent per-model branches) by timing the candidates on that epoch.  Each filter's results are bit-identical to running it alone: its
 * reduction trees depend only on its own N.  The batch drives the filters'
 * own device buffers; while a filter is in a batch, advance it only through
 * the batch.  A filter belongs to at most one batch at a time. */
typedef struct pf_batch pf_batch;

typedef struct {
  int64_t epochs;         /* batched epochs run                            */
  int64_t graph_captures; /* times the launch graph was (re)captured       */
  double last_device_ms;  /* device time of the last batched epoch         */
  int last_active;        /* filters advanced by the last batched epoch    */
  int last_tiles;         /* thread blocks (tiles) of its launches         */
  int tile_order;         /* autotuned: 0 larger filters first, 1 interleaved */
  int concurrent_models;  /* autotuned: per-model launches as graph branches */
  double tune_ms[4];      /* autotuning times of the candidate shapes
                             (order, concurrent) = (0,0), (0,1), (1,0), (1,1) */
} pf_batch_stats_t;

/* Bind n existing filters (distinct, not in another batch) into a batch that
 * runs on `stream` (NULL = a stream the batch creates and owns).  The
 * filters' own pending work is waited for.  Errors: INVALID_ARG, OOM, CUDA. */
pf_status pf_batch_create(pf_filter* const* filters, int n, void* stream, pf_batch** out);

/* One epoch for every filter f with y[f] != NULL (host, m_f doubles) at time
 * t[f]; filters with y[f] == NULL idle.  Synchronous.  status[f] (n entries)
 * receives each filter's result (PF_OK, PF_ERR_INVALID_ARG for a bad
 * observation or time, PF_ERR_DEGENERATE, PF_ERR_NUMERIC); a failed filter
 * keeps its committed state, the others advance.  Returns PF_OK unless the
 * batch itself failed (CUDA, NULL arguments). */
pf_status pf_batch_assimilate(pf_batch* b, const double* t, const double* const* y, int* status);

pf_status pf_batch_stats(const pf_batch* b, pf_batch_stats_t* out);
const char* pf_batch_last_error(const pf_batch* b);
/* Release the batch (the filters stay valid and leave the batch). */
void pf_batch_destroy(pf_batch* b);

/* ---- serving: sessions admitted by memory budget, continuous batching -----
 * No counterpart in the paper, which runs one filter: the per-observation
 * epoch of Algorithm 1 is the unit of work, and observations arrive one at a
 * time (Section 2), so independent filters can be served as they arrive.
 * A server keeps filter sessions resident on the device and assimilates their
 * observations as they arrive.  Sessions are admitted in arrival order while
 * their device memory fits the budget, otherwise they wait until closed
 * sessions free memory; session memory comes from a stream-ordered pool owned
 * by the server, so admission and closing never synchronise the device.
 * Sessions are spread over `lanes` by model and size class (<= 32768 particles
 * or more); each lane is a batch with its own stream and at most one epoch in
 * flight, and lanes overlap on the device.  Observations queue per session
 * with their arrival time.  pf_server_step never waits: it collects the lanes
 * whose epoch has finished, admits waiting sessions, and launches on every
 * idle lane one batched epoch over its sessions that have a queued
 * observation (the oldest one of each), so requests that arrive while the
 * device works join the next launch of their lane.  The latency of an
 * assimilation runs from pf_server_submit to the moment the device finishes
 * its epoch (taken on the host by a stream callback).  Session results are
 * bit-identical to the same filter run alone.  One host thread drives a
 * server. */
typedef struct pf_server pf_server;

typedef struct {
  int64_t admitted, rejected, waiting, active_sessions, queued_observations;
  int64_t assimilations;        /* completed (latency samples)              */
  int64_t epochs;               /* batched epochs launched                  */
  double mean_sessions_per_epoch;
  double p50_ms, p99_ms, mean_ms, max_ms;  /* per-assimilation latency    */
  double particle_steps_per_s;  /* from the first submit to the last result */
  int64_t device_bytes_in_use, budget_bytes;
  int64_t step_calls;           /* pf_server_step calls                     */
  double step_ms_mean, step_ms_max;  /* host time inside pf_server_step     */
  double collect_ms_max, admit_ms_max, launch_ms_max;  /* its longest parts  */
} pf_server_stats_t;

/* budget_bytes: device memory the sessions may occupy (their filters' single
 * allocations); lanes: 1..64, or 0 for one lane per model and size class (6).
 * The sessions' memory comes from a stream-ordered pool owned by the server;
 * when the budget fits in 90 % of the free device memory, creation maps all of
 * it into the pool at once (so admissions never wait for the driver), and it
 * stays reserved until pf_server_destroy.  Errors: INVALID_ARG, OOM, CUDA. */
pf_status pf_server_create(int64_t budget_bytes, int lanes, pf_server** out);
/* Queue a session (arguments as pf_create; the options' stream and timing are
 * ignored).  It is admitted by a later pf_server_step when its memory fits.
 * Errors: INVALID_ARG, BUDGET (it can never fit the budget). */
pf_status pf_server_open(pf_server* s, pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                         const pf_prior* prior, const pf_options* opt, int64_t* session);
/* Queue observation y_k (m doubles, copied) at time t_k for a session. */
pf_status pf_server_submit(pf_server* s, int64_t session, double t_k, const double* y_k);
/* Collect, admit, launch (see above; never waits); *launched = sessions in
 * the epochs it launched. */
pf_status pf_server_step(pf_server* s, int* launched);
/* Step (waiting for the device between steps) until every admitted session's
 * queue is empty and nothing is in flight.  Errors: STATE if observations stay
 * queued while no epoch is in flight and a step launches none (no wait could
 * end), or any error of pf_server_step. */
pf_status pf_server_drain(pf_server* s);
/* Close a session: it leaves once its queue is done; its memory returns to
 * the budget. */
pf_status pf_server_close(pf_server* s, int64_t session);
/* A session's filter (borrowed; NULL while waiting for admission; for the
 * read-only calls pf_estimates/pf_get_ensemble/pf_get_history, made while the
 * session has nothing in flight, e.g. after pf_server_drain), its
 * assimilation count and last status. */
pf_status pf_server_session(const pf_server* s, int64_t session, pf_filter** filter,
                            int64_t* assimilated, int* last_status);
pf_status pf_server_stats(const pf_server* s, pf_server_stats_t* out);
const char* pf_server_last_error(const pf_server* s);
void pf_server_destroy(pf_server* s);

/* ---- systematic resampling without allocation ----------------------------
 * No counterpart in the paper: a library convenience for callers that cannot
 * allocate device memory where they need to resample -- applications whose
 * pool allocator owns all device memory and forbids other allocations,
 * latency-critical loops where cudaMalloc's implicit device-wide
 * synchronisation would stall their other streams, and callers that must not
 * fail with out-of-memory in the middle of a step.
 *
 * Computes, on `stream` (NULL = the legacy default stream) and without
 * waiting, the cumulative fitness weights c_k = sum_{i<=k} exp(log_g_i -
 * max log_g) and the systematic-resampling indices
 * idx_i = min{k : c_k > ((i + u)/N) c_{N-1}} (else the first k with
 * c_k = c_{N-1}), exactly as pf_assimilate does: for the same log weights and
 * u, c and idx are bit-identical.  All three buffers are device memory owned by
 * the caller: log_g (N doubles, read; finite or -inf, anything else counts as
 * a zero weight), cumulative (N doubles, written), idx (N int32, written).  If
 * every weight is zero, c is all zero and every index is 0.
 *
 * Nothing is allocated or freed.  The scratch (per-tile sums and offsets,
 * completion counters, merge-tile corners) is one fixed array of about 530 KB in the library's
 * device image; every GPU that loads the library holds it until the process
 * exits.  Every call looks up that array's device address on the current
 * device (so a device reset leaves no stale address behind); the first call on
 * a device may also load the library's device code, so make it before any
 * stream capture.
 * All calls share the array and it keeps the last call's contents, so calls
 * whose GPU work overlaps (unordered streams, several host threads) race and
 * corrupt each other's results: order them on one stream or synchronise in
 * between.  Errors: INVALID_ARG (NULL buffer, N < 1, u outside [0, 1)),
 * BUDGET (N > PF_NOALLOC_MAX_PARTICLES), CUDA (address lookup or launch). */
#define PF_NOALLOC_MAX_PARTICLES (1LL << 24)
pf_status pf_resample_systematic_noalloc(const double* log_g, int64_t N, double u,
                                         double* cumulative, int32_t* idx, void* stream);

/* ---- the systematic search alone ------------------------------------------
 * Algorithm 1, Step 3b: the parent index of each of the N resampled particles,
 * idx_i = min{k : c_k > tau_i} with tau_i = ((i + u)/N) c_{N-1} (else the first
 * k with c_k = c_{N-1}), for given cumulative weights c.  It is the filter's own
 * search (the merge-path kernel pf_assimilate launches), so for the same c and
 * u the indices are bit-identical to the filter's.  Runs on `stream` (NULL =
 * the legacy default stream) without waiting, allocating nothing: each block
 * finds its own tile corners, so beyond about 300k particles it is slower than
 * the filter's two-launch form (which keeps its corners in scratch).
 *
 * cumulative: N doubles of device memory, read; must be non-decreasing and
 * >= +0, as a cumulative sum of non-negative weights is (other input gives
 * unspecified indices, each still in [0, N)).  idx: N int32 of device memory,
 * written.  Both are owned by the caller.  Errors: INVALID_ARG (NULL buffer,
 * N < 1 or N > 2^31 - 1, u outside [0, 1)), CUDA (launch). */
pf_status pf_systematic_indices(const double* cumulative, int64_t N, double u, int32_t* idx,
                                void* stream);

/* ---- a particle-sharded filter -------------------------------------------
 * Algorithm 1's loops over particles are independent of one another (the
 * paper's particle-parallel layout, Sec. 3.1), so one filter of N particles
 * can be split into G contiguous shards, one per GPU, each a pf_filter over
 * the global slots [first, first + n).  Per epoch the shards share only:
 *  - Step 3a: the maximum of the log fitness weights (an exact max-reduce) and
 *    the tile totals of the cumulative weights (a gather, in slot order);
 *  - Step 3b/3c: the parent of every resampled slot, which may live on another
 *    shard: each shard resamples the outputs whose parent it holds and sends
 *    each parent's record to the shard of the output's slot (an all-to-all);
 *  - Steps 5-6: the maximum of the new log weights and the moment sums (a
 *    max-reduce and a gather, added in shard order).
 * The calls below run one phase each on `opt->stream` and return what the
 * other shards need; the caller does the exchange (over NCCL, gloo or host
 * memory) and must call them in this order, on every shard, each epoch:
 *   pf_shard_stage1 -> (max of lg_max) -> pf_shard_scan -> (gather the tiles)
 *   -> pf_shard_offsets -> (plan the output ranges) -> pf_shard_resample ->
 *   (all-to-all of the records) -> pf_shard_stage2 -> (max of lw_max) ->
 *   pf_shard_moments -> (add the sums) -> pf_shard_commit.
 * After pf_shard_create the order starts at pf_shard_moments (Step 1's
 * moments, lw_max = 0) and pf_shard_commit.  A call out of order returns
 * PF_ERR_STATE; if the global maximum of a stage is -inf (every weight zero)
 * the epoch is degenerate: call pf_shard_abort on every shard, which leaves
 * the committed state as it was.
 *
 * Random numbers are keyed by the global slot, and a shard starts on a tile
 * of the whole ensemble's scan (first a multiple of pf_shard_tile(N)), so the
 * cumulative weights, the resampled parents and every propagated state are
 * bit-identical to those of one filter of all N particles given the same
 * committed state; the moments, added in shard order, equal its to rounding.
 * The whole-filter calls pf_assimilate, pf_run, pf_load_observations,
 * pf_reset, pf_save and pf_load return PF_ERR_STATE on a shard, and a shard
 * cannot join a batch; pf_estimates, pf_get_ensemble (the shard's slots, log
 * weights normalised over the whole ensemble), pf_set_ensemble, pf_set_moments,
 * pf_get_history, pf_set_history, pf_stats and pf_get_work serve it. */

/* Tile length of the cumulative-weight scan of an ensemble of N particles:
 * shard boundaries must be multiples of it.  0 if N < 1. */
int64_t pf_shard_tile(int64_t N);

/* Create the shard holding the global slots [first, first + n) of a filter of
 * N particles (other arguments as pf_create; the ODE may not be
 * PF_ODE_ADVDIFF2D).  first must be a multiple of pf_shard_tile(N), and n too
 * unless first + n = N.  Step 1 is drawn for its slots; its moments are
 * committed by pf_shard_moments + pf_shard_commit.  Errors as pf_create. */
pf_status pf_shard_create(pf_ode ode, int d, int p, int64_t N, int64_t first, int64_t n, pf_lmm lmm,
                          double dt, const pf_prior* prior, const pf_options* opt, pf_filter** out);

/* The shard's shape: the whole ensemble's N, its first slot, its number of
 * scan tiles, the whole ensemble's number of tiles, and the doubles of one
 * parent record (3d + p + 2).  Any pointer may be NULL. */
pf_status pf_shard_info(const pf_filter* f, int64_t* total, int64_t* first, int* tiles,
                        int* tiles_all, int* record);

/* Steps 2 and 3a on the shard for the observation y_k (m doubles, host) at
 * t_k; *lg_max (host) gets the shard's largest log fitness weight (-inf if
 * every one of its weights is zero). */
pf_status pf_shard_stage1(pf_filter* f, double t_k, const double* y_k, double* lg_max);

/* Step 3a's tile pass with the global maximum lg_max (finite): tiles (host,
 * pf_shard_info's `tiles` doubles) gets this shard's tile totals, *cl_last
 * (host) the tile-local cumulative weight of its last slot. */
pf_status pf_shard_scan(pf_filter* f, double lg_max, double* tiles, double* cl_last);

/* The global cumulative weights from every shard's tile totals (tiles_all:
 * host, `tiles_all` doubles in slot order; cl_last: the last shard's): into
 * tile_end (host, tiles_all doubles) the cumulative weight at the last slot of
 * every tile, into *total the last one c_{N-1}, into *u the epoch's
 * resampling uniform (the same on every shard). */
pf_status pf_shard_offsets(pf_filter* f, const double* tiles_all, double cl_last, double* tile_end,
                           double* total, double* u);

/* Step 3b for the outputs i in [i_lo, i_hi) whose parent this shard holds:
 * l_i = min{k : c_k > ((i + u)/N) c_{N-1}}, or, for i >= i_fb (where that
 * threshold reaches c_{N-1}), the first k with c_k = c_{N-1}.  The parent's
 * record (x, h1, h2: d each; phi: p; ll1; the global parent slot) of output i
 * goes to send + (i - i_lo) * (3d + p + 2) (device memory the caller owns).
 * Errors: INVALID_ARG (range outside [0, N], u outside [0, 1), total <= 0,
 * NULL send with outputs), STATE, CUDA. */
pf_status pf_shard_resample(pf_filter* f, int64_t i_lo, int64_t i_hi, int64_t i_fb, double u,
                            double total, double* send);

/* Steps 3c-5 for this shard's slots from the parent records of its slots in
 * slot order (recv: device memory the caller owns, n records); *lw_max (host)
 * gets the shard's largest new log weight. */
pf_status pf_shard_stage2(pf_filter* f, const double* recv, double* lw_max);

/* Step 6's weighted sums of the shard's new ensemble with the global maximum
 * lw_max (finite; 0 for Step 1): into sums (host, *nv doubles: sum of
 * weights, of their squares, of the weighted parameters about the committed
 * mean, of their products, of the weighted states). */
pf_status pf_shard_moments(pf_filter* f, double lw_max, double* sums, int* nv);

/* Commit with the global sums (every shard's, added in shard order; host, nv
 * doubles): the new mean, C, its factor, x-bar, ESS and the normalisation,
 * identical on every shard.  Errors: NUMERIC (non-finite moments; nothing is
 * committed and the epoch may be redone), INVALID_ARG, STATE, CUDA. */
pf_status pf_shard_commit(pf_filter* f, const double* sums, int nv);

/* Drop the epoch in progress (a degenerate one): the committed state stays. */
pf_status pf_shard_abort(pf_filter* f);

/* The global parent slot of each of the shard's n slots in the last epoch
 * (host, n int32). */
pf_status pf_shard_parents(const pf_filter* f, int32_t* parents);

/* Library version string. */
const char* pf_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
