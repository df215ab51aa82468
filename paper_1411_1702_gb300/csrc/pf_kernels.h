// pf_kernels.h -- launch interface between the C ABI and the kernels.
#pragma once
#include <string>

#include "pf_common.cuh"

namespace pfg {

// phases of an epoch (and Step 1), in launch order
enum : int {
  kPhaseStage1 = 0,
  kPhaseScanTile = 1,
  kPhaseScanAdd = 2,  // (no launch: folded into the readers of c)
  kPhaseResample = 3,
  kPhaseStage2 = 4,
  kPhaseMoments = 5,
  kPhaseInit = 6
};

// one block of a batched launch: filter index and its virtual block index
struct BatchTile {
  int f;
  int vb;
};

// blocks one filter of N particles needs in a phase
// on a device of sms SMs
int phase_blocks(int phase, int ode, int64_t N, int sms);
int bruss_stage_blocks(int64_t N);
// One batched phase over a device tile table (see pf_kernels.cu); stage
// phases take the tiles of one model (ode) and LMM family (that of lmm), the
// moments those of one model.
cudaError_t launch_batch_phase(int phase, int ode, int lmm, const FilterDev* fds,
                               const EpochParams* const* eps, const BatchTile* tiles, int ntiles,
                               size_t smem, int is_init, cudaStream_t st);
// Batched Brusselator stage (1 or 2) over its own tile table (pf_bruss.cu).
cudaError_t launch_batch_bruss_stage(int stage, const FilterDev* fds, const EpochParams* const* eps,
                                     const BatchTile* tiles, int ntiles, size_t smem,
                                     cudaStream_t st);

// Step 1 of Algorithm 1 into the pending buffer, then the moments and commit.
cudaError_t launch_init(int ode, const FilterDev& fd, cudaStream_t st);
// One epoch (Steps 2-6) with the parameter block ep (device) of S substeps.
// If marks is not NULL, marks[i] is recorded before phase i and marks[6]
// after the last (phase order: stage1, scan_tile, scan_add, resample, stage2,
// moments).  scan_add is empty -- the offsets are applied where c is read --
// and marks[3] is not recorded; the slot stays so that pf_kernel_times keeps
// its layout.
constexpr int kEpochKernels = 6;
cudaError_t launch_epoch(int ode, const FilterDev& fd, const EpochParams* ep, int S, cudaStream_t st,
                         cudaEvent_t* marks = nullptr);
// Recompute the Cholesky factor after the host set phibar and C.
cudaError_t launch_set_moments(const FilterDev& fd, cudaStream_t st);
// sum of the squared first-stage weights of the last epoch into Ctrl::g_sq
cudaError_t launch_stage1_ess(const FilterDev& fd, cudaStream_t st);

// Host-to-device copy of at most kUploadBytes bytes carried as a kernel
// parameter: never synchronises, whatever memory src is in (a copy from
// pageable memory may wait for its stream).
constexpr int kUploadBytes = 2048;
cudaError_t upload_small(void* dst, const void* src, size_t bytes, cudaStream_t st);
int moment_record_size(int ode);
// Weighted theta-space mean of the committed ensemble into Ctrl::theta_mean.
cudaError_t launch_theta_mean(const FilterDev& fd, cudaStream_t st);
// Load every kernel of the library on the current device now rather than at
// its first launch (which may wait for the device to drain); once per device.
cudaError_t preload_main_kernels();
// Let kernel k stage a full substep table (PF_MAX_SUBSTEPS entries) in dynamic
// shared memory; loads the kernel.
cudaError_t allow_step_table(const void* k);
cudaError_t preload_bruss_kernels();
cudaError_t preload_kernels();
// Brusselator stage kernels (pf_bruss.cu): stage 1 or 2 of one epoch.
cudaError_t launch_bruss_stage(int stage, const FilterDev& fd, const EpochParams* ep, int S,
                               cudaStream_t st);
size_t bruss_work_doubles(int64_t N);
// 2D advection-diffusion stage kernels (pf_advdiff.cu): one block per
// particle, the whole state in shared memory.
cudaError_t launch_ad_stage(int stage, const FilterDev& fd, const EpochParams* ep, int S,
                            cudaStream_t st);
size_t ad_stage_smem(int d, int S, int stage);
int ad_threads(int nt);
cudaError_t preload_ad_kernels();
int max_grid_blocks(int64_t N, int sms);
int scan_tiles(int64_t N, int sms);
// SM count of the current device (1024 when there is none, the most the
// fixed-size scratch of the no-alloc call is laid out for)
int device_sms();
int kernels_per_epoch(int ode);
bool ode_supported(int ode);

// A shard of a particle-sharded filter (pf_shard.cu drives these).
cudaError_t launch_init_draws(int ode, const FilterDev& fd, cudaStream_t st);
cudaError_t launch_stage(int stage, const FilterDev& fd, const EpochParams* ep, int S,
                         cudaStream_t st);
cudaError_t launch_scan_tiles(const FilterDev& fd, int ntiles, cudaStream_t st);
cudaError_t launch_shard_offsets(const FilterDev& fd, const EpochParams* ep, const double* tiles,
                                 int nb, double cl_last, double* boff_all, double* pmax_all,
                                 double* out, cudaStream_t st);
cudaError_t launch_shard_resample(const FilterDev& fd, int64_t i_lo, int64_t cnt, int64_t i_fb,
                                  double u, double total, int64_t n_all, double* send,
                                  cudaStream_t st);
cudaError_t launch_shard_unpack(const FilterDev& fd, const double* recv, const Ensemble& par,
                                double* par_ll1, int32_t* gparent, cudaStream_t st);
cudaError_t launch_shard_moments(const FilterDev& fd, cudaStream_t st);
cudaError_t launch_shard_commit(const FilterDev& fd, const double* sums, int is_init, cudaStream_t st);

// Substep table of one observation interval (host code, pf_grid.cu).
int build_substeps(int lmm, int spacing, double dt, int substeps, double q0, double t_prev,
                   double t_next, int depth, double hprev1, double hprev2, StepCoef* tab,
                   int max_steps, int* depth_out, double* times_out = nullptr);
bool lmm_known(int lmm);
bool lmm_needs_uniform(int lmm);
// M1's input Phi(t) (host, pf_grid.cu)
double mm_input(double t);

}  // namespace pfg
