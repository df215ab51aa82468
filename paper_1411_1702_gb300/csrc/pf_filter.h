// pf_filter.h -- the library-owned filter object behind the opaque pf_filter
// handle (shared by the single-filter C ABI and the batch of filters).
#pragma once
#include <nvtx3/nvToolsExt.h>

#include <string>
#include <vector>

#include "pf_kernels.h"

namespace pfg {

// NVTX range over one host call (visible in Nsight Systems / Compute
// timelines; free when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// The first phases of a shard's epoch (pf_shard.cu): committed and idle, or
// Step 1 drawn with its moments still to be committed.
constexpr int kShardIdle = 0;
constexpr int kShardInitDrawn = 1;

struct HistoryState {
  int64_t epochs;
  int depth;
  double t_prev, hprev1, hprev2;
};

void set_thread_error(const std::string& msg);

}  // namespace pfg

struct pf_filter {
  // configuration
  int ode, d, p, m, lmm, K, spacing, substeps, history, transform, noise;
  double dt, q0, a, kappa;
  uint64_t seed;
  uint32_t filter_id;
  int64_t N;
  int obs[pfg::kMMax];
  double sigma[pfg::kMMax];
  int prior_kind[pfg::kPMax];
  double prior_lo[pfg::kPMax], prior_hi[pfg::kPMax];
  std::vector<double> x0;
  double t0;
  // CUDA resources
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool ext_mem = false;                    // dmem belongs to the caller (pf_create_with_buffers)
  cudaMemPool_t pool = nullptr;           // dmem is stream-ordered from this pool
  void* dmem = nullptr;
  size_t dbytes = 0;
  pfg::FilterDev fd{};
  pfg::EpochParams* ep_dev = nullptr;    // online parameter slot
  pfg::EpochParams* ep_host = nullptr;   // staging (pinned; pageable when pooled)
  pfg::Ctrl* ctrl_host = nullptr;        // pinned; pageable when pooled
  double* xbar_host = nullptr;           // pinned mirror of x-bar (not pooled)
  bool est_fresh = false;                 // ctrl_host and xbar_host hold the committed estimates
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // pf_assimilate's epoch as one CUDA graph (pinned host blocks, timing off):
  // the parameter upload, the kernels and the two read-backs, captured for a
  // substep count S and launched whenever an epoch has that S (a few S kept)
  static constexpr int kEpochGraphs = 4;
  cudaGraphExec_t epoch_exec[kEpochGraphs] = {};
  int epoch_exec_S[kEpochGraphs] = {};
  int epoch_exec_next = 0;
  cudaEvent_t ready = nullptr;            // pooled: the work queued on `stream` is done
  // committed history (host view)
  pfg::HistoryState hist{};
  // device-resident observation series
  pfg::EpochParams* series_dev = nullptr;
  int series_T = 0;
  int series_next = 0;
  std::vector<int> series_S;
  std::vector<pfg::HistoryState> series_after;  // history after epoch k of the series
  pfg::HistoryState series_start{};
  // per-kernel timing (pf_options.timing)
  int timing = 0;  // pf_options.timing: 0 off, 1 every kernel, 2 stage 2 only
  std::vector<cudaEvent_t*> mark_free;     // sets of kEpochKernels + 1 events
  std::vector<cudaEvent_t*> mark_pending;  // recorded, not yet read
  double kernel_ms[pfg::kEpochKernels] = {0};
  int64_t kernel_launches[pfg::kEpochKernels] = {0};
  // bookkeeping
  double last_ms = 0.0;
  int64_t h2d_bytes = 0, d2h_bytes = 0;
  bool in_batch = false;                  // epochs are driven by a pf_batch
  // a shard of a particle-sharded filter (pf_shard_create): the global slots
  // [shard_first, shard_first + N) of an ensemble of shard_total particles
  int64_t shard_total = 0;                // 0: a filter of its own
  int64_t shard_first = 0;
  int shard_tiles_all = 0;                // scan tiles of the whole ensemble
  pfg::Ensemble sh_parent{};              // received parents by slot (SoA)
  double* sh_parent_ll1 = nullptr;
  int32_t* sh_gparent = nullptr;          // global parent slot of each slot
  double* sh_tiles = nullptr;             // every shard's tile totals (upload)
  double* sh_boff = nullptr;              // the whole ensemble's tile offsets
  double* sh_pmax = nullptr;              // and floors
  double* sh_out = nullptr;               // tile ends, c_{N-1}, u
  double* sh_sums = nullptr;              // moment sums (this shard's, then the global ones)
  int sh_stage = 0;                       // last stage call of the epoch in progress
  int sh_depth_out = 0;                   // history after the epoch in progress
  double sh_t = 0.0;
  std::string err;
};

namespace pfg {
// Parameter block of one epoch of f from history h (host); returns S or -1.
int fill_epoch(const pf_filter* f, const HistoryState& h, double t_k, const double* y,
               EpochParams* ep, int* depth_out);
// Argument checks of pf_create (no allocation, no CUDA call).
pf_status check_create_args(pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                            const pf_prior* prior, const pf_options* opt);
// pf_create with the device allocation taken, stream-ordered, from `pool` and
// pageable host staging, so that neither creation nor pf_destroy makes an
// implicitly device-wide synchronising call (the server's sessions).  A NULL
// pool is pf_create.  ext_mem (with ext_bytes) is caller-owned device memory
// the filter lays itself out in instead (pf_create_with_buffers).
// shard_total > 0 makes a shard of that many particles holding the global
// slots [shard_first, shard_first + N): Step 1 draws its particles but leaves
// the commit to pf_shard_commit with the global moment sums.
pf_status filter_create(pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                        const pf_prior* prior, const pf_options* opt, cudaMemPool_t pool,
                        pf_filter** out, void* ext_mem = nullptr, size_t ext_bytes = 0,
                        int64_t shard_total = 0, int64_t shard_first = 0);
// a fail() for other translation units: records msg on f (or the thread)
pf_status record_error(pf_filter* f, pf_status st, const std::string& msg);
// The control block into f->ctrl_host (waits for the stream).
pf_status read_control(pf_filter* f);
// Device bytes of a filter of this shape (its single allocation).
size_t filter_device_bytes(int ode, int d, int p, int64_t N);
// History after an epoch with parameter block ep.
HistoryState advance_history(const HistoryState& h, double t_k, const EpochParams* ep, int depth_out);
}  // namespace pfg
