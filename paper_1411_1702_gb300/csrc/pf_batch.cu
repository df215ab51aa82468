// pf_batch.cu -- many filters advanced together, and the serving loop built
// on top of them.
//
// Batch.  One epoch of every member filter with a new observation runs as a
// handful of tile-scheduled launches (one per phase, split by model where the
// kernels differ).  The batch drives the filters' own device buffers.  Per
// epoch the host
//  1. builds each active filter's parameter block (substep table, y, 1/sigma)
//     into a pinned slot and uploads every slot with one strided copy;
//  2. rebuilds the tile tables (filter, virtual block) when the set of active
//     filters changes;
//  3. launches the phases -- from a captured CUDA graph when the active set
//     repeats, directly otherwise; on its first epoch a batch created with
//     autotuning times the candidate launch shapes (tile order within a phase;
//     per-model launches back to back or as concurrent graph branches) on the
//     real epoch's phases up to stage 2 (none of which touches the committed
//     state) and keeps the fastest;
//  4. gathers every member's status and epoch count with one kernel and one
//     read-back, and commits the host-side history of the filters that
//     succeeded.
// A filter's results are bit-identical alone and in a batch (its reductions
// depend only on its own N; see pf_kernels.cu).  Members can join and leave
// between epochs (slots), which the server uses for continuous batching.
//
// Server.  Sessions (filters) are admitted against a device-memory budget and
// wait in arrival order while they do not fit; their memory comes from a
// stream-ordered pool, so admitting and closing sessions never synchronises the
// device.  Observations queue per session with their arrival time.  Sessions
// are spread over lanes by model and size class; a lane is a batch with its
// own stream and at most one epoch in flight, so lanes overlap on the device
// and a long epoch of large filters does not hold back small ones.
// pf_server_step never waits: it collects the lanes whose epoch has finished
// (the completion time of each assimilation is taken on the host by a stream
// callback as soon as the device reaches it), admits waiting sessions whose
// memory is now free, and launches on every idle lane one batched epoch over
// its sessions with a queued observation, so requests that arrive while the
// device works join the next launch of their lane.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>

#include "pf_filter.h"

using namespace pfg;

namespace pfg {

__global__ void k_batch_status(const FilterDev* __restrict__ fds, const int* __restrict__ slots,
                               int n, int64_t* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const Ctrl* c = fds[slots[i]].ctrl;
    out[2 * i] = c->status;
    out[2 * i + 1] = c->epochs_done;
  }
}

__global__ void k_batch_clear(const FilterDev* __restrict__ fds, const int* __restrict__ which, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const FilterDev& fd = fds[which[i]];
    fd.ctrl->status = PF_OK;
    for (int k = 0; k < 8; ++k) fd.ticket[k] = 0u;
  }
}

}  // namespace pfg

namespace {

// Launch groups: the stage kernels differ by problem and LMM family, the
// moments kernel by problem.  Group g's kernels are those of (kGroupOde[g],
// kGroupLmm[g]).
constexpr int kStageGroups = 13;
constexpr int kGroupOde[kStageGroups] = {1, 1, 1, 1, 2, 2, 2, 2, 3, 5, 5, 5, 5};
constexpr int kGroupLmm[kStageGroups] = {2, 3, 12, 22, 2, 3, 12, 22, 2, 2, 3, 12, 22};
constexpr int kMomentGroups = 4;
constexpr int kMomentOde[kMomentGroups] = {1, 2, 3, 5};
int family_of(int lmm) { return lmm == PF_LMM_BDF3 ? 1 : lmm / 10 == 1 ? 2 : lmm / 10 == 2 ? 3 : 0; }
int stage_group(int ode, int lmm) {
  const int fam = family_of(lmm);
  switch (ode) {
    case PF_ODE_LINEAR2: return fam;
    case PF_ODE_ROBERTSON: return 4 + fam;
    case PF_ODE_BRUSSELATOR1D: return 8;
    case PF_ODE_MICHAELIS3: return 9 + fam;
  }
  return -1;
}
int moment_group(int ode) {
  for (int g = 0; g < kMomentGroups; ++g)
    if (kMomentOde[g] == ode) return g;
  return -1;
}
// cost classes of the server's lanes: linear2, Robertson and M1, Brusselator
constexpr int kCostModels = 3;
int cost_model(int ode) {
  return ode == PF_ODE_BRUSSELATOR1D ? 2 : ode == PF_ODE_LINEAR2 ? 0 : 1;
}
constexpr size_t kInitialTiles = 1 << 18;

struct Range {
  int off = 0, cnt = 0;
};

// launch shape chosen by the autotuner
struct Shape {
  int order;       // 0: larger filters first; 1: filters interleaved block by block
  int concurrent;  // per-model launches of a phase as parallel graph branches
};
const Shape kShapes[] = {{0, 0}, {0, 1}, {1, 0}, {1, 1}};

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

namespace {

// A few host threads that build the members' parameter blocks of an epoch in
// parallel (a block is a substep table of tens of entries: about a
// microsecond each, which adds up for hundreds of members).  run() splits
// [0, count) into one range per worker and one for the caller and returns
// once all are done; it is called by one thread at a time.
class FillPool {
 public:
  explicit FillPool(int workers) {
    try {
      for (int w = 0; w < workers; ++w) th_.emplace_back([this, w] { loop(w + 1); });
    } catch (...) {
      stop_all();  // the threads that did start
      throw;
    }
  }
  ~FillPool() { stop_all(); }
  void run(int count, const std::function<void(int, int)>& fn) {
    {
      std::lock_guard<std::mutex> g(m_);
      fn_ = &fn;
      count_ = count;
      left_ = (int)th_.size();
      ++gen_;
    }
    cv_.notify_all();
    fn(lo(0), lo(1));
    std::unique_lock<std::mutex> lk(m_);
    done_.wait(lk, [this] { return left_ == 0; });
    fn_ = nullptr;
  }

 private:
  void stop_all() {
    {
      std::lock_guard<std::mutex> g(m_);
      stop_ = true;
      ++gen_;
    }
    cv_.notify_all();
    for (std::thread& t : th_) t.join();
    th_.clear();
  }
  int lo(int part) const { return (int)((int64_t)count_ * part / ((int)th_.size() + 1)); }
  void loop(int part) {
    int seen = 0;
    std::unique_lock<std::mutex> lk(m_);
    for (;;) {
      cv_.wait(lk, [&] { return gen_ != seen; });
      seen = gen_;
      if (stop_) return;
      const std::function<void(int, int)>* fn = fn_;
      const int a = lo(part), b = lo(part + 1);
      lk.unlock();
      (*fn)(a, b);
      lk.lock();
      if (--left_ == 0) done_.notify_one();
    }
  }
  std::vector<std::thread> th_;
  std::mutex m_;
  std::condition_variable cv_, done_;
  const std::function<void(int, int)>* fn_ = nullptr;
  int count_ = 0, left_ = 0, gen_ = 0;
  bool stop_ = false;
};

// members with an observation from which the parameter blocks are built in
// parallel, and the pool's worker threads
constexpr int kParallelFill = 128;
constexpr int kFillWorkers = 3;

}  // namespace

struct pf_batch {
  int cap = 0;                           // slots
  std::vector<pf_filter*> slot;          // nullptr = free slot
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;           // second branch of the captured graph
  cudaEvent_t fork = nullptr, join = nullptr;
  Shape shape{0, 1};
  bool autotune = true, tuned = false;
  double tune_ms[4] = {0, 0, 0, 0};
  FilterDev* fds_dev = nullptr;          // cap descriptors
  EpochParams** eps_dev = nullptr;       // cap pointers into params_dev
  EpochParams* params_dev = nullptr;     // cap parameter slots
  EpochParams* params_host = nullptr;    // pinned mirror
  BatchTile* tiles_dev = nullptr;
  size_t tiles_cap = 0;
  std::vector<BatchTile> tiles_host;
  BatchTile* tiles_pin = nullptr;        // pinned staging of the tile upload (tiles_cap)
  Range stage[2][kStageGroups];
  Range moments[kMomentGroups];
  Range scan_tile, resample;
  int* slots_dev = nullptr;              // active slots of the epoch in flight
  int* slots_pin = nullptr;              // pinned staging (cap)
  int64_t* status_dev = nullptr;
  int64_t* status_host = nullptr;        // pinned
  int* clear_dev = nullptr;
  // tiles and graph of the last active set
  std::vector<char> tiles_active;
  size_t tiles_smem = 0;
  cudaGraphExec_t graph = nullptr;
  int64_t captures = 0, epochs = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEvent_t ev_done = nullptr;         // after the status read-back of the epoch in flight
  double last_ms = 0.0;
  int last_active = 0, last_tiles = 0;
  // epoch in flight (launch -> collect)
  bool in_flight = false;
  std::vector<int> fl_slots, fl_depth;
  std::vector<double> fl_t;
  double fl_done_ms = 0.0;               // host time the device finished (callback)
  std::vector<int> fl_S;                 // per slot: its epoch's S, -1 invalid, -2 idle
  std::unique_ptr<FillPool> fill_pool;   // created at the first epoch with many members
  std::string err;
};

static pf_status bfail(pf_batch* b, pf_status st, const std::string& msg) {
  if (b) b->err = msg;
  else set_thread_error(msg);
  return st;
}

#define PF_BCUDA(b, call)                                                                  \
  do {                                                                                     \
    cudaError_t e__ = (call);                                                              \
    if (e__ != cudaSuccess)                                                                \
      return bfail(b, PF_ERR_CUDA, std::string("CUDA error in ") + #call + ": " +         \
                                       cudaGetErrorName(e__) + " (" + cudaGetErrorString(e__) + ")"); \
  } while (0)

// Tile tables of one active set: per phase (and per model for the stages and
// the moments), the filters' virtual blocks, either larger filters first (the
// longest tails start early) or interleaved block by block across filters.
static void build_tiles(pf_batch* b, const std::vector<char>& active, int order_kind) {
  std::vector<int> order;
  for (int f = 0; f < b->cap; ++f)
    if (active[f]) order.push_back(f);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->slot[x]->N > b->slot[y]->N; });
  b->tiles_host.clear();
  // group: -1 every filter; else the stage group (stage phases) or the
  // moment group (moments) the filter must belong to
  auto member = [&](const pf_filter* F, int phase, int group) {
    if (group < 0) return true;
    return phase == kPhaseMoments ? moment_group(F->ode) == group : stage_group(F->ode, F->lmm) == group;
  };
  auto add = [&](int phase, int model) {
    Range r;
    r.off = (int)b->tiles_host.size();
    if (order_kind == 0) {
      for (int f : order) {
        const pf_filter* F = b->slot[f];
        if (!member(F, phase, model)) continue;
        const int nb = phase_blocks(phase, F->ode, F->N, F->fd.sms);
        for (int v = 0; v < nb; ++v) b->tiles_host.push_back(BatchTile{f, v});
      }
    } else {
      int most = 0;
      for (int f : order)
        most = std::max(most, phase_blocks(phase, b->slot[f]->ode, b->slot[f]->N, b->slot[f]->fd.sms));
      for (int v = 0; v < most; ++v)
        for (int f : order) {
          const pf_filter* F = b->slot[f];
          if (!member(F, phase, model)) continue;
          if (v < phase_blocks(phase, F->ode, F->N, F->fd.sms)) b->tiles_host.push_back(BatchTile{f, v});
        }
    }
    r.cnt = (int)b->tiles_host.size() - r.off;
    return r;
  };
  for (int g = 0; g < kStageGroups; ++g) b->stage[0][g] = add(kPhaseStage1, g);
  b->scan_tile = add(kPhaseScanTile, -1);
  b->resample = add(kPhaseResample, -1);
  for (int g = 0; g < kStageGroups; ++g) b->stage[1][g] = add(kPhaseStage2, g);
  for (int g = 0; g < kMomentGroups; ++g) b->moments[g] = add(kPhaseMoments, g);
}

// Host copies go through pinned staging, so they never wait for the device.
static cudaError_t upload_tiles(pf_batch* b) {
  const size_t need = b->tiles_host.size();
  if (need > b->tiles_cap) {
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return e;
    cudaFree(b->tiles_dev);
    if (b->tiles_pin) cudaFreeHost(b->tiles_pin);
    b->tiles_dev = nullptr;
    b->tiles_pin = nullptr;
    const size_t cap = std::max(need, 2 * b->tiles_cap);
    e = cudaMalloc(&b->tiles_dev, sizeof(BatchTile) * cap);
    if (e == cudaSuccess) e = cudaMallocHost(&b->tiles_pin, sizeof(BatchTile) * cap);
    if (e != cudaSuccess) {
      b->tiles_cap = 0;
      return e;
    }
    b->tiles_cap = cap;
  }
  std::memcpy(b->tiles_pin, b->tiles_host.data(), sizeof(BatchTile) * need);
  return cudaMemcpyAsync(b->tiles_dev, b->tiles_pin, sizeof(BatchTile) * need,
                         cudaMemcpyHostToDevice, b->stream);
}

// Enqueue the phases on b->stream.  With a concurrent shape, each per-model
// group of a phase forks onto two branches (the model with the most tiles on
// the main branch) and joins before the next phase.
static cudaError_t launch_phases(pf_batch* b, size_t smem, const Shape& shape, bool with_moments) {
  const FilterDev* fds = b->fds_dev;
  const EpochParams* const* eps = b->eps_dev;
  const BatchTile* T = b->tiles_dev;
  cudaError_t e = cudaSuccess;
  auto run = [&](int phase, int ode, int lmm, const Range& r, cudaStream_t st) {
    if (e == cudaSuccess && r.cnt > 0)
      e = launch_batch_phase(phase, ode, lmm, fds, eps, T + r.off, r.cnt, smem, 0, st);
  };
  // the groups of a phase, the largest on the main branch and (concurrent
  // shape) the others on the side branch
  auto per_model = [&](int phase, const Range* rs, int ngroups, const int* odes, const int* lmms) {
    int used = 0, big = -1;
    for (int m = 0; m < ngroups; ++m)
      if (rs[m].cnt > 0) {
        ++used;
        if (big < 0 || rs[m].cnt > rs[big].cnt) big = m;
      }
    auto lmm_of = [&](int m) { return lmms ? lmms[m] : PF_LMM_BDF2; };
    if (!shape.concurrent || used < 2) {
      for (int m = 0; m < ngroups; ++m) run(phase, odes[m], lmm_of(m), rs[m], b->stream);
      return;
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
    run(phase, odes[big], lmm_of(big), rs[big], b->stream);
    for (int m = 0; m < ngroups; ++m)
      if (m != big) run(phase, odes[m], lmm_of(m), rs[m], b->side);
    if (e == cudaSuccess) e = cudaEventRecord(b->join, b->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join, 0);
  };
  per_model(kPhaseStage1, b->stage[0], kStageGroups, kGroupOde, kGroupLmm);
  run(kPhaseScanTile, 0, 0, b->scan_tile, b->stream);
  run(kPhaseResample, 0, 0, b->resample, b->stream);
  per_model(kPhaseStage2, b->stage[1], kStageGroups, kGroupOde, kGroupLmm);
  if (with_moments) per_model(kPhaseMoments, b->moments, kMomentGroups, kMomentOde, nullptr);
  return e;
}

static cudaError_t capture(pf_batch* b, size_t smem, const Shape& shape, bool with_moments,
                           cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = launch_phases(b, smem, shape, with_moments);
  e = cudaStreamEndCapture(b->stream, &g);
  if (le != cudaSuccess) e = le;
  if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

// Time each launch shape on the pending epoch's phases up to stage 2 (they
// leave the committed state untouched and are idempotent), keep the fastest.
static cudaError_t run_autotune(pf_batch* b, const std::vector<char>& active, size_t smem) {
  double best = 1e300;
  int best_i = 0;
  for (int i = 0; i < 4; ++i) {
    build_tiles(b, active, kShapes[i].order);
    cudaError_t e = upload_tiles(b);
    cudaGraphExec_t gx = nullptr;
    if (e == cudaSuccess) e = capture(b, smem, kShapes[i], false, &gx);
    double t = 1e300;
    for (int rep = 0; e == cudaSuccess && rep < 2; ++rep) {
      e = cudaEventRecord(b->ev0, b->stream);
      if (e == cudaSuccess) e = cudaGraphLaunch(gx, b->stream);
      if (e == cudaSuccess) e = cudaEventRecord(b->ev1, b->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(b->ev1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, b->ev0, b->ev1);
      if (e == cudaSuccess) t = std::min(t, (double)ms);
    }
    if (gx) cudaGraphExecDestroy(gx);
    if (e != cudaSuccess) return e;
    b->tune_ms[i] = t;
    if (t < best) {
      best = t;
      best_i = i;
    }
  }
  b->shape = kShapes[best_i];
  b->tuned = true;
  b->tiles_active.clear();  // the tables now hold the last candidate's order
  return cudaSuccess;
}

// The tile tables and the graph describe the members of the slots they were
// built for; a membership change invalidates them (the next launch rebuilds
// the tables and drops the graph, after any epoch in flight has been queued).
static void forget_tiles(pf_batch* b) { b->tiles_active.clear(); }

// Grow every per-slot array to hold at least `want` slots.
static cudaError_t grow(pf_batch* b, int want) {
  if (want <= b->cap) return cudaSuccess;
  const int cap = std::max(want, 2 * b->cap);
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return e;
  FilterDev* fds = nullptr;
  EpochParams** eps = nullptr;
  EpochParams* pd = nullptr;
  EpochParams* ph = nullptr;
  int *slots = nullptr, *clear = nullptr, *spin = nullptr;
  int64_t *sd = nullptr, *sh = nullptr;
  e = cudaMalloc(&fds, sizeof(FilterDev) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&eps, sizeof(EpochParams*) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&pd, sizeof(EpochParams) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&slots, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&clear, sizeof(int) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&sd, sizeof(int64_t) * 2 * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&ph, sizeof(EpochParams) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&sh, sizeof(int64_t) * 2 * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&spin, sizeof(int) * cap);
  if (e != cudaSuccess) {
    cudaFree(fds); cudaFree(eps); cudaFree(pd); cudaFree(slots); cudaFree(clear); cudaFree(sd);
    if (ph) cudaFreeHost(ph);
    if (sh) cudaFreeHost(sh);
    if (spin) cudaFreeHost(spin);
    return e;
  }
  std::memset(ph, 0, sizeof(EpochParams) * cap);
  std::vector<FilterDev> hd(cap);
  std::vector<EpochParams*> he(cap);
  for (int i = 0; i < cap; ++i) {
    if (i < b->cap && b->slot[i]) hd[i] = b->slot[i]->fd;
    else std::memset(&hd[i], 0, sizeof(FilterDev));
    he[i] = pd + i;
  }
  e = cudaMemcpyAsync(fds, hd.data(), sizeof(FilterDev) * cap, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(eps, he.data(), sizeof(EpochParams*) * cap, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(b->fds_dev); cudaFree(b->eps_dev); cudaFree(b->params_dev); cudaFree(b->slots_dev);
  cudaFree(b->clear_dev); cudaFree(b->status_dev);
  if (b->params_host) cudaFreeHost(b->params_host);
  if (b->status_host) cudaFreeHost(b->status_host);
  if (b->slots_pin) cudaFreeHost(b->slots_pin);
  b->slots_pin = spin;
  b->fds_dev = fds; b->eps_dev = eps; b->params_dev = pd; b->slots_dev = slots;
  b->clear_dev = clear; b->status_dev = sd; b->params_host = ph; b->status_host = sh;
  b->slot.resize(cap, nullptr);
  b->cap = cap;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  forget_tiles(b);
  return e;
}

// stream == NULL: the batch creates its streams with the given priority.
static pf_status batch_new(void* stream, int cap, bool autotune, int priority, pf_batch** out) {
  pf_batch* b = new (std::nothrow) pf_batch();
  if (!b) return bfail(nullptr, PF_ERR_OOM, "host allocation failed");
  b->autotune = autotune;
  cudaError_t e = preload_kernels();
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(k_batch_status));
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(k_batch_clear));
  if (e != cudaSuccess) {
  } else if (stream) {
    b->stream = (cudaStream_t)stream;
    e = cudaStreamGetPriority(b->stream, &priority);
  } else {
    e = cudaStreamCreateWithPriority(&b->stream, cudaStreamNonBlocking, priority);
    b->own_stream = (e == cudaSuccess);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&b->side, cudaStreamNonBlocking, priority);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = grow(b, std::max(cap, 1));
  if (e == cudaSuccess) {  // room for the tiles of a few hundred thousand blocks
    e = cudaMalloc(&b->tiles_dev, sizeof(BatchTile) * kInitialTiles);
    if (e == cudaSuccess) e = cudaMallocHost(&b->tiles_pin, sizeof(BatchTile) * kInitialTiles);
    b->tiles_cap = e == cudaSuccess ? kInitialTiles : 0;
  }
  if (e != cudaSuccess) {
    set_thread_error(std::string("batch creation failed: ") + cudaGetErrorString(e));
    pf_batch_destroy(b);
    return PF_ERR_CUDA;
  }
  *out = b;
  return PF_OK;
}

// Add f to a free slot (growing the slots when none is free, which waits for
// the epoch in flight).  An epoch in flight is not disturbed: the descriptor
// goes to a slot it does not use, on the filter's own stream, and the tile
// tables are rebuilt at the next launch.
static pf_status batch_add(pf_batch* b, pf_filter* f, int* slot_out) {
  if (!f) return bfail(b, PF_ERR_INVALID_ARG, "NULL filter");
  if (f->in_batch) return bfail(b, PF_ERR_INVALID_ARG, "filter already in a batch");
  if (f->ode == PF_ODE_ADVDIFF2D)
    return bfail(b, PF_ERR_INVALID_ARG, "2D advection-diffusion filters do not batch (one block per particle)");
  int s = -1;
  for (int i = 0; i < b->cap; ++i)
    if (!b->slot[i]) {
      s = i;
      break;
    }
  if (s < 0) {
    if (b->in_flight) return bfail(b, PF_ERR_STATE, "no free slot while an epoch is in flight");
    s = b->cap;
    PF_BCUDA(b, grow(b, b->cap + 1));
  }
  static_assert(sizeof(FilterDev) <= (size_t)kUploadBytes, "FilterDev fits a parameter upload");
  PF_BCUDA(b, upload_small(b->fds_dev + s, &f->fd, sizeof(FilterDev), f->stream));
  if (f->ready) {
    // the batch's next launch waits, on the device, for the filter's pending
    // work (its initialisation) and the descriptor
    PF_BCUDA(b, cudaEventRecord(f->ready, f->stream));
    PF_BCUDA(b, cudaStreamWaitEvent(b->stream, f->ready, 0));
  } else {
    PF_BCUDA(b, cudaStreamSynchronize(f->stream));  // also the filter's own pending work
  }
  b->slot[s] = f;
  f->in_batch = true;
  forget_tiles(b);
  if (slot_out) *slot_out = s;
  return PF_OK;
}

static pf_status batch_remove(pf_batch* b, pf_filter* f) {
  if (b->in_flight) return bfail(b, PF_ERR_STATE, "an epoch is in flight");
  for (int i = 0; i < b->cap; ++i)
    if (b->slot[i] == f) {
      b->slot[i] = nullptr;
      f->in_batch = false;
      forget_tiles(b);
      return PF_OK;
    }
  return bfail(b, PF_ERR_INVALID_ARG, "filter is not in this batch");
}

static void CUDART_CB mark_done(void* p) { *static_cast<double*>(p) = now_ms(); }

// Launch one epoch for the slots with y[slot] != NULL (no waiting).  status[s]
// gets PF_ERR_INVALID_ARG for a rejected observation.
static pf_status batch_launch(pf_batch* b, const double* t, const double* const* y, int* status) {
  for (int i = 0; i < b->cap; ++i)
    if (b->slot[i]) b->slot[i]->est_fresh = false;  // batched epochs change the estimates
  if (b->in_flight) return bfail(b, PF_ERR_STATE, "an epoch is already in flight");
  const int cap = b->cap;
  std::vector<char> active(cap, 0);
  b->fl_slots.clear();
  b->fl_depth.assign(cap, 0);
  b->fl_t.assign(cap, 0.0);
  int S_max = 0;
  // each member's parameter block (slots are independent: own block, own
  // depth), in parallel when many members have an observation
  b->fl_S.assign(cap, -2);
  const std::function<void(int, int)> fill = [&](int lo, int hi) {
    for (int s = lo; s < hi; ++s) {
      const pf_filter* F = b->slot[s];
      if (!F || !y[s]) continue;
      bool ok = std::isfinite(t[s]) && t[s] > F->hist.t_prev;
      for (int i = 0; ok && i < F->m; ++i) ok = std::isfinite(y[s][i]);
      b->fl_S[s] = ok ? fill_epoch(F, F->hist, t[s], y[s], b->params_host + s, &b->fl_depth[s]) : -1;
    }
  };
  int n_obs = 0;
  for (int s = 0; s < cap; ++s) n_obs += (b->slot[s] && y[s]) ? 1 : 0;
  if (n_obs >= kParallelFill && !b->fill_pool && std::thread::hardware_concurrency() > kFillWorkers) {
    try {
      b->fill_pool.reset(new FillPool(kFillWorkers));
    } catch (...) {
      b->fill_pool.reset();  // no threads to be had: the blocks are built serially
    }
  }
  if (n_obs >= kParallelFill && b->fill_pool) b->fill_pool->run(cap, fill);
  else fill(0, cap);
  for (int s = 0; s < cap; ++s) {
    if (status) status[s] = PF_OK;
    const int S = b->fl_S[s];
    if (S == -2) continue;
    if (S < 1) {
      if (status) status[s] = PF_ERR_INVALID_ARG;
      continue;
    }
    active[s] = 1;
    b->fl_slots.push_back(s);
    b->fl_t[s] = t[s];
    S_max = std::max(S_max, S);
  }
  if (b->fl_slots.empty()) return PF_OK;
  const int n_act = (int)b->fl_slots.size();
  // 1. every slot's header and step table in one strided copy
  const size_t width = kEpochHeaderBytes + sizeof(StepCoef) * (size_t)S_max;
  PF_BCUDA(b, cudaMemcpy2DAsync(b->params_dev, sizeof(EpochParams), b->params_host,
                                sizeof(EpochParams), width, (size_t)cap, cudaMemcpyHostToDevice,
                                b->stream));
  std::memcpy(b->slots_pin, b->fl_slots.data(), sizeof(int) * n_act);
  PF_BCUDA(b, cudaMemcpyAsync(b->slots_dev, b->slots_pin, sizeof(int) * n_act,
                              cudaMemcpyHostToDevice, b->stream));
  // 2-3. tiles, then the graph (active set seen before) or direct launches
  const size_t smem = sizeof(StepCoef) * (size_t)S_max;
  if (b->autotune && !b->tuned) PF_BCUDA(b, run_autotune(b, active, smem));
  const bool same = b->tiles_active == active && b->tiles_smem == smem;
  if (!same) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    build_tiles(b, active, b->shape.order);
    PF_BCUDA(b, upload_tiles(b));
    b->tiles_active = active;
    b->tiles_smem = smem;
  } else if (!b->graph) {
    cudaError_t ce = capture(b, smem, b->shape, true, &b->graph);
    if (ce != cudaSuccess) {
      b->graph = nullptr;
      return bfail(b, PF_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(ce));
    }
    ++b->captures;
  }
  PF_BCUDA(b, cudaEventRecord(b->ev0, b->stream));
  if (b->graph) {
    PF_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  } else {
    PF_BCUDA(b, launch_phases(b, smem, b->shape, true));
  }
  PF_BCUDA(b, cudaEventRecord(b->ev1, b->stream));
  b->fl_done_ms = 0.0;
  PF_BCUDA(b, cudaLaunchHostFunc(b->stream, mark_done, &b->fl_done_ms));
  // 4. statuses of the active slots in one read-back
  k_batch_status<<<(n_act + 127) / 128, 128, 0, b->stream>>>(b->fds_dev, b->slots_dev, n_act,
                                                             b->status_dev);
  PF_BCUDA(b, cudaGetLastError());
  PF_BCUDA(b, cudaMemcpyAsync(b->status_host, b->status_dev, sizeof(int64_t) * 2 * n_act,
                              cudaMemcpyDeviceToHost, b->stream));
  PF_BCUDA(b, cudaEventRecord(b->ev_done, b->stream));
  b->in_flight = true;
  b->last_active = n_act;
  b->last_tiles = (int)b->tiles_host.size();
  return PF_OK;
}

// True when no epoch is in flight or the one in flight has finished (an error
// also counts: batch_collect reports it).
static bool batch_ready(const pf_batch* b) {
  if (!b->in_flight) return true;
  const cudaError_t e = cudaEventQuery(b->ev_done);
  return e != cudaErrorNotReady;
}

// Wait for the epoch in flight and commit the filters that succeeded.
static pf_status batch_collect(pf_batch* b, int* status) {
  if (!b->in_flight) return PF_OK;
  b->in_flight = false;
  // the epoch's own completion (work queued after it, e.g. a new member's
  // initialisation, is not waited for)
  PF_BCUDA(b, cudaEventSynchronize(b->ev_done));
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess) b->last_ms = ms;
  ++b->epochs;
  std::vector<int> failed;
  for (size_t i = 0; i < b->fl_slots.size(); ++i) {
    const int s = b->fl_slots[i];
    pf_filter* F = b->slot[s];
    const int st = (int)b->status_host[2 * i];
    if (st == PF_OK) {
      F->hist = advance_history(F->hist, b->fl_t[s], b->params_host + s, b->fl_depth[s]);
      F->h2d_bytes += (int64_t)(kEpochHeaderBytes + sizeof(StepCoef) * b->params_host[s].S);
    } else {
      if (status) status[s] = st;
      failed.push_back(s);
    }
  }
  if (!failed.empty()) {
    // failed filters keep their committed state; clear their sticky status
    PF_BCUDA(b, cudaMemcpyAsync(b->clear_dev, failed.data(), sizeof(int) * failed.size(),
                                cudaMemcpyHostToDevice, b->stream));
    k_batch_clear<<<((int)failed.size() + 127) / 128, 128, 0, b->stream>>>(b->fds_dev, b->clear_dev,
                                                                          (int)failed.size());
    PF_BCUDA(b, cudaGetLastError());
    PF_BCUDA(b, cudaStreamSynchronize(b->stream));
  }
  return PF_OK;
}

// ============================================================== the server
namespace {

constexpr int kDefaultLanes = 2 * kCostModels;
constexpr int64_t kLargeSession = 32768;  // particles; larger sessions get their own lanes

struct Pending {
  double t;
  std::vector<double> y;
  double arrive_ms;
};

struct Session {
  int64_t id;
  pf_filter* f = nullptr;  // NULL while waiting for admission
  int lane = 0, slot = -1;
  // creation arguments, kept until admission
  pf_ode ode;
  int d, p;
  int64_t N;
  pf_lmm lmm;
  double dt;
  std::vector<int> prior_kind, obs;
  std::vector<double> prior_lo, prior_hi, x0, sigma;
  double t0;
  pf_options opt;
  size_t bytes = 0;
  std::deque<Pending> queue;
  bool closing = false;
  int64_t done = 0;
  int last_status = PF_OK;
  double in_flight_arrive = -1.0;  // arrival time of the observation in flight
};

}  // namespace

struct pf_server {
  std::vector<pf_batch*> lanes;  // one stream and one epoch in flight each
  cudaMemPool_t pool = nullptr;  // the sessions' device memory
  cudaStream_t init_stream = nullptr;  // greatest priority; every session initialises on it
  int64_t reserved = 0;          // bytes of the budget mapped in the pool at creation
  int64_t budget = 0, in_use = 0;
  int64_t next_id = 1;
  std::map<int64_t, Session> sessions;
  std::deque<int64_t> waiting;   // admission order
  std::vector<double> latencies;
  int64_t admitted = 0, rejected = 0, epochs = 0, batched_sessions = 0;
  double steps_done = 0.0, first_ms = -1.0, last_ms = -1.0;
  int64_t step_calls = 0;
  double step_ms_total = 0.0, step_ms_max = 0.0;  // host time inside pf_server_step
  double collect_ms_max = 0.0, admit_ms_max = 0.0, launch_ms_max = 0.0;
  std::string err;
};

static pf_status sfail(pf_server* s, pf_status st, const std::string& msg) {
  if (s) s->err = msg;
  else set_thread_error(msg);
  return st;
}

// Sessions of one cost class (linear2; Robertson and M1; Brusselator) and
// size class share a lane, so a long epoch of large or expensive filters does
// not hold back the small ones.  A lane's batch mixes any problems and LMMs.
static int session_class(pf_ode ode, int64_t N) {
  return cost_model(ode) * 2 + (N > kLargeSession ? 1 : 0);
}
static int lane_of(const pf_server* s, pf_ode ode, int64_t N) {
  return session_class(ode, N) % (int)s->lanes.size();
}
// Cost rank of a class's epochs (0 = cheapest): small linear2, Robertson and M1,
// large ones, small Brusselator, large Brusselator.  Lanes of cheaper classes
// run on higher-priority streams, so their short epochs are scheduled ahead of
// the pending blocks of long ones (shortest job first).
static int class_rank(int cls) {
  static const int rank[2 * kCostModels] = {0, 1, 0, 1, 2, 3};
  return rank[cls];
}

static pf_status admit(pf_server* s, Session& ss) {
  pf_prior pr{ss.p, ss.prior_kind.data(), ss.prior_lo.data(), ss.prior_hi.data(), ss.d,
              ss.x0.data(), ss.t0};
  pf_options o = ss.opt;
  o.obs_idx = ss.obs.data();
  o.sigma = ss.sigma.data();
  // the server's own init stream: creating a stream per session had held an
  // admission for tens of milliseconds
  o.stream = s->init_stream;
  o.timing = 0;
  pf_filter* f = nullptr;
  pf_status st = filter_create(ss.ode, ss.d, ss.p, ss.N, ss.lmm, ss.dt, &pr, &o, s->pool, &f);
  if (st != PF_OK) return sfail(s, st, std::string("session creation failed: ") + pf_last_error(nullptr));
  pf_batch* lane = s->lanes[ss.lane];
  st = batch_add(lane, f, &ss.slot);
  if (st != PF_OK) {
    pf_destroy(f);
    return sfail(s, st, lane->err);
  }
  ss.f = f;
  s->in_use += (int64_t)ss.bytes;
  ++s->admitted;
  return PF_OK;
}

static void release(pf_server* s, Session& ss) {
  if (ss.f) {
    batch_remove(s->lanes[ss.lane], ss.f);
    pf_destroy(ss.f);
    ss.f = nullptr;
    s->in_use -= (int64_t)ss.bytes;
  }
}

// Collect a lane's finished epoch: latencies, per-session results, closings.
static pf_status collect_lane(pf_server* s, int li) {
  pf_batch* b = s->lanes[li];
  if (!b->in_flight) return PF_OK;
  std::vector<int> status(b->cap, PF_OK);
  pf_status st = batch_collect(b, status.data());
  if (st != PF_OK) return sfail(s, st, b->err);
  const double done = b->fl_done_ms > 0.0 ? b->fl_done_ms : now_ms();
  for (auto it = s->sessions.begin(); it != s->sessions.end();) {
    Session& ss = it->second;
    if (ss.lane != li || !ss.f) {
      ++it;
      continue;
    }
    if (ss.in_flight_arrive >= 0.0) {
      ss.last_status = status[ss.slot];
      s->latencies.push_back(done - ss.in_flight_arrive);
      if (ss.last_status == PF_OK) {
        ++ss.done;
        s->steps_done += 2.0 * (double)b->params_host[ss.slot].S * (double)ss.N;
      }
      ss.in_flight_arrive = -1.0;
    }
    // a closed session leaves once its queue is done, and frees its memory
    if (ss.closing && ss.queue.empty()) {
      release(s, ss);
      it = s->sessions.erase(it);
    } else {
      ++it;
    }
  }
  s->last_ms = std::max(s->last_ms, done);
  return PF_OK;
}

static bool server_pending(const pf_server* s) {
  for (const pf_batch* b : s->lanes)
    if (b->in_flight) return true;
  for (const auto& kv : s->sessions)
    if (kv.second.f && !kv.second.queue.empty()) return true;
  return false;
}

extern "C" {

pf_status pf_batch_create(pf_filter* const* filters, int n, void* stream, pf_batch** out) {
  if (!out) return bfail(nullptr, PF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!filters || n < 1) return bfail(nullptr, PF_ERR_INVALID_ARG, "need n >= 1 filters");
  for (int i = 0; i < n; ++i) {
    if (!filters[i]) return bfail(nullptr, PF_ERR_INVALID_ARG, "NULL filter");
    if (filters[i]->in_batch) return bfail(nullptr, PF_ERR_INVALID_ARG, "filter already in a batch");
    if (filters[i]->shard_total > 0) return bfail(nullptr, PF_ERR_INVALID_ARG, "a shard cannot join a batch");
    for (int j = 0; j < i; ++j)
      if (filters[j] == filters[i]) return bfail(nullptr, PF_ERR_INVALID_ARG, "filter listed twice");
  }
  pf_batch* b = nullptr;
  pf_status st = batch_new(stream, n, true, 0, &b);
  if (st != PF_OK) return st;
  for (int i = 0; i < n; ++i) {
    int slot = -1;
    st = batch_add(b, filters[i], &slot);
    if (st != PF_OK) {
      set_thread_error(b->err);
      pf_batch_destroy(b);
      return st;
    }
  }
  *out = b;
  return PF_OK;
}

void pf_batch_destroy(pf_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (pf_filter* f : b->slot)
    if (f) f->in_batch = false;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->fds_dev);
  cudaFree(b->eps_dev);
  cudaFree(b->params_dev);
  cudaFree(b->tiles_dev);
  cudaFree(b->slots_dev);
  cudaFree(b->status_dev);
  cudaFree(b->clear_dev);
  if (b->params_host) cudaFreeHost(b->params_host);
  if (b->status_host) cudaFreeHost(b->status_host);
  if (b->slots_pin) cudaFreeHost(b->slots_pin);
  if (b->tiles_pin) cudaFreeHost(b->tiles_pin);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* pf_batch_last_error(const pf_batch* b) { return b ? b->err.c_str() : ""; }

pf_status pf_batch_assimilate(pf_batch* b, const double* t, const double* const* y, int* status) {
  const pfg::NvtxRange nvtx_range("pf_batch_assimilate");
  if (!b) return bfail(nullptr, PF_ERR_INVALID_ARG, "batch is NULL");
  if (!t || !y || !status) return bfail(b, PF_ERR_INVALID_ARG, "NULL argument");
  pf_status st = batch_launch(b, t, y, status);
  if (st != PF_OK) return st;
  return batch_collect(b, status);
}

pf_status pf_batch_stats(const pf_batch* b, pf_batch_stats_t* out) {
  if (!b || !out) return bfail(const_cast<pf_batch*>(b), PF_ERR_INVALID_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->epochs = b->epochs;
  out->graph_captures = b->captures;
  out->last_device_ms = b->last_ms;
  out->last_active = b->last_active;
  out->last_tiles = b->last_tiles;
  out->tile_order = b->shape.order;
  out->concurrent_models = b->shape.concurrent;
  for (int i = 0; i < 4; ++i) out->tune_ms[i] = b->tune_ms[i];
  return PF_OK;
}

// Reserve the budget in the pool once, at creation: allocating it and freeing
// it maps its pages now, and the release threshold keeps them, so admissions
// only sub-allocate mapped memory.  Growing the pool during admission instead
// held a pf_server_step for tens of milliseconds (the driver mapping the
// pages of a large session).  A budget beyond the free device memory is not
// reserved; the pool then grows as sessions arrive.
static void reserve_budget(pf_server* s) {
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  if ((double)s->budget > 0.9 * (double)free_b) return;
  cudaStream_t rs = nullptr;
  if (cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  void* p = nullptr;
  if (cudaMallocFromPoolAsync(&p, (size_t)s->budget, s->pool, rs) == cudaSuccess) {
    cudaFreeAsync(p, rs);
    s->reserved = s->budget;
  }
  cudaGetLastError();  // a reservation that did not fit is not an error
  cudaStreamSynchronize(rs);
  cudaStreamDestroy(rs);
}

pf_status pf_server_create(int64_t budget_bytes, int lanes, pf_server** out) {
  if (!out) return sfail(nullptr, PF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (budget_bytes <= 0) return sfail(nullptr, PF_ERR_INVALID_ARG, "budget must be positive");
  if (lanes < 0 || lanes > 64) return sfail(nullptr, PF_ERR_INVALID_ARG, "need 0 <= lanes <= 64");
  if (lanes == 0) lanes = kDefaultLanes;
  pf_server* s = new (std::nothrow) pf_server();
  if (!s) return sfail(nullptr, PF_ERR_OOM, "host allocation failed");
  s->budget = budget_bytes;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) {
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    e = cudaMemPoolCreate(&s->pool, &props);
  }
  if (e == cudaSuccess) {
    // freed session memory stays in the pool for the next admission
    uint64_t keep = (uint64_t)budget_bytes;
    e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e != cudaSuccess) {
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
    return sfail(nullptr, PF_ERR_CUDA, std::string("memory pool creation failed: ") +
                                           cudaGetErrorString(e));
  }
  reserve_budget(s);
  int least = 0, greatest = 0;
  cudaDeviceGetStreamPriorityRange(&least, &greatest);
  e = cudaStreamCreateWithPriority(&s->init_stream, cudaStreamNonBlocking, greatest);
  if (e != cudaSuccess) {
    s->init_stream = nullptr;
    pf_server_destroy(s);
    return sfail(nullptr, PF_ERR_CUDA, std::string("init stream creation failed: ") +
                                           cudaGetErrorString(e));
  }
  for (int i = 0; i < lanes; ++i) {
    int rank = 3;
    for (int cls = 0; cls < 2 * kCostModels; ++cls)
      if (cls % lanes == i) rank = std::min(rank, class_rank(cls));
    const int prio = lanes == 1 ? least : std::min(least, greatest + rank);
    pf_batch* b = nullptr;
    pf_status st = batch_new(nullptr, 64, false, prio, &b);
    if (st != PF_OK) {
      pf_server_destroy(s);
      return st;
    }
    s->lanes.push_back(b);
  }
  *out = s;
  return PF_OK;
}

void pf_server_destroy(pf_server* s) {
  if (!s) return;
  for (pf_batch* b : s->lanes) {
    cudaStreamSynchronize(b->stream);
    b->in_flight = false;
  }
  for (auto& kv : s->sessions) release(s, kv.second);
  for (pf_batch* b : s->lanes) pf_batch_destroy(b);
  if (s->pool) {
    cudaDeviceSynchronize();  // the stream-ordered frees of the sessions
    cudaMemPoolDestroy(s->pool);
  }
  if (s->init_stream) cudaStreamDestroy(s->init_stream);
  delete s;
}

const char* pf_server_last_error(const pf_server* s) { return s ? s->err.c_str() : ""; }

pf_status pf_server_open(pf_server* s, pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                         const pf_prior* prior, const pf_options* opt, int64_t* session) {
  if (!s || !prior || !opt || !session) return sfail(s, PF_ERR_INVALID_ARG, "NULL argument");
  {
    const pf_status cs = check_create_args(ode, d, p, N, lmm, dt, prior, opt);
    if (cs != PF_OK) return sfail(s, cs, pf_last_error(nullptr));
  }
  if (ode == PF_ODE_ADVDIFF2D)
    return sfail(s, PF_ERR_INVALID_ARG, "2D advection-diffusion sessions are not served (no batched kernels)");
  Session ss;
  ss.id = s->next_id++;
  ss.ode = ode; ss.d = d; ss.p = p; ss.N = N; ss.lmm = lmm; ss.dt = dt;
  ss.prior_kind.assign(prior->kind, prior->kind + p);
  ss.prior_lo.assign(prior->lo, prior->lo + p);
  ss.prior_hi.assign(prior->hi, prior->hi + p);
  ss.x0.assign(prior->x0, prior->x0 + d);
  ss.t0 = prior->t0;
  ss.opt = *opt;
  ss.obs.assign(opt->obs_idx, opt->obs_idx + opt->m);
  ss.sigma.assign(opt->sigma, opt->sigma + opt->m);
  ss.bytes = filter_device_bytes(ode, d, p, N);
  ss.lane = lane_of(s, ode, N);
  if ((int64_t)ss.bytes > s->budget) {
    ++s->rejected;
    return sfail(s, PF_ERR_BUDGET, "the session alone exceeds the memory budget");
  }
  const int64_t id = ss.id;
  s->sessions.emplace(id, std::move(ss));
  s->waiting.push_back(id);
  *session = id;
  return PF_OK;
}

pf_status pf_server_submit(pf_server* s, int64_t session, double t_k, const double* y_k) {
  if (!s || !y_k) return sfail(s, PF_ERR_INVALID_ARG, "NULL argument");
  auto it = s->sessions.find(session);
  if (it == s->sessions.end() || it->second.closing)
    return sfail(s, PF_ERR_INVALID_ARG, "unknown or closing session");
  Session& ss = it->second;
  Pending pd{t_k, std::vector<double>(y_k, y_k + ss.opt.m), now_ms()};
  if (s->first_ms < 0.0) s->first_ms = pd.arrive_ms;
  ss.queue.push_back(std::move(pd));
  return PF_OK;
}

static pf_status server_step(pf_server* s, int* launched, int* consumed);

pf_status pf_server_step(pf_server* s, int* launched) {
  const pfg::NvtxRange nvtx_range("pf_server_step");
  if (!s) return sfail(nullptr, PF_ERR_INVALID_ARG, "server is NULL");
  const double t0 = now_ms();
  const pf_status st = server_step(s, launched, nullptr);
  const double dt = now_ms() - t0;
  ++s->step_calls;
  s->step_ms_total += dt;
  s->step_ms_max = std::max(s->step_ms_max, dt);
  return st;
}

// consumed (if set): observations taken off the queues, launched or rejected
static pf_status server_step(pf_server* s, int* launched, int* consumed) {
  if (launched) *launched = 0;
  if (consumed) *consumed = 0;
  int taken = 0;
  const int L = (int)s->lanes.size();
  // 1. collect the lanes whose epoch has finished (no waiting)
  for (int li = 0; li < L; ++li)
    if (s->lanes[li]->in_flight && batch_ready(s->lanes[li])) {
      const double t0 = now_ms();
      pf_status st = collect_lane(s, li);
      s->collect_ms_max = std::max(s->collect_ms_max, now_ms() - t0);
      if (st != PF_OK) return st;
    }
  // 2. admit waiting sessions in arrival order while they fit the budget (into
  //    their lane even while it has an epoch in flight); one whose lane is
  //    full and busy keeps its place for a later step
  for (auto w = s->waiting.begin(); w != s->waiting.end();) {
    auto it = s->sessions.find(*w);
    if (it == s->sessions.end()) {
      w = s->waiting.erase(w);
      continue;
    }
    Session& ss = it->second;
    if (s->in_use + (int64_t)ss.bytes > s->budget) break;
    const double t0 = now_ms();
    const pf_status ast = admit(s, ss);
    s->admit_ms_max = std::max(s->admit_ms_max, now_ms() - t0);
    if (ast == PF_ERR_STATE) {  // its lane is full and busy: keeps its place
      ++w;
      continue;
    }
    if (ast != PF_OK) {  // e.g. the device itself is out of memory: the session
      ss.last_status = ast;  // stays queryable, takes no observations, holds nothing
      ss.closing = true;
      ss.queue.clear();
      ++s->rejected;
    }
    w = s->waiting.erase(w);
  }
  // 3. on every idle lane, one batched epoch over its sessions that have a
  //    queued observation (the oldest one of each)
  int total = 0;
  for (int li = 0; li < L; ++li) {
    pf_batch* b = s->lanes[li];
    if (b->in_flight) continue;
    std::vector<double> t(b->cap, 0.0);
    std::vector<const double*> y(b->cap, nullptr);
    std::vector<Session*> in;
    for (auto& kv : s->sessions) {
      Session& ss = kv.second;
      if (ss.lane != li || !ss.f || ss.queue.empty()) continue;
      t[ss.slot] = ss.queue.front().t;
      y[ss.slot] = ss.queue.front().y.data();
      in.push_back(&ss);
    }
    if (in.empty()) continue;
    std::vector<int> status(b->cap, PF_OK);
    const double t0 = now_ms();
    pf_status st = batch_launch(b, t.data(), y.data(), status.data());
    s->launch_ms_max = std::max(s->launch_ms_max, now_ms() - t0);
    if (st != PF_OK) return sfail(s, st, b->err);
    int n = 0;
    for (Session* ss : in) {
      if (status[ss->slot] != PF_OK) {
        ss->last_status = status[ss->slot];  // rejected observation: dropped
      } else {
        ss->in_flight_arrive = ss->queue.front().arrive_ms;
        ++n;
      }
      ss->queue.pop_front();
      ++taken;
    }
    if (n > 0) {
      ++s->epochs;
      s->batched_sessions += n;
    }
    total += n;
  }
  if (launched) *launched = total;
  if (consumed) *consumed = taken;
  return PF_OK;
}

pf_status pf_server_drain(pf_server* s) {
  if (!s) return sfail(nullptr, PF_ERR_INVALID_ARG, "server is NULL");
  for (;;) {
    int launched = 0, consumed = 0;
    const double t0 = now_ms();
    pf_status st = server_step(s, &launched, &consumed);
    const double dt = now_ms() - t0;
    ++s->step_calls;
    s->step_ms_total += dt;
    s->step_ms_max = std::max(s->step_ms_max, dt);
    if (st != PF_OK) return st;
    // sessions still waiting for admission cannot make progress here
    if (!server_pending(s)) return PF_OK;
    // rejected observations leave their queues without an epoch: step again
    if (launched == 0 && consumed == 0) {
      // wait until some lane's epoch finishes; with nothing in flight no wait
      // can end (observations are queued that no step launches), so report
      // that instead of spinning
      bool flying = false;
      for (const pf_batch* b : s->lanes) flying = flying || b->in_flight;
      if (!flying)
        return sfail(s, PF_ERR_STATE, "drain: observations are queued but no epoch can launch");
      bool any = false;
      while (!any) {
        for (pf_batch* b : s->lanes)
          if (b->in_flight && batch_ready(b)) any = true;
        if (!any) std::this_thread::yield();
      }
    }
  }
}

pf_status pf_server_close(pf_server* s, int64_t session) {
  if (!s) return sfail(nullptr, PF_ERR_INVALID_ARG, "server is NULL");
  auto it = s->sessions.find(session);
  if (it == s->sessions.end()) return sfail(s, PF_ERR_INVALID_ARG, "unknown session");
  Session& ss = it->second;
  ss.closing = true;
  const bool is_waiting =
      std::find(s->waiting.begin(), s->waiting.end(), session) != s->waiting.end();
  if (!ss.f && (ss.queue.empty() || !is_waiting)) {  // nothing to do: drop it
    s->waiting.erase(std::remove(s->waiting.begin(), s->waiting.end(), session), s->waiting.end());
    s->sessions.erase(it);
    return PF_OK;
  }
  if (ss.queue.empty() && !s->lanes[ss.lane]->in_flight) {
    release(s, ss);
    s->sessions.erase(it);
  }
  return PF_OK;
}

pf_status pf_server_session(const pf_server* s, int64_t session, pf_filter** filter,
                            int64_t* assimilated, int* last_status) {
  if (!s) return sfail(nullptr, PF_ERR_INVALID_ARG, "server is NULL");
  auto it = s->sessions.find(session);
  if (it == s->sessions.end()) return sfail(const_cast<pf_server*>(s), PF_ERR_INVALID_ARG, "unknown session");
  if (filter) *filter = it->second.f;
  if (assimilated) *assimilated = it->second.done;
  if (last_status) *last_status = it->second.last_status;
  return PF_OK;
}

pf_status pf_server_stats(const pf_server* s, pf_server_stats_t* out) {
  if (!s || !out) return sfail(const_cast<pf_server*>(s), PF_ERR_INVALID_ARG, "NULL argument");
  std::memset(out, 0, sizeof(*out));
  out->admitted = s->admitted;
  out->rejected = s->rejected;
  out->waiting = (int64_t)s->waiting.size();
  int64_t active = 0, queued = 0;
  for (const auto& kv : s->sessions) {
    if (kv.second.f) ++active;
    queued += (int64_t)kv.second.queue.size();
  }
  out->active_sessions = active;
  out->queued_observations = queued;
  out->assimilations = (int64_t)s->latencies.size();
  out->epochs = s->epochs;
  out->mean_sessions_per_epoch = s->epochs ? (double)s->batched_sessions / (double)s->epochs : 0.0;
  out->device_bytes_in_use = s->in_use;
  out->budget_bytes = s->budget;
  out->step_calls = s->step_calls;
  out->step_ms_mean = s->step_calls ? s->step_ms_total / (double)s->step_calls : 0.0;
  out->step_ms_max = s->step_ms_max;
  out->collect_ms_max = s->collect_ms_max;
  out->admit_ms_max = s->admit_ms_max;
  out->launch_ms_max = s->launch_ms_max;
  if (!s->latencies.empty()) {
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
      const size_t k = (size_t)std::min<double>((double)(v.size() - 1), std::ceil(q * v.size()) - 1.0);
      return v[k];
    };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.back();
    double sum = 0.0;
    for (double x : v) sum += x;
    out->mean_ms = sum / (double)v.size();
  }
  if (s->first_ms >= 0.0 && s->last_ms > s->first_ms)
    out->particle_steps_per_s = s->steps_done / ((s->last_ms - s->first_ms) * 1e-3);
  return PF_OK;
}

}  // extern "C"
