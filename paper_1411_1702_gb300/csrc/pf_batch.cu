// pf_batch.cu -- many filters advanced together: one epoch of every filter
// with a new observation runs as a handful of tile-scheduled launches (one per
// phase, split by model where the kernels differ), captured in a CUDA graph.
//
// The batch drives the filters' own device buffers.  Per epoch the host
//  1. builds each active filter's parameter block (substep table, y, 1/sigma)
//     into a pinned slot and uploads every slot with one strided copy;
//  2. rebuilds the tile tables (filter, virtual block) when the set of active
//     filters changes, ordering each phase's tiles largest filter first;
//  3. launches the captured graph of the phases (recaptured only when the
//     active set or the step-table size changes);  on its first epoch the
//     batch autotunes the launch shape -- the tile order within a phase and
//     whether the per-model launches of a phase run back to back or as
//     concurrent graph branches -- by timing each candidate on the real
//     epoch's phases up to stage 2 (none of which touches the committed
//     state), then keeps the fastest;
//  4. gathers every filter's status and epoch count with one kernel and one
//     read-back, and commits the host-side history of the filters that
//     succeeded.
// A filter's results are bit-identical alone and in a batch (its reductions
// depend only on its own N; see pf_kernels.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "pf_filter.h"

using namespace pfg;

namespace pfg {

__global__ void k_batch_status(const FilterDev* __restrict__ fds, int n, int64_t* out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < n) {
    const Ctrl* c = fds[f].ctrl;
    out[2 * f] = c->status;
    out[2 * f + 1] = c->epochs_done;
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

constexpr int kModels = 3;  // linear2, robertson, brusselator
int model_index(int ode) { return ode - 1; }

struct Range {
  int off = 0, cnt = 0;
};

// launch shape chosen by the autotuner
struct Shape {
  int order;       // 0: larger filters first; 1: filters interleaved block by block
  int concurrent;  // per-model launches of a phase as parallel graph branches
};
const Shape kShapes[] = {{0, 0}, {0, 1}, {1, 0}, {1, 1}};

}  // namespace

struct pf_batch {
  int n = 0;
  std::vector<pf_filter*> filters;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;          // second branch of the captured graph
  cudaEvent_t fork = nullptr, join = nullptr;
  Shape shape{0, 0};
  bool tuned = false;
  double tune_ms[4] = {0, 0, 0, 0};
  FilterDev* fds_dev = nullptr;
  EpochParams** eps_dev = nullptr;
  EpochParams* params_dev = nullptr;
  EpochParams* params_host = nullptr;  // pinned
  BatchTile* tiles_dev = nullptr;
  int tiles_cap = 0;
  std::vector<BatchTile> tiles_host;
  Range stage[2][kModels];
  Range moments[kModels];
  Range scan_tile, scan_add, resample;
  int64_t* status_dev = nullptr;
  int64_t* status_host = nullptr;  // pinned
  int* clear_dev = nullptr;
  // graph of the last active set
  cudaGraphExec_t graph = nullptr;
  std::vector<char> graph_active;
  size_t graph_smem = 0;
  int64_t captures = 0, epochs = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double last_ms = 0.0;
  int last_active = 0, last_tiles = 0;
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
  for (int f = 0; f < b->n; ++f)
    if (active[f]) order.push_back(f);
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->filters[x]->N > b->filters[y]->N; });
  b->tiles_host.clear();
  auto add = [&](int phase, int model) {
    Range r;
    r.off = (int)b->tiles_host.size();
    if (order_kind == 0) {
      for (int f : order) {
        const pf_filter* F = b->filters[f];
        if (model >= 0 && model_index(F->ode) != model) continue;
        const int nb = phase_blocks(phase, F->ode, F->N);
        for (int v = 0; v < nb; ++v) b->tiles_host.push_back(BatchTile{f, v});
      }
    } else {
      int most = 0;
      for (int f : order) most = std::max(most, phase_blocks(phase, b->filters[f]->ode, b->filters[f]->N));
      for (int v = 0; v < most; ++v)
        for (int f : order) {
          const pf_filter* F = b->filters[f];
          if (model >= 0 && model_index(F->ode) != model) continue;
          if (v < phase_blocks(phase, F->ode, F->N)) b->tiles_host.push_back(BatchTile{f, v});
        }
    }
    r.cnt = (int)b->tiles_host.size() - r.off;
    return r;
  };
  for (int m = 0; m < kModels; ++m) b->stage[0][m] = add(kPhaseStage1, m);
  b->scan_tile = add(kPhaseScanTile, -1);
  b->scan_add = add(kPhaseScanAdd, -1);
  b->resample = add(kPhaseResample, -1);
  for (int m = 0; m < kModels; ++m) b->stage[1][m] = add(kPhaseStage2, m);
  for (int m = 0; m < kModels; ++m) b->moments[m] = add(kPhaseMoments, m);
}

// Enqueue the phases on b->stream (inside a capture).  With a concurrent
// shape, each per-model group of a phase forks onto two branches (the model
// with the most tiles on the main branch) and joins before the next phase.
static cudaError_t launch_phases(pf_batch* b, size_t smem, const Shape& shape, bool with_moments) {
  const FilterDev* fds = b->fds_dev;
  const EpochParams* const* eps = b->eps_dev;
  const BatchTile* T = b->tiles_dev;
  cudaError_t e = cudaSuccess;
  auto run = [&](int phase, int ode, const Range& r, cudaStream_t st) {
    if (e == cudaSuccess && r.cnt > 0)
      e = launch_batch_phase(phase, ode, fds, eps, T + r.off, r.cnt, smem, 0, st);
  };
  auto per_model = [&](int phase, const Range* rs) {
    int used = 0, big = -1;
    for (int m = 0; m < kModels; ++m)
      if (rs[m].cnt > 0) {
        ++used;
        if (big < 0 || rs[m].cnt > rs[big].cnt) big = m;
      }
    if (!shape.concurrent || used < 2) {
      for (int m = 0; m < kModels; ++m) run(phase, m + 1, rs[m], b->stream);
      return;
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->fork, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->fork, 0);
    run(phase, big + 1, rs[big], b->stream);
    for (int m = 0; m < kModels; ++m)
      if (m != big) run(phase, m + 1, rs[m], b->side);
    if (e == cudaSuccess) e = cudaEventRecord(b->join, b->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join, 0);
  };
  per_model(kPhaseStage1, b->stage[0]);
  run(kPhaseScanTile, 0, b->scan_tile, b->stream);
  run(kPhaseScanAdd, 0, b->scan_add, b->stream);
  run(kPhaseResample, 0, b->resample, b->stream);
  per_model(kPhaseStage2, b->stage[1]);
  if (with_moments) per_model(kPhaseMoments, b->moments);
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
static cudaError_t autotune(pf_batch* b, const std::vector<char>& active, size_t smem) {
  double best = 1e300;
  int best_i = 0;
  for (int i = 0; i < 4; ++i) {
    build_tiles(b, active, kShapes[i].order);
    cudaError_t e = cudaMemcpyAsync(b->tiles_dev, b->tiles_host.data(),
                                    sizeof(BatchTile) * b->tiles_host.size(),
                                    cudaMemcpyHostToDevice, b->stream);
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
  return cudaSuccess;
}

extern "C" {

pf_status pf_batch_create(pf_filter* const* filters, int n, void* stream, pf_batch** out) {
  if (!out) return bfail(nullptr, PF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!filters || n < 1) return bfail(nullptr, PF_ERR_INVALID_ARG, "need n >= 1 filters");
  for (int i = 0; i < n; ++i) {
    if (!filters[i]) return bfail(nullptr, PF_ERR_INVALID_ARG, "NULL filter");
    if (filters[i]->in_batch) return bfail(nullptr, PF_ERR_INVALID_ARG, "filter already in a batch");
    for (int j = 0; j < i; ++j)
      if (filters[j] == filters[i]) return bfail(nullptr, PF_ERR_INVALID_ARG, "filter listed twice");
  }
  pf_batch* b = new (std::nothrow) pf_batch();
  if (!b) return bfail(nullptr, PF_ERR_OOM, "host allocation failed");
  b->n = n;
  b->filters.assign(filters, filters + n);
  pf_status st = PF_OK;
  auto bail = [&](pf_status s) {
    set_thread_error(b->err);
    pf_batch_destroy(b);
    return s;
  };
  cudaError_t e;
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(bfail(b, PF_ERR_CUDA, "stream creation failed"));
    b->own_stream = true;
  }
  e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
  if (e != cudaSuccess) return bail(bfail(b, PF_ERR_CUDA, "stream/event creation failed"));
  // the filters' own streams must be idle before the batch drives them
  for (pf_filter* f : b->filters) {
    e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return bail(bfail(b, PF_ERR_CUDA, "filter stream synchronisation failed"));
  }
  int cap = 0;
  for (pf_filter* f : b->filters)
    for (int ph = 0; ph <= kPhaseMoments; ++ph) cap += phase_blocks(ph, f->ode, f->N);
  b->tiles_cap = cap;
  std::vector<FilterDev> fds(n);
  std::vector<EpochParams*> eps(n);
  e = cudaMalloc(&b->fds_dev, sizeof(FilterDev) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->eps_dev, sizeof(EpochParams*) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->params_dev, sizeof(EpochParams) * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->tiles_dev, sizeof(BatchTile) * (size_t)cap);
  if (e == cudaSuccess) e = cudaMalloc(&b->status_dev, sizeof(int64_t) * 2 * n);
  if (e == cudaSuccess) e = cudaMalloc(&b->clear_dev, sizeof(int) * n);
  if (e == cudaSuccess) e = cudaMallocHost(&b->params_host, sizeof(EpochParams) * n);
  if (e == cudaSuccess) e = cudaMallocHost(&b->status_host, sizeof(int64_t) * 2 * n);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e != cudaSuccess) return bail(bfail(b, PF_ERR_OOM, "batch allocation failed"));
  std::memset(b->params_host, 0, sizeof(EpochParams) * n);
  for (int i = 0; i < n; ++i) {
    fds[i] = b->filters[i]->fd;
    eps[i] = b->params_dev + i;
  }
  e = cudaMemcpyAsync(b->fds_dev, fds.data(), sizeof(FilterDev) * n, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->eps_dev, eps.data(), sizeof(EpochParams*) * n, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bail(bfail(b, PF_ERR_CUDA, "batch upload failed"));
  for (pf_filter* f : b->filters) f->in_batch = true;
  *out = b;
  return st;
}

void pf_batch_destroy(pf_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (pf_filter* f : b->filters)
    if (f) f->in_batch = false;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->fds_dev);
  cudaFree(b->eps_dev);
  cudaFree(b->params_dev);
  cudaFree(b->tiles_dev);
  cudaFree(b->status_dev);
  cudaFree(b->clear_dev);
  if (b->params_host) cudaFreeHost(b->params_host);
  if (b->status_host) cudaFreeHost(b->status_host);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

const char* pf_batch_last_error(const pf_batch* b) { return b ? b->err.c_str() : ""; }

pf_status pf_batch_assimilate(pf_batch* b, const double* t, const double* const* y, int* status) {
  if (!b) return bfail(nullptr, PF_ERR_INVALID_ARG, "batch is NULL");
  if (!t || !y || !status) return bfail(b, PF_ERR_INVALID_ARG, "NULL argument");
  const int n = b->n;
  std::vector<char> active(n, 0);
  std::vector<int> depth_out(n, 0);
  int S_max = 0, n_active = 0;
  for (int f = 0; f < n; ++f) {
    status[f] = PF_OK;
    if (!y[f]) continue;
    pf_filter* F = b->filters[f];
    bool ok = std::isfinite(t[f]) && t[f] > F->hist.t_prev;
    for (int i = 0; ok && i < F->m; ++i) ok = std::isfinite(y[f][i]);
    int S = ok ? fill_epoch(F, F->hist, t[f], y[f], b->params_host + f, &depth_out[f]) : -1;
    if (S < 1) {
      status[f] = PF_ERR_INVALID_ARG;
      continue;
    }
    active[f] = 1;
    ++n_active;
    S_max = std::max(S_max, S);
  }
  if (n_active == 0) return PF_OK;
  // 1. every slot's header and step table in one strided copy
  const size_t width = kEpochHeaderBytes + sizeof(StepCoef) * (size_t)S_max;
  PF_BCUDA(b, cudaMemcpy2DAsync(b->params_dev, sizeof(EpochParams), b->params_host,
                                sizeof(EpochParams), width, (size_t)n, cudaMemcpyHostToDevice,
                                b->stream));
  // 2-3. tiles and graph of this active set
  const size_t smem = sizeof(StepCoef) * (size_t)S_max;
  const bool same = b->graph && b->graph_active == active && b->graph_smem == smem;
  if (!same) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    if (!b->tuned) PF_BCUDA(b, autotune(b, active, smem));
    build_tiles(b, active, b->shape.order);
    PF_BCUDA(b, cudaMemcpyAsync(b->tiles_dev, b->tiles_host.data(),
                                sizeof(BatchTile) * b->tiles_host.size(), cudaMemcpyHostToDevice,
                                b->stream));
    cudaError_t ce = capture(b, smem, b->shape, true, &b->graph);
    if (ce != cudaSuccess) {
      b->graph = nullptr;
      return bfail(b, PF_ERR_CUDA, std::string("graph capture failed: ") + cudaGetErrorString(ce));
    }
    b->graph_active = active;
    b->graph_smem = smem;
    ++b->captures;
  }
  PF_BCUDA(b, cudaEventRecord(b->ev0, b->stream));
  PF_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
  PF_BCUDA(b, cudaEventRecord(b->ev1, b->stream));
  // 4. statuses of every filter in one read-back
  k_batch_status<<<(n + 127) / 128, 128, 0, b->stream>>>(b->fds_dev, n, b->status_dev);
  PF_BCUDA(b, cudaGetLastError());
  PF_BCUDA(b, cudaMemcpyAsync(b->status_host, b->status_dev, sizeof(int64_t) * 2 * n,
                              cudaMemcpyDeviceToHost, b->stream));
  PF_BCUDA(b, cudaStreamSynchronize(b->stream));
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess) b->last_ms = ms;
  b->last_active = n_active;
  b->last_tiles = (int)b->tiles_host.size();
  ++b->epochs;
  std::vector<int> failed;
  for (int f = 0; f < n; ++f) {
    if (!active[f]) continue;
    pf_filter* F = b->filters[f];
    const int s = (int)b->status_host[2 * f];
    if (s == PF_OK) {
      F->hist = advance_history(F->hist, t[f], b->params_host + f, depth_out[f]);
      F->h2d_bytes += (int64_t)(kEpochHeaderBytes + sizeof(StepCoef) * b->params_host[f].S);
    } else {
      status[f] = s;
      failed.push_back(f);
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

}  // extern "C"
