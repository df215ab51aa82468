// pf_capi.cu -- the C ABI of include/pf.h: argument checks, device memory,
// the host side of each epoch (substep table, parameter upload, launch,
// commit check) and the checkpoint/inspection calls.  All of the method's
// arithmetic on particles runs in the kernels of pf_kernels.cu.
#include <mutex>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "pf_filter.h"
#include "pf_scan.cuh"

using namespace pfg;

namespace {
thread_local std::string g_thread_error;
}  // namespace

namespace pfg {
void set_thread_error(const std::string& msg) { g_thread_error = msg; }
}  // namespace pfg

// A set of timing events for one epoch, or NULL when timing is off.
static cudaEvent_t* take_marks(pf_filter* f) {
  if (!f->timing) return nullptr;
  if (!f->mark_free.empty()) {
    cudaEvent_t* m = f->mark_free.back();
    f->mark_free.pop_back();
    f->mark_pending.push_back(m);
    return m;
  }
  // timing 2: only the events around stage 2 (slot kPhaseStage2, marks 4 and 5)
  cudaEvent_t* m = new cudaEvent_t[kEpochKernels + 1];
  for (int i = 0; i <= kEpochKernels; ++i) {
    m[i] = nullptr;
    if (f->timing == 2 && i != kPhaseStage2 && i != kPhaseStage2 + 1) continue;
    if (cudaEventCreate(&m[i]) != cudaSuccess) {
      for (int j = 0; j < i; ++j)
        if (m[j]) cudaEventDestroy(m[j]);
      delete[] m;
      return nullptr;
    }
  }
  f->mark_pending.push_back(m);
  return m;
}

static void free_marks(pf_filter* f) {
  for (auto* v : {&f->mark_free, &f->mark_pending}) {
    for (cudaEvent_t* m : *v) {
      for (int i = 0; i <= kEpochKernels; ++i)
        if (m[i]) cudaEventDestroy(m[i]);
      delete[] m;
    }
    v->clear();
  }
}

static pf_status fail(pf_filter* f, pf_status st, const std::string& msg) {
  if (f) f->err = msg;
  else g_thread_error = msg;
  return st;
}

static pf_status cuda_fail(pf_filter* f, cudaError_t e, const char* what) {
  std::string msg = std::string("CUDA error in ") + what + ": " + cudaGetErrorName(e) + " (" +
                    cudaGetErrorString(e) + ")";
  return fail(f, PF_ERR_CUDA, msg);
}

#define PF_CUDA(f, call)                                  \
  do {                                                    \
    cudaError_t e__ = (call);                             \
    if (e__ != cudaSuccess) return cuda_fail(f, e__, #call); \
  } while (0)

// Parameter count and fixed state dimension (0: a dimension the caller picks).
static bool ode_dims(int ode, int* d, int* p) {
  switch (ode) {
    case PF_ODE_LINEAR2: *d = 2; *p = 2; return true;
    case PF_ODE_ROBERTSON: *d = 3; *p = 3; return true;
    case PF_ODE_BRUSSELATOR1D: *d = 64; *p = 3; return true;
    case PF_ODE_ADVDIFF2D: *d = 0; *p = 5; return true;
    case PF_ODE_MICHAELIS3: *d = 3; *p = 4; return true;
  }
  return false;
}

// M2 grids: d = nt^2 with nt odd, 3 <= nt <= 45
static bool advdiff_dim_ok(int d) {
  for (int nt = 3; nt <= 45; nt += 2)
    if (nt * nt == d) return true;
  return false;
}

static size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Carve the filter's single device allocation.
static size_t layout(pf_filter* f, char* base) {
  const int64_t N = f->N;
  const int d = f->d, p = f->p;
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* ptr = base ? base + off : nullptr;
    off = align_up(off + bytes);
    return ptr;
  };
  for (int b = 0; b < 2; ++b) {
    f->fd.ens[b].x = (double*)take(sizeof(double) * N * d);
    f->fd.ens[b].h1 = (double*)take(sizeof(double) * N * d);
    f->fd.ens[b].h2 = (double*)take(sizeof(double) * N * d);
    f->fd.ens[b].phi = (double*)take(sizeof(double) * N * p);
    f->fd.ens[b].lw = (double*)take(sizeof(double) * N);
  }
  f->fd.ll1 = (double*)take(sizeof(double) * N);
  f->fd.lg = (double*)take(sizeof(double) * N);
  f->fd.c = (double*)take(sizeof(double) * N);
  f->fd.idx = (int32_t*)take(sizeof(int32_t) * N);
  const int sms = f->fd.sms;
  f->fd.blk = (double*)take(sizeof(double) * max_grid_blocks(N, sms));
  if (f->shard_total > 0) {
    // a shard keeps the whole ensemble's tile offsets; its own tiles are the
    // slice from its first tile on
    const int nb = f->shard_tiles_all;
    const int64_t t0 = f->shard_first / scan_tile_len(f->shard_total, sms);
    f->sh_boff = (double*)take(sizeof(double) * nb);
    f->sh_pmax = (double*)take(sizeof(double) * nb);
    f->sh_tiles = (double*)take(sizeof(double) * nb);
    f->sh_out = (double*)take(sizeof(double) * (nb + 2));
    f->sh_sums = (double*)take(sizeof(double) * f->fd.nrec);
    f->fd.boff = f->sh_boff ? f->sh_boff + t0 : nullptr;
    f->fd.pmax = f->sh_pmax ? f->sh_pmax + t0 : nullptr;
    f->sh_parent.x = (double*)take(sizeof(double) * N * d);
    f->sh_parent.h1 = (double*)take(sizeof(double) * N * d);
    f->sh_parent.h2 = (double*)take(sizeof(double) * N * d);
    f->sh_parent.phi = (double*)take(sizeof(double) * N * p);
    f->sh_parent.lw = nullptr;
    f->sh_parent_ll1 = (double*)take(sizeof(double) * N);
    f->sh_gparent = (int32_t*)take(sizeof(int32_t) * N);
  } else {
    f->fd.boff = (double*)take(sizeof(double) * scan_tiles(N, sms));
    f->fd.pmax = (double*)take(sizeof(double) * scan_tiles(N, sms));
  }
  f->fd.tsq = (double*)take(sizeof(double) * moment_blocks_max(sms));
  f->fd.part = (double*)take(sizeof(double) * moment_blocks_max(sms) * f->fd.nrec);
  // model work arrays: the Brusselator's stage buffers; the 2D system's
  // committed weights exp(lw - max lw), which the moments store for x-bar
  f->fd.wk = (f->ode == PF_ODE_BRUSSELATOR1D) ? (double*)take(sizeof(double) * bruss_work_doubles(N))
             : (f->ode == PF_ODE_ADVDIFF2D)   ? (double*)take(sizeof(double) * N)
                                              : nullptr;
  f->fd.x0 = (const double*)take(sizeof(double) * d);
  f->fd.xbar = (double*)take(sizeof(double) * d);
  f->fd.ticket = (unsigned*)take(sizeof(unsigned) * 8);
  f->fd.ctrl = (Ctrl*)take(sizeof(Ctrl));
  f->ep_dev = (EpochParams*)take(sizeof(EpochParams));
  return off;
}

namespace pfg {
size_t filter_device_bytes(int ode, int d, int p, int64_t N) {
  pf_filter probe;
  probe.ode = ode;
  probe.d = d;
  probe.p = p;
  probe.N = N;
  probe.fd.nrec = moment_record_size(ode);
  probe.fd.sms = device_sms();
  return layout(&probe, nullptr);
}
}  // namespace pfg

static double prior_center_phi(const pf_filter* f, int i) {
  const double lo = f->prior_lo[i], hi = f->prior_hi[i];
  if (f->prior_kind[i] == PF_PRIOR_LOGUNIFORM) {
    const double c = 0.5 * (std::log(lo) + std::log(hi));
    return f->transform == PF_TRANSFORM_LOG ? c : std::exp(c);
  }
  const double c = 0.5 * (lo + hi);
  return f->transform == PF_TRANSFORM_LOG ? std::log(c) : c;
}

// Ordered copy on the filter's stream, waited for (host buffers may be pageable).
static cudaError_t copy_sync(pf_filter* f, void* dst, const void* src, size_t bytes,
                             cudaMemcpyKind kind) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, kind, f->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(f->stream);
}

static pf_status read_ctrl(pf_filter* f) {
  PF_CUDA(f, cudaMemcpyAsync(f->ctrl_host, f->fd.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, f->stream));
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  f->d2h_bytes += sizeof(Ctrl);
  return PF_OK;
}

namespace pfg {
pf_status record_error(pf_filter* f, pf_status st, const std::string& msg) { return fail(f, st, msg); }

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    return kMaxSms;
  }
  return sms < kMaxSms ? sms : kMaxSms;
}
pf_status read_control(pf_filter* f) { return read_ctrl(f); }
}  // namespace pfg

namespace pfg {

cudaError_t preload_kernels() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64 || done[dev]) return cudaSuccess;
  e = preload_main_kernels();
  if (e == cudaSuccess) e = preload_bruss_kernels();
  if (e == cudaSuccess) e = preload_ad_kernels();
  if (e == cudaSuccess) done[dev] = true;
  return e;
}

}  // namespace pfg

// Step 1 into the existing buffers.
// check: wait for the initial moments and verify them.  Without it (pooled
// filters) nothing waits; a non-finite start shows up as the sticky status of
// the filter's first epoch.
static pf_status do_init(pf_filter* f, bool check = true) {
  const bool shard = f->shard_total > 0;
  Ctrl* h = f->ctrl_host;
  std::memset(h, 0, sizeof(Ctrl));
  h->cur = 0;
  h->status = PF_OK;
  for (int i = 0; i < f->p; ++i) h->phibar[i] = prior_center_phi(f, i);
  h->lw_max = 0.0;
  // small uploads as kernel parameters: a pooled filter's host blocks are
  // pageable, and a pageable copy may wait for the stream
  static_assert(sizeof(Ctrl) <= (size_t)kUploadBytes, "Ctrl fits a parameter upload");
  PF_CUDA(f, upload_small(f->fd.ctrl, h, sizeof(Ctrl), f->stream));
  PF_CUDA(f, upload_small(const_cast<double*>(f->fd.x0), f->x0.data(), sizeof(double) * f->d,
                          f->stream));
  PF_CUDA(f, cudaMemsetAsync(f->fd.ticket, 0, sizeof(unsigned) * 8, f->stream));
  // a shard draws its particles; the moments wait for every shard's sums
  PF_CUDA(f, shard ? launch_init_draws(f->ode, f->fd, f->stream) : launch_init(f->ode, f->fd, f->stream));
  f->hist = HistoryState{0, 0, f->t0, 0.0, 0.0};
  if (shard) {
    f->sh_stage = kShardInitDrawn;  // its moments wait for pf_shard_moments + pf_shard_commit
    return PF_OK;
  }
  if (!check) return PF_OK;
  pf_status st = read_ctrl(f);
  if (st != PF_OK) return st;
  if (f->ctrl_host->status != PF_OK)
    return fail(f, (pf_status)f->ctrl_host->status, "initial moments are not finite");
  return PF_OK;
}

namespace pfg {
// Parameter block of one epoch from the history state h.
int fill_epoch(const pf_filter* f, const HistoryState& h, double t_k, const double* y,
               EpochParams* ep, int* depth_out) {
  const int depth = (f->history == PF_HISTORY_RESTART) ? 0 : h.depth;
  static thread_local double times[kSMax + 1];
  const int S = build_substeps(f->lmm, f->spacing, f->dt, f->substeps, f->q0, h.t_prev, t_k, depth,
                               h.hprev1, h.hprev2, ep->sc, kSMax, depth_out, times);
  if (S < 1) return -1;
  ep->in_hist[0] = ep->in_hist[1] = 0.0;
  if (f->ode == PF_ODE_MICHAELIS3) {
    // M1's input at every substep's end points, and at t_n - h, t_n - 2h for
    // the Adams derivative history (constant step h)
    for (int i = 0; i < S; ++i) {
      ep->sc[i].in0 = mm_input(times[i]);
      ep->sc[i].in1 = mm_input(times[i + 1]);
    }
    const double h0 = times[1] - times[0];
    ep->in_hist[0] = mm_input(times[0] - h0);
    ep->in_hist[1] = mm_input(times[0] - 2.0 * h0);
  }
  ep->t = t_k;
  ep->S = S;
  ep->epoch = (uint32_t)h.epochs;
  ep->pad = 0;
  for (int i = 0; i < kMMax; ++i) {
    ep->y[i] = 0.0;
    ep->inv_sigma[i] = 0.0;
  }
  for (int i = 0; i < f->m; ++i) {
    ep->y[i] = y[i];
    double sig = f->sigma[i];
    if (f->noise == PF_NOISE_RELATIVE) sig = f->sigma[i] * std::fmax(std::fabs(y[i]), 1e-300);
    ep->inv_sigma[i] = 1.0 / sig;
  }
  return S;
}

HistoryState advance_history(const HistoryState& h, double t_k, const EpochParams* ep,
                             int depth_out) {
  HistoryState n = h;
  const int S = ep->S;
  n.epochs = h.epochs + 1;
  n.depth = depth_out;
  n.hprev1 = ep->sc[S - 1].h;
  n.hprev2 = S >= 2 ? ep->sc[S - 2].h : h.hprev1;
  n.t_prev = t_k;
  return n;
}
}  // namespace pfg

static pf_status clear_device_status(pf_filter* f) {
  PF_CUDA(f, cudaMemsetAsync(&f->fd.ctrl->status, 0, sizeof(int), f->stream));
  PF_CUDA(f, cudaMemsetAsync(f->fd.ticket, 0, sizeof(unsigned) * 8, f->stream));
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  return PF_OK;
}

static const char* status_text(int st) {
  switch (st) {
    case PF_ERR_DEGENERATE: return "degenerate epoch: every weight is zero or not finite";
    case PF_ERR_NUMERIC: return "non-finite weighted moments";
    case PF_ERR_TIMEOUT: return "device wait timed out";
  }
  return "epoch failed";
}

namespace pfg {
// Argument checks of pf_create (no allocation, no CUDA call).
pf_status check_create_args(pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                            const pf_prior* prior, const pf_options* opt) {
  int dd, pp;
  if (!ode_dims(ode, &dd, &pp)) return fail(nullptr, PF_ERR_INVALID_ARG, "unknown ODE");
  if (!ode_supported(ode)) return fail(nullptr, PF_ERR_INVALID_ARG, "ODE not available in this build");
  if (p != pp || (dd > 0 ? d != dd : !advdiff_dim_ok(d)))
    return fail(nullptr, PF_ERR_INVALID_ARG, "d or p does not match the ODE");
  if (N < 1 || N > PF_MAX_PARTICLES) return fail(nullptr, PF_ERR_INVALID_ARG, "N out of range");
  if (!lmm_known(lmm)) return fail(nullptr, PF_ERR_INVALID_ARG, "unknown LMM");
  if (lmm_needs_uniform(lmm) && ode != PF_ODE_LINEAR2 && ode != PF_ODE_ROBERTSON &&
      ode != PF_ODE_MICHAELIS3)
    return fail(nullptr, PF_ERR_INVALID_ARG, "BDF3 and the Adams methods run on the small problems only");
  if (!prior || !opt) return fail(nullptr, PF_ERR_INVALID_ARG, "prior or options is NULL");
  if (prior->p != p || prior->d != d || !prior->kind || !prior->lo || !prior->hi || !prior->x0)
    return fail(nullptr, PF_ERR_INVALID_ARG, "prior does not match the ODE");
  for (int i = 0; i < p; ++i) {
    const double lo = prior->lo[i], hi = prior->hi[i];
    if (!(std::isfinite(lo) && std::isfinite(hi) && lo <= hi))
      return fail(nullptr, PF_ERR_INVALID_ARG, "prior bounds must satisfy lo <= hi");
    if (prior->kind[i] == PF_PRIOR_LOGUNIFORM) {
      if (!(lo > 0.0)) return fail(nullptr, PF_ERR_INVALID_ARG, "log-uniform prior needs lo > 0");
    } else if (prior->kind[i] != PF_PRIOR_UNIFORM) {
      return fail(nullptr, PF_ERR_INVALID_ARG, "unknown prior kind");
    }
  }
  for (int i = 0; i < d; ++i)
    if (!std::isfinite(prior->x0[i])) return fail(nullptr, PF_ERR_INVALID_ARG, "x0 not finite");
  if (!(opt->a > 0.0 && opt->a <= 1.0)) return fail(nullptr, PF_ERR_INVALID_ARG, "need 0 < a <= 1");
  if (opt->newton_iters < 1 || opt->newton_iters > 64)
    return fail(nullptr, PF_ERR_INVALID_ARG, "newton_iters out of range");
  if (opt->m < 1 || opt->m > kMMax || !opt->obs_idx || !opt->sigma)
    return fail(nullptr, PF_ERR_INVALID_ARG, "need 1 <= m <= 32 observed components");
  for (int i = 0; i < opt->m; ++i) {
    if (opt->obs_idx[i] < 0 || opt->obs_idx[i] >= d)
      return fail(nullptr, PF_ERR_INVALID_ARG, "observation index out of range");
    if (!(opt->sigma[i] > 0.0) || !std::isfinite(opt->sigma[i]))
      return fail(nullptr, PF_ERR_INVALID_ARG, "sigma must be positive");
  }
  if (lmm_needs_uniform(lmm) && opt->spacing != PF_SPACING_UNIFORM)
    return fail(nullptr, PF_ERR_INVALID_ARG, "BDF3 and the Adams methods need uniform spacing");
  if (opt->spacing == PF_SPACING_UNIFORM) {
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, PF_ERR_INVALID_ARG, "dt must be positive");
  } else if (opt->spacing == PF_SPACING_GEOMETRIC) {
    if (opt->substeps < 1 || opt->substeps > kSMax)
      return fail(nullptr, PF_ERR_INVALID_ARG, "substeps out of range");
  } else {
    return fail(nullptr, PF_ERR_INVALID_ARG, "unknown spacing");
  }
  if (opt->history != PF_HISTORY_CARRY && opt->history != PF_HISTORY_RESTART)
    return fail(nullptr, PF_ERR_INVALID_ARG, "unknown history mode");
  if (opt->transform != PF_TRANSFORM_LOG && opt->transform != PF_TRANSFORM_IDENTITY)
    return fail(nullptr, PF_ERR_INVALID_ARG, "unknown transform");
  if (opt->noise != PF_NOISE_ADDITIVE && opt->noise != PF_NOISE_RELATIVE)
    return fail(nullptr, PF_ERR_INVALID_ARG, "unknown noise model");
  if (!(opt->kappa >= 0.0) || !std::isfinite(opt->kappa))
    return fail(nullptr, PF_ERR_INVALID_ARG, "kappa must be >= 0");
  if (opt->timing < 0 || opt->timing > 2) return fail(nullptr, PF_ERR_INVALID_ARG, "timing must be 0, 1 or 2");
  return PF_OK;
}
}  // namespace pfg

extern "C" {

const char* pf_version(void) { return "paper_1411_1702_gb300 0.1 (sm_103a, FP64)"; }

pf_status pf_create(pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                    const pf_prior* prior, const pf_options* opt, pf_filter** out) {
  const pfg::NvtxRange nvtx_range("pf_create");
  return filter_create(ode, d, p, N, lmm, dt, prior, opt, nullptr, out);
}

pf_status pf_device_bytes(pf_ode ode, int d, int p, int64_t N, size_t* bytes) {
  if (!bytes) return fail(nullptr, PF_ERR_INVALID_ARG, "bytes is NULL");
  if (!pfg::ode_supported(ode) || d < 1 || p < 1 || p > pfg::kPMax || N < 1)
    return fail(nullptr, PF_ERR_INVALID_ARG, "need a supported ode, d >= 1, 1 <= p <= 5, N >= 1");
  *bytes = pfg::filter_device_bytes(ode, d, p, N);
  return PF_OK;
}

pf_status pf_create_with_buffers(pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                                 const pf_prior* prior, const pf_options* opt, void* device_mem,
                                 size_t device_bytes, pf_filter** out) {
  const pfg::NvtxRange nvtx_range("pf_create_with_buffers");
  if (!device_mem) return fail(nullptr, PF_ERR_INVALID_ARG, "device_mem is NULL");
  return filter_create(ode, d, p, N, lmm, dt, prior, opt, nullptr, out, device_mem, device_bytes);
}

}  // extern "C"

namespace pfg {

pf_status filter_create(pf_ode ode, int d, int p, int64_t N, pf_lmm lmm, double dt,
                        const pf_prior* prior, const pf_options* opt, cudaMemPool_t pool,
                        pf_filter** out, void* ext_mem, size_t ext_bytes, int64_t shard_total,
                        int64_t shard_first) {
  if (!out) return fail(nullptr, PF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  {
    const pf_status cs = check_create_args(ode, d, p, N, lmm, dt, prior, opt);
    if (cs != PF_OK) return cs;
  }
  if (ext_mem) {
    if ((reinterpret_cast<uintptr_t>(ext_mem) & 255u) != 0)
      return fail(nullptr, PF_ERR_INVALID_ARG, "device_mem must be 256-byte aligned");
    const size_t need = filter_device_bytes(ode, d, p, N);
    if (ext_bytes < need)
      return fail(nullptr, PF_ERR_INVALID_ARG,
                  "device_bytes " + std::to_string(ext_bytes) + " < the " + std::to_string(need) +
                      " bytes pf_device_bytes reports");
    // device (or managed) memory of the current device; anything else would
    // only show as a fault in the first kernel
    cudaPointerAttributes pa{};
    int dev = -1;
    const bool known = cudaPointerGetAttributes(&pa, ext_mem) == cudaSuccess &&
                       cudaGetDevice(&dev) == cudaSuccess;
    if (!known) cudaGetLastError();
    if (!known || (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) ||
        pa.device != dev)
      return fail(nullptr, PF_ERR_INVALID_ARG, "device_mem is not device memory of the current device");
  }

  {
    const cudaError_t pe = preload_kernels();
    if (pe != cudaSuccess) return cuda_fail(nullptr, pe, "loading the kernels");
  }
  pf_filter* f = new (std::nothrow) pf_filter();
  if (!f) return fail(nullptr, PF_ERR_OOM, "host allocation failed");
  f->ode = ode; f->d = d; f->p = p; f->m = opt->m; f->lmm = lmm; f->K = opt->newton_iters;
  f->spacing = opt->spacing; f->substeps = opt->substeps; f->history = opt->history;
  f->transform = opt->transform; f->noise = opt->noise;
  f->dt = dt; f->q0 = opt->q0; f->a = opt->a; f->kappa = opt->kappa;
  f->seed = opt->seed; f->filter_id = opt->filter_id; f->N = N; f->t0 = prior->t0;
  f->timing = opt->timing;
  for (int i = 0; i < opt->m; ++i) { f->obs[i] = opt->obs_idx[i]; f->sigma[i] = opt->sigma[i]; }
  for (int i = 0; i < p; ++i) {
    f->prior_kind[i] = prior->kind[i]; f->prior_lo[i] = prior->lo[i]; f->prior_hi[i] = prior->hi[i];
  }
  f->x0.assign(prior->x0, prior->x0 + d);

  FilterDev& fd = f->fd;
  fd.N = N; fd.ode = ode; fd.lmm = lmm; fd.d = d; fd.p = p; fd.m = f->m; fd.K = f->K; fd.transform = f->transform;
  for (int i = 0; i < kMMax; ++i) fd.obs[i] = i < f->m ? f->obs[i] : 0;
  fd.a = f->a; fd.s = std::sqrt(1.0 - f->a * f->a); fd.kappa = f->kappa;
  fd.seed = f->seed; fd.stream_id = f->filter_id;
  fd.nrec = moment_record_size(ode);
  fd.slot0 = (uint32_t)shard_first;
  fd.Ntile = shard_total > 0 ? shard_total : N;
  fd.shard_sums = nullptr;
  fd.sms = device_sms();
  f->shard_total = shard_total;
  f->shard_first = shard_first;
  f->shard_tiles_all = shard_total > 0 ? scan_tile_count(shard_total, fd.sms) : 0;
  for (int i = 0; i < kPMax; ++i) {
    fd.prior_kind[i] = i < p ? f->prior_kind[i] : 0;
    fd.prior_lo[i] = i < p ? f->prior_lo[i] : 0.0;
    fd.prior_hi[i] = i < p ? f->prior_hi[i] : 0.0;
  }

  pf_status st = PF_OK;
  cudaError_t e;
  if (opt->stream) {
    f->stream = (cudaStream_t)opt->stream;
  } else {
    // a pooled filter's stream only initialises it: at the greatest priority,
    // so creation is not queued behind long kernels of other streams (the
    // server passes its own such stream, shared by all sessions)
    int least = 0, greatest = 0;
    if (pool) cudaDeviceGetStreamPriorityRange(&least, &greatest);
    e = cudaStreamCreateWithPriority(&f->stream, cudaStreamNonBlocking, pool ? greatest : 0);
    if (e != cudaSuccess) { st = cuda_fail(nullptr, e, "cudaStreamCreateWithPriority"); pf_destroy(f); return st; }
    f->own_stream = true;
  }
  f->dbytes = layout(f, nullptr);
  f->pool = pool;
  if (ext_mem) {
    f->dmem = ext_mem;
    f->ext_mem = true;
    e = cudaSuccess;
  } else {
    e = pool ? cudaMallocFromPoolAsync(&f->dmem, f->dbytes, pool, f->stream)
             : cudaMalloc(&f->dmem, f->dbytes);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    f->dmem = nullptr;
    g_thread_error = "device allocation of " + std::to_string(f->dbytes) + " bytes failed";
    pf_destroy(f);
    return PF_ERR_OOM;
  }
  layout(f, (char*)f->dmem);
  if (pool) {
    f->ep_host = new (std::nothrow) EpochParams();
    f->ctrl_host = new (std::nothrow) Ctrl();
    e = (f->ep_host && f->ctrl_host) ? cudaSuccess : cudaErrorMemoryAllocation;
  } else {
    e = cudaMallocHost(&f->ep_host, sizeof(EpochParams));
    if (e == cudaSuccess) e = cudaMallocHost(&f->ctrl_host, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaMallocHost(&f->xbar_host, sizeof(double) * f->d);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&f->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&f->ev1);
  if (e == cudaSuccess && pool) e = cudaEventCreateWithFlags(&f->ready, cudaEventDisableTiming);
  if (e != cudaSuccess) { st = cuda_fail(nullptr, e, "pinned buffers/events"); pf_destroy(f); return st; }
  st = do_init(f, pool == nullptr);
  if (st != PF_OK) {
    g_thread_error = f->err;
    pf_destroy(f);
    return st;
  }
  *out = f;
  return PF_OK;
}

}  // namespace pfg

extern "C" {

void pf_destroy(pf_filter* f) {
  if (!f) return;
  // A pooled filter (a server session) initialises on the server's shared init
  // stream and frees its memory in that stream's order, so it does not wait
  // for the other sessions' initialisations; its host blocks have no copy in
  // flight (its uploads travel as kernel parameters, its reads are waited for).
  if (f->stream && !f->pool) cudaStreamSynchronize(f->stream);
  if (f->series_dev) cudaFree(f->series_dev);
  if (f->pool) {
    if (f->dmem) cudaFreeAsync(f->dmem, f->stream);
    delete f->ep_host;
    delete f->ctrl_host;
  } else {
    if (f->dmem && !f->ext_mem) cudaFree(f->dmem);  // caller memory stays the caller's
    if (f->ep_host) cudaFreeHost(f->ep_host);
    if (f->ctrl_host) cudaFreeHost(f->ctrl_host);
    if (f->xbar_host) cudaFreeHost(f->xbar_host);
  }
  free_marks(f);
  for (cudaGraphExec_t x : f->epoch_exec)
    if (x) cudaGraphExecDestroy(x);
  if (f->ev0) cudaEventDestroy(f->ev0);
  if (f->ev1) cudaEventDestroy(f->ev1);
  if (f->ready) cudaEventDestroy(f->ready);
  if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
  delete f;
}

const char* pf_last_error(const pf_filter* f) {
  return f ? f->err.c_str() : g_thread_error.c_str();
}

static cudaError_t capture_epoch(pf_filter* f, int S, size_t bytes, cudaGraphExec_t* out);

// Returns the graph for S (captured into the next slot if none has it) or
// NULL when the stream cannot be captured.
static cudaGraphExec_t epoch_graph(pf_filter* f, int S, size_t bytes) {
  for (int i = 0; i < pf_filter::kEpochGraphs; ++i)
    if (f->epoch_exec[i] && f->epoch_exec_S[i] == S) return f->epoch_exec[i];
  const int slot = f->epoch_exec_next;
  f->epoch_exec_next = (slot + 1) % pf_filter::kEpochGraphs;
  if (f->epoch_exec[slot]) {
    cudaGraphExecDestroy(f->epoch_exec[slot]);
    f->epoch_exec[slot] = nullptr;
    f->epoch_exec_S[slot] = 0;
  }
  cudaGraphExec_t x = nullptr;
  if (capture_epoch(f, S, bytes, &x) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  f->epoch_exec[slot] = x;
  f->epoch_exec_S[slot] = S;
  return x;
}

// pf_assimilate's epoch as one graph: upload of the parameter block (bytes),
// the epoch's kernels, and the read-back of x-bar and the control block.  One
// graph launch replaces seven stream calls; the epoch's timing events are
// recorded around it, on the stream.
static cudaError_t capture_epoch(pf_filter* f, int S, size_t bytes, cudaGraphExec_t* out) {
  cudaError_t e = cudaStreamBeginCapture(f->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t le = cudaMemcpyAsync(f->ep_dev, f->ep_host, bytes, cudaMemcpyHostToDevice, f->stream);
  if (le == cudaSuccess) le = launch_epoch(f->ode, f->fd, f->ep_dev, S, f->stream, nullptr);
  if (le == cudaSuccess)
    le = cudaMemcpyAsync(f->xbar_host, f->fd.xbar, sizeof(double) * f->d, cudaMemcpyDeviceToHost,
                         f->stream);
  if (le == cudaSuccess)
    le = cudaMemcpyAsync(f->ctrl_host, f->fd.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, f->stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(f->stream, &g);
  if (le == cudaSuccess) le = e;
  *out = nullptr;
  if (le == cudaSuccess) le = cudaGraphInstantiate(out, g, 0);
  if (g) cudaGraphDestroy(g);
  if (le != cudaSuccess) *out = nullptr;
  return le;
}

pf_status pf_assimilate(pf_filter* f, double t_k, const double* y_k) {
  const pfg::NvtxRange nvtx_range("pf_assimilate");
  if (f && f->shard_total > 0) return fail(f, PF_ERR_STATE, "a shard's epochs run through the pf_shard_* calls");
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  if (!y_k) return fail(f, PF_ERR_INVALID_ARG, "y_k is NULL");
  for (int i = 0; i < f->m; ++i)
    if (!std::isfinite(y_k[i])) return fail(f, PF_ERR_INVALID_ARG, "observation is not finite");
  if (!std::isfinite(t_k) || !(t_k > f->hist.t_prev))
    return fail(f, PF_ERR_INVALID_ARG, "t_k must exceed the previous observation time");
  int depth_out = 0;
  const int S = fill_epoch(f, f->hist, t_k, y_k, f->ep_host, &depth_out);
  if (S < 1) return fail(f, PF_ERR_INVALID_ARG, "substep grid of the interval is invalid");
  f->est_fresh = false;
  const size_t bytes = kEpochHeaderBytes + sizeof(StepCoef) * (size_t)S;
  // the whole epoch as one graph launch where the host blocks are pinned and
  // no per-kernel events are wanted; a stream that cannot be captured (the
  // legacy default stream) takes the calls one by one
  bool graphed = false;
  if (!f->timing && f->xbar_host && !f->pool && f->stream) {
    const cudaGraphExec_t x = epoch_graph(f, S, bytes);
    if (x) {
      PF_CUDA(f, cudaEventRecord(f->ev0, f->stream));
      PF_CUDA(f, cudaGraphLaunch(x, f->stream));
      PF_CUDA(f, cudaEventRecord(f->ev1, f->stream));
      PF_CUDA(f, cudaStreamSynchronize(f->stream));
      graphed = true;
    }
  }
  f->h2d_bytes += (int64_t)bytes;
  if (f->xbar_host) f->d2h_bytes += (int64_t)(sizeof(double) * f->d);
  if (graphed) {
    f->d2h_bytes += sizeof(Ctrl);
  } else {
    PF_CUDA(f, cudaMemcpyAsync(f->ep_dev, f->ep_host, bytes, cudaMemcpyHostToDevice, f->stream));
    PF_CUDA(f, cudaEventRecord(f->ev0, f->stream));
    PF_CUDA(f, launch_epoch(f->ode, f->fd, f->ep_dev, S, f->stream, take_marks(f)));
    PF_CUDA(f, cudaEventRecord(f->ev1, f->stream));
    // x-bar comes back with the control block in the same wait, so estimates
    // asked for right after need no second round trip
    if (f->xbar_host)
      PF_CUDA(f, cudaMemcpyAsync(f->xbar_host, f->fd.xbar, sizeof(double) * f->d,
                                 cudaMemcpyDeviceToHost, f->stream));
    pf_status st = read_ctrl(f);
    if (st != PF_OK) return st;
  }
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, f->ev0, f->ev1) == cudaSuccess) f->last_ms = ms;
  else cudaGetLastError();  // a diagnostic only: leave no error behind
  const int dst = f->ctrl_host->status;
  if (dst != PF_OK) {
    pf_status cs = clear_device_status(f);
    if (cs != PF_OK) return cs;
    return fail(f, (pf_status)dst, status_text(dst));
  }
  f->hist = advance_history(f->hist, t_k, f->ep_host, depth_out);
  f->est_fresh = f->xbar_host != nullptr;
  return PF_OK;
}

pf_status pf_estimates(const pf_filter* cf, double* theta_bar, double* C, double* x_bar) {
  pf_filter* f = const_cast<pf_filter*>(cf);
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  if (f->est_fresh) {
    // right after pf_assimilate: its wait already brought the estimates back
    if (x_bar) std::memcpy(x_bar, f->xbar_host, sizeof(double) * f->d);
  } else {
    PF_CUDA(f, cudaMemcpyAsync(f->ctrl_host, f->fd.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                               f->stream));
    if (x_bar)
      PF_CUDA(f, cudaMemcpyAsync(x_bar, f->fd.xbar, sizeof(double) * f->d, cudaMemcpyDeviceToHost,
                                 f->stream));
    PF_CUDA(f, cudaStreamSynchronize(f->stream));
    f->d2h_bytes += sizeof(Ctrl) + (x_bar ? sizeof(double) * f->d : 0);
  }
  const Ctrl* h = f->ctrl_host;
  if (theta_bar) for (int i = 0; i < f->p; ++i) theta_bar[i] = h->phibar[i];
  if (C)
    for (int i = 0; i < f->p; ++i)
      for (int j = 0; j < f->p; ++j) C[i * f->p + j] = h->C[i * kPMax + j];
  return PF_OK;
}

pf_status pf_stats(const pf_filter* cf, pf_stats_t* out) {
  pf_filter* f = const_cast<pf_filter*>(cf);
  if (!f || !out) return fail(f, PF_ERR_INVALID_ARG, "NULL argument");
  PF_CUDA(f, launch_theta_mean(f->fd, f->stream));
  const bool have_lg = f->hist.epochs > 0;  // the first-stage weights of an epoch exist
  if (have_lg) PF_CUDA(f, launch_stage1_ess(f->fd, f->stream));
  pf_status st = read_ctrl(f);
  if (st != PF_OK) return st;
  const Ctrl* h = f->ctrl_host;
  std::memset(out, 0, sizeof(*out));
  out->epochs = h->epochs_done;
  out->ess = h->ess;
  out->log_weight_sum = h->logW;
  out->unique_parents = h->n_unique;
  out->nonfinite = h->n_nonfinite;
  for (int i = 0; i < f->p && i < 8; ++i) out->theta_mean[i] = h->theta_mean[i];
  out->last_epoch_ms = f->last_ms;
  out->h2d_bytes = f->h2d_bytes;
  out->d2h_bytes = f->d2h_bytes;
  out->ess_stage1 = (have_lg && h->g_sq > 0.0) ? h->c_total * h->c_total / h->g_sq : 0.0;
  return PF_OK;
}

pf_status pf_kernel_times(pf_filter* f, double* ms, int64_t* launches, int n) {
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  if (!ms || !launches || n < kEpochKernels) return fail(f, PF_ERR_INVALID_ARG, "need 6 slots");
  if (!f->timing) return fail(f, PF_ERR_STATE, "timing was not enabled at creation");
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  for (cudaEvent_t* m : f->mark_pending) {
    for (int i = 0; i < kEpochKernels; ++i) {
      // the scan_add slot has no launch and no event of its own (an empty
      // pair of events still costs the device about 2 us): 0, and the
      // resampling phase runs from the scan's end mark
      const cudaEvent_t a = m[i == kPhaseResample ? kPhaseScanAdd : i], b = m[i + 1];
      if (i == kPhaseScanAdd || !a || !b) continue;
      float t = 0.0f;
      PF_CUDA(f, cudaEventElapsedTime(&t, a, b));
      f->kernel_ms[i] += t;
      f->kernel_launches[i] += 1;
    }
    f->mark_free.push_back(m);
  }
  f->mark_pending.clear();
  for (int i = 0; i < n; ++i) {
    ms[i] = i < kEpochKernels ? f->kernel_ms[i] : 0.0;
    launches[i] = i < kEpochKernels ? f->kernel_launches[i] : 0;
  }
  for (int i = 0; i < kEpochKernels; ++i) {
    f->kernel_ms[i] = 0.0;
    f->kernel_launches[i] = 0;
  }
  return PF_OK;
}

pf_status pf_load_observations(pf_filter* f, int T, const double* t, const double* y) {
  if (f && f->shard_total > 0) return fail(f, PF_ERR_STATE, "a shard's epochs run through the pf_shard_* calls");
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  if (T < 1 || !t || !y) return fail(f, PF_ERR_INVALID_ARG, "need T >= 1 observations");
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  std::vector<EpochParams> host((size_t)T);
  std::vector<int> S((size_t)T);
  std::vector<HistoryState> after((size_t)T);
  HistoryState h = f->hist;
  for (int k = 0; k < T; ++k) {
    for (int i = 0; i < f->m; ++i)
      if (!std::isfinite(y[(size_t)k * f->m + i]))
        return fail(f, PF_ERR_INVALID_ARG, "observation is not finite");
    if (!std::isfinite(t[k]) || !(t[k] > h.t_prev))
      return fail(f, PF_ERR_INVALID_ARG, "observation times must increase");
    int depth_out = 0;
    S[k] = fill_epoch(f, h, t[k], y + (size_t)k * f->m, &host[k], &depth_out);
    if (S[k] < 1) return fail(f, PF_ERR_INVALID_ARG, "substep grid of an interval is invalid");
    h = advance_history(h, t[k], &host[k], depth_out);
    after[k] = h;
  }
  if (f->series_dev) {
    cudaFree(f->series_dev);
    f->series_dev = nullptr;
    f->series_T = 0;
  }
  EpochParams* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, sizeof(EpochParams) * (size_t)T);
  if (e != cudaSuccess) return fail(f, PF_ERR_OOM, "device allocation of the series failed");
  e = copy_sync(f, dev, host.data(), sizeof(EpochParams) * (size_t)T, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return cuda_fail(f, e, "cudaMemcpy(series)");
  }
  f->series_dev = dev;
  f->series_T = T;
  f->series_next = 0;
  f->series_S = S;
  f->series_after = after;
  f->series_start = f->hist;
  return PF_OK;
}

pf_status pf_run(pf_filter* f, int k0, int k1) {
  if (f && f->shard_total > 0) return fail(f, PF_ERR_STATE, "a shard's epochs run through the pf_shard_* calls");
  if (f) f->est_fresh = false;
  const pfg::NvtxRange nvtx_range("pf_run");
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  if (!f->series_dev) return fail(f, PF_ERR_STATE, "no observation series loaded");
  if (k0 != f->series_next) return fail(f, PF_ERR_STATE, "epochs must run in order");
  if (k1 < k0 || k1 > f->series_T) return fail(f, PF_ERR_INVALID_ARG, "epoch range out of bounds");
  for (int k = k0; k < k1; ++k) {
    PF_CUDA(f, launch_epoch(f->ode, f->fd, f->series_dev + k, f->series_S[k], f->stream,
                            take_marks(f)));
    f->hist = f->series_after[k];
  }
  f->series_next = k1;
  return PF_OK;
}

pf_status pf_synchronize(pf_filter* f) {
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  pf_status st = read_ctrl(f);
  if (st != PF_OK) return st;
  const int dst = f->ctrl_host->status;
  if (dst == PF_OK) return PF_OK;
  // roll the host view back to the last committed epoch
  const int64_t done = f->ctrl_host->epochs_done;
  const int64_t k = done - f->series_start.epochs;  // series index of the failed epoch
  if (f->series_dev && k >= 0 && k <= f->series_T) {
    f->hist = (k == 0) ? f->series_start : f->series_after[(size_t)k - 1];
    f->series_next = (int)k;
  }
  pf_status cs = clear_device_status(f);
  if (cs != PF_OK) return cs;
  return fail(f, (pf_status)dst, status_text(dst));
}

pf_status pf_reset(pf_filter* f) {
  if (f && f->shard_total > 0) return fail(f, PF_ERR_STATE, "a shard's epochs run through the pf_shard_* calls");
  if (f) f->est_fresh = false;
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  pf_status st = do_init(f);
  if (st != PF_OK) return st;
  if (f->series_dev) {
    const HistoryState& s = f->series_start;
    const bool from_start = s.epochs == 0 && s.depth == 0 && s.t_prev == f->t0;
    if (from_start) {
      f->series_next = 0;
    } else {
      cudaFree(f->series_dev);
      f->series_dev = nullptr;
      f->series_T = 0;
    }
  }
  return PF_OK;
}

pf_status pf_get_ensemble(const pf_filter* cf, double* x, double* h1, double* h2, double* phi,
                          double* logw) {
  pf_filter* f = const_cast<pf_filter*>(cf);
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  pf_status st = read_ctrl(f);
  if (st != PF_OK) return st;
  const Ensemble& E = f->ctrl_host->cur ? f->fd.ens[1] : f->fd.ens[0];
  const int64_t N = f->N;
  std::vector<double> tmp;
  auto pull = [&](const double* src, int rows, double* dst) -> pf_status {
    if (!dst) return PF_OK;
    tmp.resize((size_t)rows * N);
    PF_CUDA(f, copy_sync(f, tmp.data(), src, sizeof(double) * rows * N, cudaMemcpyDeviceToHost));
    f->d2h_bytes += (int64_t)(sizeof(double) * rows * N);
    for (int64_t n = 0; n < N; ++n)
      for (int i = 0; i < rows; ++i) dst[n * rows + i] = tmp[(size_t)i * N + n];
    return PF_OK;
  };
  if ((st = pull(E.x, f->d, x)) != PF_OK) return st;
  if ((st = pull(E.h1, f->d, h1)) != PF_OK) return st;
  if ((st = pull(E.h2, f->d, h2)) != PF_OK) return st;
  if ((st = pull(E.phi, f->p, phi)) != PF_OK) return st;
  if (logw) {
    if ((st = pull(E.lw, 1, logw)) != PF_OK) return st;
    const double lw0 = f->ctrl_host->logW;
    for (int64_t n = 0; n < N; ++n) logw[n] = logw[n] - lw0;
  }
  return PF_OK;
}

pf_status pf_set_ensemble(pf_filter* f, const double* x, const double* h1, const double* h2,
                          const double* phi, const double* logw) {
  if (f) f->est_fresh = false;
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  pf_status st = read_ctrl(f);
  if (st != PF_OK) return st;
  const Ensemble& E = f->ctrl_host->cur ? f->fd.ens[1] : f->fd.ens[0];
  const int64_t N = f->N;
  std::vector<double> tmp;
  auto push = [&](double* dst, int rows, const double* src) -> pf_status {
    if (!src) return PF_OK;
    tmp.resize((size_t)rows * N);
    for (int64_t n = 0; n < N; ++n)
      for (int i = 0; i < rows; ++i) tmp[(size_t)i * N + n] = src[n * rows + i];
    PF_CUDA(f, copy_sync(f, dst, tmp.data(), sizeof(double) * rows * N, cudaMemcpyHostToDevice));
    f->h2d_bytes += (int64_t)(sizeof(double) * rows * N);
    return PF_OK;
  };
  if ((st = push(E.x, f->d, x)) != PF_OK) return st;
  if ((st = push(E.h1, f->d, h1)) != PF_OK) return st;
  if ((st = push(E.h2, f->d, h2)) != PF_OK) return st;
  if ((st = push(E.phi, f->p, phi)) != PF_OK) return st;
  if (logw) {
    if ((st = push(E.lw, 1, logw)) != PF_OK) return st;
    const double zero = 0.0;
    PF_CUDA(f, copy_sync(f, &f->fd.ctrl->logW, &zero, sizeof(double), cudaMemcpyHostToDevice));
  }
  return PF_OK;
}

pf_status pf_set_moments(pf_filter* f, const double* phibar, const double* C) {
  if (f) f->est_fresh = false;
  if (!f || !phibar || !C) return fail(f, PF_ERR_INVALID_ARG, "NULL argument");
  pf_status st = read_ctrl(f);
  if (st != PF_OK) return st;
  Ctrl* h = f->ctrl_host;
  for (int i = 0; i < f->p; ++i) h->phibar[i] = phibar[i];
  for (int i = 0; i < f->p; ++i)
    for (int j = 0; j < f->p; ++j) h->C[i * kPMax + j] = C[i * f->p + j];
  PF_CUDA(f, cudaMemcpyAsync(f->fd.ctrl, h, sizeof(Ctrl), cudaMemcpyHostToDevice, f->stream));
  PF_CUDA(f, launch_set_moments(f->fd, f->stream));
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  return PF_OK;
}

// The maximum of two doubles >= +0 by their bit patterns (max_nonneg's rule).
static double max_nonneg_host(double a, double b) {
  long long x, y;
  std::memcpy(&x, &a, sizeof x);
  std::memcpy(&y, &b, sizeof y);
  return x > y ? a : b;
}

pf_status pf_get_work(const pf_filter* cf, double* loglik1, double* log_g, double* cumulative,
                      int32_t* idx) {
  pf_filter* f = const_cast<pf_filter*>(cf);
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  const size_t nb = sizeof(double) * f->N;
  if (loglik1) PF_CUDA(f, copy_sync(f, loglik1, f->fd.ll1, nb, cudaMemcpyDeviceToHost));
  if (log_g) PF_CUDA(f, copy_sync(f, log_g, f->fd.lg, nb, cudaMemcpyDeviceToHost));
  size_t tile_bytes = 0;
  if (cumulative) {
    // c as the scan leaves it (tile-local sums) with the tile offsets and
    // floors, combined here exactly as the device reads them (CumTiles)
    // (a shard: its own tiles of the whole ensemble's tiling)
    const int64_t len = scan_tile_len(f->fd.Ntile, f->fd.sms);
    const int nt = (int)((f->N + len - 1) / len);
    std::vector<double> boff(nt), pmax(nt);
    PF_CUDA(f, copy_sync(f, cumulative, f->fd.c, nb, cudaMemcpyDeviceToHost));
    PF_CUDA(f, copy_sync(f, boff.data(), f->fd.boff, sizeof(double) * nt, cudaMemcpyDeviceToHost));
    PF_CUDA(f, copy_sync(f, pmax.data(), f->fd.pmax, sizeof(double) * nt, cudaMemcpyDeviceToHost));
    tile_bytes = 2 * sizeof(double) * (size_t)nt;
    for (int64_t k = 0; k < f->N; ++k) {
      const int64_t t = k / len;
      cumulative[k] = max_nonneg_host(boff[t] + cumulative[k], pmax[t]);
    }
  }
  if (idx) PF_CUDA(f, copy_sync(f, idx, f->fd.idx, sizeof(int32_t) * f->N, cudaMemcpyDeviceToHost));
  f->d2h_bytes += (int64_t)((loglik1 ? nb : 0) + (log_g ? nb : 0) + (cumulative ? nb : 0) +
                            tile_bytes + (idx ? sizeof(int32_t) * f->N : 0));
  return PF_OK;
}

// ---- checkpoint / resume ---------------------------------------------------
// Blob: a header, the raw control block, the committed ensemble in its device
// layout (x, h1, h2: d*N each, component-major; phi: p*N; unnormalised log
// weights: N) and the committed weighted mean state (d).  Native byte order.
namespace {
struct CkptHeader {
  char magic[8];
  uint32_t version;
  int32_t ode, d, p, lmm;
  int32_t depth;
  int64_t N;
  int64_t epochs;
  double t_prev, hprev1, hprev2;
  uint64_t seed;
  uint32_t filter_id;
  uint32_t pad;
  uint64_t total_bytes;
};
constexpr char kCkptMagic[8] = {'P', 'F', 'C', 'K', 'P', 'T', '0', '1'};

size_t ckpt_bytes(const pf_filter* f) {
  const size_t N = (size_t)f->N;
  return sizeof(CkptHeader) + sizeof(Ctrl) +
         sizeof(double) * (N * (3 * (size_t)f->d + (size_t)f->p + 1) + (size_t)f->d);
}
}  // namespace

pf_status pf_checkpoint_size(const pf_filter* f, size_t* bytes) {
  if (!f || !bytes) return fail(nullptr, PF_ERR_INVALID_ARG, "NULL argument");
  *bytes = ckpt_bytes(f);
  return PF_OK;
}

pf_status pf_save(const pf_filter* cf, void* buf, size_t bytes) {
  if (cf && cf->shard_total > 0) return fail(const_cast<pf_filter*>(cf), PF_ERR_STATE, "a shard's epochs run through the pf_shard_* calls");
  pf_filter* f = const_cast<pf_filter*>(cf);
  if (!f || !buf) return fail(nullptr, PF_ERR_INVALID_ARG, "NULL argument");
  const size_t need = ckpt_bytes(f);
  if (bytes < need) return fail(f, PF_ERR_INVALID_ARG, "checkpoint buffer too small");
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  pf_status st = read_ctrl(f);
  if (st != PF_OK) return st;
  if (f->ctrl_host->status != PF_OK) return fail(f, PF_ERR_STATE, "the filter has a failed epoch pending");
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, 8);
  h.version = 1;
  h.ode = f->ode; h.d = f->d; h.p = f->p; h.lmm = f->lmm;
  h.depth = f->hist.depth;
  h.N = f->N;
  h.epochs = f->hist.epochs;
  h.t_prev = f->hist.t_prev; h.hprev1 = f->hist.hprev1; h.hprev2 = f->hist.hprev2;
  h.seed = f->seed; h.filter_id = f->filter_id;
  h.total_bytes = need;
  char* out = static_cast<char*>(buf);
  std::memcpy(out, &h, sizeof h);
  out += sizeof h;
  std::memcpy(out, f->ctrl_host, sizeof(Ctrl));
  out += sizeof(Ctrl);
  const Ensemble& E = f->ctrl_host->cur ? f->fd.ens[1] : f->fd.ens[0];
  const size_t N = (size_t)f->N, d = (size_t)f->d, p = (size_t)f->p;
  const struct { const double* src; size_t n; } parts[] = {
      {E.x, d * N}, {E.h1, d * N}, {E.h2, d * N}, {E.phi, p * N}, {E.lw, N}, {f->fd.xbar, d}};
  for (const auto& part : parts) {
    PF_CUDA(f, copy_sync(f, out, part.src, sizeof(double) * part.n, cudaMemcpyDeviceToHost));
    f->d2h_bytes += (int64_t)(sizeof(double) * part.n);
    out += sizeof(double) * part.n;
  }
  return PF_OK;
}

pf_status pf_load(pf_filter* f, const void* buf, size_t bytes) {
  if (f && f->shard_total > 0) return fail(f, PF_ERR_STATE, "a shard's epochs run through the pf_shard_* calls");
  if (f) f->est_fresh = false;
  if (!f || !buf) return fail(nullptr, PF_ERR_INVALID_ARG, "NULL argument");
  if (f->in_batch) return fail(f, PF_ERR_STATE, "the filter is a member of a batch");
  CkptHeader h;
  if (bytes < sizeof h) return fail(f, PF_ERR_INVALID_ARG, "checkpoint too short");
  std::memcpy(&h, buf, sizeof h);
  if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1)
    return fail(f, PF_ERR_INVALID_ARG, "not a checkpoint of this library");
  if (h.ode != f->ode || h.d != f->d || h.p != f->p || h.lmm != f->lmm || h.N != f->N)
    return fail(f, PF_ERR_INVALID_ARG, "checkpoint of a different problem, LMM or N");
  if (h.seed != f->seed || h.filter_id != f->filter_id)
    return fail(f, PF_ERR_INVALID_ARG, "checkpoint of a filter with another seed or filter id");
  const size_t need = ckpt_bytes(f);
  if (h.total_bytes != need || bytes < need) return fail(f, PF_ERR_INVALID_ARG, "checkpoint truncated");
  if (h.epochs < 0 || h.depth < 0 || h.depth > 2 || !std::isfinite(h.t_prev))
    return fail(f, PF_ERR_INVALID_ARG, "checkpoint history out of range");
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  const char* in = static_cast<const char*>(buf) + sizeof h;
  Ctrl c;
  std::memcpy(&c, in, sizeof c);
  in += sizeof c;
  c.cur = 0;
  c.status = PF_OK;
  const Ensemble& E = f->fd.ens[0];
  const size_t N = (size_t)f->N, d = (size_t)f->d, p = (size_t)f->p;
  const struct { double* dst; size_t n; } parts[] = {
      {E.x, d * N}, {E.h1, d * N}, {E.h2, d * N}, {E.phi, p * N}, {E.lw, N}, {f->fd.xbar, d}};
  for (const auto& part : parts) {
    PF_CUDA(f, copy_sync(f, part.dst, in, sizeof(double) * part.n, cudaMemcpyHostToDevice));
    f->h2d_bytes += (int64_t)(sizeof(double) * part.n);
    in += sizeof(double) * part.n;
  }
  *f->ctrl_host = c;
  PF_CUDA(f, copy_sync(f, f->fd.ctrl, f->ctrl_host, sizeof(Ctrl), cudaMemcpyHostToDevice));
  PF_CUDA(f, cudaMemsetAsync(f->fd.ticket, 0, sizeof(unsigned) * 8, f->stream));
  PF_CUDA(f, cudaStreamSynchronize(f->stream));
  f->hist = HistoryState{h.epochs, h.depth, h.t_prev, h.hprev1, h.hprev2};
  if (f->series_dev) {
    cudaFree(f->series_dev);
    f->series_dev = nullptr;
    f->series_T = 0;
  }
  return PF_OK;
}

pf_status pf_get_history(const pf_filter* f, int64_t* epochs, int* depth, double* t_prev,
                         double* hprev1, double* hprev2) {
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  if (epochs) *epochs = f->hist.epochs;
  if (depth) *depth = f->hist.depth;
  if (t_prev) *t_prev = f->hist.t_prev;
  if (hprev1) *hprev1 = f->hist.hprev1;
  if (hprev2) *hprev2 = f->hist.hprev2;
  return PF_OK;
}

pf_status pf_set_history(pf_filter* f, int64_t epochs, int depth, double t_prev, double hprev1,
                         double hprev2) {
  if (f) f->est_fresh = false;
  if (!f) return fail(nullptr, PF_ERR_INVALID_ARG, "filter is NULL");
  if (epochs < 0 || depth < 0 || depth > 2 || !std::isfinite(t_prev))
    return fail(f, PF_ERR_INVALID_ARG, "history out of range");
  f->hist = HistoryState{epochs, depth, t_prev, hprev1, hprev2};
  PF_CUDA(f, copy_sync(f, &f->fd.ctrl->epochs_done, &epochs, sizeof(int64_t), cudaMemcpyHostToDevice));
  if (f->series_dev) {
    cudaFree(f->series_dev);
    f->series_dev = nullptr;
    f->series_T = 0;
  }
  return PF_OK;
}

}  // extern "C"
