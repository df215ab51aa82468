// pf_shard.cu -- one shard of a particle-sharded filter (the pf_shard_* calls
// of include/pf.h).
//
// Algorithm 1's loops over particles are independent, which is the paper's
// particle-parallel layout (Sec. 3.1).  A filter of N particles can therefore
// be split into contiguous shards, one per GPU, that couple only through
// global quantities each epoch: the log-sum-exp shifts of Steps 3a and 5, the
// cumulative weights of Step 3b (their tile totals), the parents of the
// resampled slots (Step 3c: a parent may live on another shard) and the
// moment sums of Step 6.  A shard is a pf_filter over its own slots whose
// random streams are keyed by the global slot; the calls below run one phase
// each and hand the host exactly what the other shards need, so that a caller
// (the coordinator in paper_1411_1702_gb300/shard.py) can exchange it over
// NCCL, gloo or host memory.
//
// A shard starts on a tile boundary of the whole ensemble's scan tiling
// (pf_shard_tile), so its tile totals are those of a filter of the whole
// ensemble and the offsets that k_shard_offsets derives from all of them are
// the same bits: the cumulative weights, and so the resampled parents, are
// bit-identical to a single filter's.  The moment sums are added in shard
// order, so the committed moments equal a single filter's up to rounding.
#include <cmath>
#include <cstring>
#include <string>

#include "pf_filter.h"
#include "pf_scan.cuh"

using namespace pfg;

namespace {

// phases of a shard's epoch, in call order (the first two are shared with
// the Step 1 code of pf_capi.cu through pf_filter.h)
constexpr int kShIdle = kShardIdle;
constexpr int kShInitDrawn = kShardInitDrawn;
enum : int {
  kShStage1 = 2,
  kShScan = 3,
  kShOffsets = 4,
  kShResample = 5,
  kShStage2 = 6,
  kShSummed = 7,      // this shard's moment sums taken; the next call is pf_shard_commit
  kShInitSummed = 8
};

pf_status sfail(pf_filter* f, pf_status st, const std::string& msg) { return record_error(f, st, msg); }

#define SH_CUDA(f, call)                                                                       \
  do {                                                                                         \
    cudaError_t e__ = (call);                                                                  \
    if (e__ != cudaSuccess)                                                                    \
      return sfail(f, PF_ERR_CUDA, std::string("CUDA error in ") + #call + ": " +             \
                                      cudaGetErrorName(e__) + " (" + cudaGetErrorString(e__) + ")"); \
  } while (0)

int record_doubles(const pf_filter* f) { return 3 * f->d + f->p + 2; }

int64_t local_tiles(const pf_filter* f) {
  const int64_t L = scan_tile_len(f->shard_total, f->fd.sms);
  return (f->N + L - 1) / L;
}

pf_status need(pf_filter* f, int stage, const char* call) {
  if (!f) return sfail(nullptr, PF_ERR_INVALID_ARG, std::string(call) + ": filter is NULL");
  if (f->shard_total <= 0) return sfail(f, PF_ERR_STATE, std::string(call) + ": not a shard");
  if (f->sh_stage != stage)
    return sfail(f, PF_ERR_STATE, std::string(call) + ": called out of order (phase " +
                                      std::to_string(f->sh_stage) + ")");
  return PF_OK;
}

// A shard's own maximum may be -inf (its particles all failed) while the
// epoch is not degenerate: only the global maximum decides, so the sticky
// status a stage tail set for the local maximum is cleared.
pf_status clear_local_degenerate(pf_filter* f) {
  Ctrl* h = f->ctrl_host;
  if (h->status == PF_ERR_DEGENERATE) {
    SH_CUDA(f, cudaMemsetAsync(&f->fd.ctrl->status, 0, sizeof(int), f->stream));
    h->status = PF_OK;
  } else if (h->status != PF_OK) {
    return sfail(f, (pf_status)h->status, "shard epoch failed");
  }
  return PF_OK;
}

pf_status set_ctrl_double(pf_filter* f, double* dev_field, double v) {
  SH_CUDA(f, upload_small(dev_field, &v, sizeof(double), f->stream));
  return PF_OK;
}

}  // namespace

extern "C" {

int64_t pf_shard_tile(int64_t N) { return N >= 1 ? scan_tile_len(N, device_sms()) : 0; }

pf_status pf_shard_create(pf_ode ode, int d, int p, int64_t N, int64_t first, int64_t n, pf_lmm lmm,
                          double dt, const pf_prior* prior, const pf_options* opt, pf_filter** out) {
  const pfg::NvtxRange nvtx_range("pf_shard_create");
  if (out) *out = nullptr;
  if (ode != PF_ODE_LINEAR2 && ode != PF_ODE_ROBERTSON && ode != PF_ODE_MICHAELIS3 &&
      ode != PF_ODE_BRUSSELATOR1D) {
    set_thread_error("pf_shard_create: the 2D advection-diffusion system has no shard kernels");
    return PF_ERR_INVALID_ARG;
  }
  if (N < 1 || N > PF_MAX_PARTICLES || n < 1 || first < 0 || first + n > N) {
    set_thread_error("pf_shard_create: need 1 <= n and 0 <= first, first + n <= N <= PF_MAX_PARTICLES");
    return PF_ERR_INVALID_ARG;
  }
  const int64_t L = scan_tile_len(N, device_sms());
  if (first % L != 0 || (first + n != N && n % L != 0)) {
    set_thread_error("pf_shard_create: a shard must start on a multiple of pf_shard_tile(N) and, "
                     "unless it is the last, hold a multiple of it");
    return PF_ERR_INVALID_ARG;
  }
  return filter_create(ode, d, p, n, lmm, dt, prior, opt, nullptr, out, nullptr, 0, N, first);
}

pf_status pf_shard_info(const pf_filter* cf, int64_t* total, int64_t* first, int* tiles,
                        int* tiles_all, int* record) {
  pf_filter* f = const_cast<pf_filter*>(cf);
  if (!f) return sfail(nullptr, PF_ERR_INVALID_ARG, "pf_shard_info: filter is NULL");
  if (f->shard_total <= 0) return sfail(f, PF_ERR_STATE, "pf_shard_info: not a shard");
  if (total) *total = f->shard_total;
  if (first) *first = f->shard_first;
  if (tiles) *tiles = (int)local_tiles(f);
  if (tiles_all) *tiles_all = f->shard_tiles_all;
  if (record) *record = record_doubles(f);
  return PF_OK;
}

pf_status pf_shard_stage1(pf_filter* f, double t_k, const double* y_k, double* lg_max) {
  const pfg::NvtxRange nvtx_range("pf_shard_stage1");
  pf_status st = need(f, kShIdle, "pf_shard_stage1");
  if (st != PF_OK) return st;
  if (!y_k || !lg_max) return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_stage1: NULL argument");
  for (int i = 0; i < f->m; ++i)
    if (!std::isfinite(y_k[i])) return sfail(f, PF_ERR_INVALID_ARG, "observation is not finite");
  if (!std::isfinite(t_k) || !(t_k > f->hist.t_prev))
    return sfail(f, PF_ERR_INVALID_ARG, "t_k must exceed the previous observation time");
  const int S = fill_epoch(f, f->hist, t_k, y_k, f->ep_host, &f->sh_depth_out);
  if (S < 1) return sfail(f, PF_ERR_INVALID_ARG, "substep grid of the interval is invalid");
  f->est_fresh = false;
  const size_t bytes = kEpochHeaderBytes + sizeof(StepCoef) * (size_t)S;
  SH_CUDA(f, cudaMemcpyAsync(f->ep_dev, f->ep_host, bytes, cudaMemcpyHostToDevice, f->stream));
  f->h2d_bytes += (int64_t)bytes;
  SH_CUDA(f, launch_stage(1, f->fd, f->ep_dev, S, f->stream));
  if ((st = read_control(f)) != PF_OK) return st;
  *lg_max = f->ctrl_host->lg_max;
  if ((st = clear_local_degenerate(f)) != PF_OK) return st;
  f->sh_t = t_k;
  f->sh_stage = kShStage1;
  return PF_OK;
}

pf_status pf_shard_scan(pf_filter* f, double lg_max, double* tiles, double* cl_last) {
  const pfg::NvtxRange nvtx_range("pf_shard_scan");
  pf_status st = need(f, kShStage1, "pf_shard_scan");
  if (st != PF_OK) return st;
  if (!tiles || !cl_last) return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_scan: NULL argument");
  if (!(lg_max > -INFINITY) || !std::isfinite(lg_max))
    return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_scan: the global maximum must be finite");
  if ((st = set_ctrl_double(f, &f->fd.ctrl->lg_max, lg_max)) != PF_OK) return st;
  const int nt = (int)local_tiles(f);
  SH_CUDA(f, launch_scan_tiles(f->fd, nt, f->stream));
  // the tile totals are in the per-block scratch; the last slot's tile-local
  // value decides c_{N-1} when this is the last shard
  SH_CUDA(f, cudaMemcpyAsync(tiles, f->fd.blk, sizeof(double) * nt, cudaMemcpyDeviceToHost, f->stream));
  SH_CUDA(f, cudaMemcpyAsync(cl_last, f->fd.c + (f->N - 1), sizeof(double), cudaMemcpyDeviceToHost,
                             f->stream));
  SH_CUDA(f, cudaStreamSynchronize(f->stream));
  f->d2h_bytes += (int64_t)(sizeof(double) * (nt + 1));
  f->sh_stage = kShScan;
  return PF_OK;
}

pf_status pf_shard_offsets(pf_filter* f, const double* tiles_all, double cl_last, double* tile_end,
                           double* total, double* u) {
  const pfg::NvtxRange nvtx_range("pf_shard_offsets");
  pf_status st = need(f, kShScan, "pf_shard_offsets");
  if (st != PF_OK) return st;
  if (!tiles_all || !tile_end || !total || !u)
    return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_offsets: NULL argument");
  const int nb = f->shard_tiles_all;
  SH_CUDA(f, cudaMemcpyAsync(f->sh_tiles, tiles_all, sizeof(double) * nb, cudaMemcpyHostToDevice,
                             f->stream));
  SH_CUDA(f, launch_shard_offsets(f->fd, f->ep_dev, f->sh_tiles, nb, cl_last, f->sh_boff,
                                  f->sh_pmax, f->sh_out, f->stream));
  SH_CUDA(f, cudaMemcpyAsync(tile_end, f->sh_out, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                             f->stream));
  double tu[2];
  SH_CUDA(f, cudaMemcpyAsync(tu, f->sh_out + nb, sizeof(double) * 2, cudaMemcpyDeviceToHost, f->stream));
  SH_CUDA(f, cudaStreamSynchronize(f->stream));
  f->h2d_bytes += (int64_t)(sizeof(double) * nb);
  f->d2h_bytes += (int64_t)(sizeof(double) * (nb + 2));
  *total = tu[0];
  *u = tu[1];
  f->sh_stage = kShOffsets;
  return PF_OK;
}

pf_status pf_shard_resample(pf_filter* f, int64_t i_lo, int64_t i_hi, int64_t i_fb, double u,
                            double total, double* send) {
  const pfg::NvtxRange nvtx_range("pf_shard_resample");
  pf_status st = need(f, kShOffsets, "pf_shard_resample");
  if (st != PF_OK) return st;
  const int64_t NA = f->shard_total;
  if (i_lo < 0 || i_hi < i_lo || i_hi > NA || i_fb < 0 || i_fb > NA || !(u >= 0.0 && u < 1.0) ||
      !(total > 0.0) || (i_hi > i_lo && !send))
    return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_resample: bad output range, u, total or buffer");
  SH_CUDA(f, launch_shard_resample(f->fd, i_lo, i_hi - i_lo, i_fb, u, total, NA, send, f->stream));
  SH_CUDA(f, cudaStreamSynchronize(f->stream));
  f->sh_stage = kShResample;
  return PF_OK;
}

pf_status pf_shard_stage2(pf_filter* f, const double* recv, double* lw_max) {
  const pfg::NvtxRange nvtx_range("pf_shard_stage2");
  pf_status st = need(f, kShResample, "pf_shard_stage2");
  if (st != PF_OK) return st;
  if (!recv || !lw_max) return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_stage2: NULL argument");
  SH_CUDA(f, launch_shard_unpack(f->fd, recv, f->sh_parent, f->sh_parent_ll1, f->sh_gparent, f->stream));
  // stage 2 gathers from the received parents: the committed buffers of this
  // descriptor are the parent buffers (lw is not read), the gather index is
  // the identity the unpack wrote; it writes the pending buffer as usual
  if ((st = read_control(f)) != PF_OK) return st;
  FilterDev fp = f->fd;
  const int cur = f->ctrl_host->cur;
  fp.ens[cur].x = f->sh_parent.x;
  fp.ens[cur].h1 = f->sh_parent.h1;
  fp.ens[cur].h2 = f->sh_parent.h2;
  fp.ens[cur].phi = f->sh_parent.phi;
  fp.ll1 = f->sh_parent_ll1;
  SH_CUDA(f, launch_stage(2, fp, f->ep_dev, f->ep_host->S, f->stream));
  if ((st = read_control(f)) != PF_OK) return st;
  *lw_max = f->ctrl_host->lw_max;
  if ((st = clear_local_degenerate(f)) != PF_OK) return st;
  f->sh_stage = kShStage2;
  return PF_OK;
}

pf_status pf_shard_moments(pf_filter* f, double lw_max, double* sums, int* nv) {
  const pfg::NvtxRange nvtx_range("pf_shard_moments");
  if (!f) return sfail(nullptr, PF_ERR_INVALID_ARG, "pf_shard_moments: filter is NULL");
  const bool init = f->sh_stage == kShInitDrawn;
  pf_status st = need(f, init ? kShInitDrawn : kShStage2, "pf_shard_moments");
  if (st != PF_OK) return st;
  if (!sums || !nv) return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_moments: NULL argument");
  if (!std::isfinite(lw_max))
    return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_moments: the global maximum must be finite");
  if ((st = set_ctrl_double(f, &f->fd.ctrl->lw_max, lw_max)) != PF_OK) return st;
  FilterDev fs = f->fd;
  fs.shard_sums = f->sh_sums;
  SH_CUDA(f, launch_shard_moments(fs, f->stream));
  SH_CUDA(f, cudaMemcpyAsync(sums, f->sh_sums, sizeof(double) * f->fd.nrec, cudaMemcpyDeviceToHost,
                             f->stream));
  SH_CUDA(f, cudaStreamSynchronize(f->stream));
  f->d2h_bytes += (int64_t)(sizeof(double) * f->fd.nrec);
  *nv = f->fd.nrec;
  f->sh_stage = init ? kShInitSummed : kShSummed;
  return PF_OK;
}

pf_status pf_shard_commit(pf_filter* f, const double* sums, int nv) {
  const pfg::NvtxRange nvtx_range("pf_shard_commit");
  if (!f) return sfail(nullptr, PF_ERR_INVALID_ARG, "pf_shard_commit: filter is NULL");
  const bool init = f->sh_stage == kShInitSummed;
  pf_status st = need(f, init ? kShInitSummed : kShSummed, "pf_shard_commit");
  if (st != PF_OK) return st;
  if (!sums || nv != f->fd.nrec) return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_commit: need the nv sums");
  SH_CUDA(f, cudaMemcpyAsync(f->sh_sums, sums, sizeof(double) * nv, cudaMemcpyHostToDevice, f->stream));
  SH_CUDA(f, launch_shard_commit(f->fd, f->sh_sums, init ? 1 : 0, f->stream));
  if ((st = read_control(f)) != PF_OK) return st;
  const int dst = f->ctrl_host->status;
  if (dst != PF_OK) {
    // nothing was committed: the epoch can be redone from stage 1
    SH_CUDA(f, cudaMemsetAsync(&f->fd.ctrl->status, 0, sizeof(int), f->stream));
    SH_CUDA(f, cudaStreamSynchronize(f->stream));
    f->sh_stage = init ? kShInitDrawn : kShIdle;
    return sfail(f, (pf_status)dst, "non-finite weighted moments");
  }
  if (!init) f->hist = advance_history(f->hist, f->sh_t, f->ep_host, f->sh_depth_out);
  f->sh_stage = kShIdle;
  return PF_OK;
}

pf_status pf_shard_abort(pf_filter* f) {
  if (!f) return sfail(nullptr, PF_ERR_INVALID_ARG, "pf_shard_abort: filter is NULL");
  if (f->shard_total <= 0) return sfail(f, PF_ERR_STATE, "pf_shard_abort: not a shard");
  if (f->sh_stage == kShInitDrawn || f->sh_stage == kShInitSummed)
    return sfail(f, PF_ERR_STATE, "pf_shard_abort: Step 1 has no committed state to return to");
  SH_CUDA(f, cudaMemsetAsync(&f->fd.ctrl->status, 0, sizeof(int), f->stream));
  SH_CUDA(f, cudaMemsetAsync(f->fd.ticket, 0, sizeof(unsigned) * 8, f->stream));
  SH_CUDA(f, cudaStreamSynchronize(f->stream));
  f->sh_stage = kShIdle;
  return PF_OK;
}

pf_status pf_shard_parents(const pf_filter* cf, int32_t* parents) {
  pf_filter* f = const_cast<pf_filter*>(cf);
  if (!f || !parents) return sfail(f, PF_ERR_INVALID_ARG, "pf_shard_parents: NULL argument");
  if (f->shard_total <= 0) return sfail(f, PF_ERR_STATE, "pf_shard_parents: not a shard");
  SH_CUDA(f, cudaMemcpyAsync(parents, f->sh_gparent, sizeof(int32_t) * f->N, cudaMemcpyDeviceToHost,
                             f->stream));
  SH_CUDA(f, cudaStreamSynchronize(f->stream));
  return PF_OK;
}

}  // extern "C"
