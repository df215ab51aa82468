// pf_kernels.cu -- the per-observation epoch of Algorithm 1 (Arnold, Calvetti,
// Somersalo) as CUDA kernels for sm_103a, for one filter or for a batch.
//
// One epoch j -> j+1 is five phases:
//   stage1      Steps 2, 3a: shrink phi, propagate by Psi, first-stage log
//               weights log g = log w + log pi(y | xbar); the filter's last
//               block takes the maximum (log-sum-exp shift)
//   scan_tile   Step 3a/3b: g = exp(log g - max), tile-local inclusive scan;
//               the filter's last block scans the tile totals into offsets
//   resample    Step 3b: systematic resampling, l_i = min{k : c_k > tau_i},
//               reading c_k = tile offset + tile-local sum on the fly
//               (CumTiles: no pass of its own stores the final c)
//   stage2      Steps 3c, 4, 5: gather by l, proliferate phi, repropagate with
//               the Milne local-error sums, innovation, new log weights
//   moments     Steps 5-6: normalisation, weighted mean/covariance of phi,
//               mean state, ESS; the filter's last block commits (flips the
//               ensemble buffer) unless the epoch is degenerate
// Every phase is a device function of a virtual block index vb in [0, vg):
// a single-filter launch runs it with (blockIdx.x, gridDim.x); a batched
// launch reads (filter, vb) from a tile table, so one launch serves any number
// of filters of any size.  A filter's reduction trees depend only on its N,
// never on where its tiles land, so a filter gives bit-identical results alone
// and in a batch.  Every phase returns at once if an earlier epoch of its
// filter failed (Ctrl::status), so epochs can be enqueued ahead.  A filter's
// own epoch (linear2, Robertson, M1) launches its kernels with programmatic
// dependent launch: each waits (pdl_wait) before touching the epoch's state.
#include <cstring>

#include "pf_common.cuh"
#include "pf_epoch.cuh"
#include "pf_kernels.h"
#include "pf_models.cuh"
#include "pf_scan.cuh"

namespace pfg {

constexpr int kSmallThreads = 128;
constexpr int kInitThreads = 256;

// Gaussian log-likelihood of the observed components, without the constant
// terms (they cancel in every normalisation of Steps 3a and 5).
template <int D>
__device__ __forceinline__ double loglik(const FilterDev& fd, const EpochParams* __restrict__ ep,
                                         const double (&x)[D]) {
  double s = 0.0;
  for (int i = 0; i < fd.m; ++i) {
    const int o = fd.obs[i];
    double xo = x[0];
#pragma unroll
    for (int j = 1; j < D; ++j) xo = (o == j) ? x[j] : xo;
    const double z = (ep->y[i] - xo) * ep->inv_sigma[i];
    s = fma(z, z, s);
  }
  return -0.5 * s;
}

// LMM families of the propagation kernels (one instantiation each).
enum : int { kFamBdf12 = 0, kFamBdf3 = 1, kFamAm = 2, kFamAb = 3 };

__host__ __device__ constexpr int lmm_family(int lmm) {
  return lmm == PF_LMM_BDF3 ? kFamBdf3 : lmm / 10 == 1 ? kFamAm : lmm / 10 == 2 ? kFamAb : kFamBdf12;
}

// f(t, x) with the input value u = input(t) for forced problems
template <class M>
__device__ __forceinline__ void feval(const typename M::Th& T, double u, const double* x, double* out) {
  M::gf(T, 1.0, x, out);
  if constexpr (M::kForced) out[0] += u;
}

// Psi of Algorithm 1 for one particle over the S substeps of the interval.
// (x, h1, h2) = (x_n, x_{n-1}, x_{n-2}).  With ERR the squared Milne local
// error estimates are summed into E (Step 4b).
//  F = kFamBdf12: BDF1/BDF2 steps (kinds 1, 2).
//  F = kFamBdf3:  BDF1 cold starts and BDF3 steps, whose predictor needs the
//                 slope f(t_n, x_n).
//  F = kFamAm / kFamAb: Adams-Moulton / Adams-Bashforth; the derivative
//                 history f_n, f_{n-1}, f_{n-2} is rebuilt from the stored
//                 states with this particle's theta at the interval's start
//                 and then carried in registers (weights beyond the step's
//                 order are zero, the unused slots hold a finite copy).
template <class M, bool ERR, int F>
__device__ __forceinline__ void propagate(const typename M::Th& T, const StepCoef* sc, int S, int K,
                                          const EpochParams* __restrict__ ep, double (&x)[M::D],
                                          double (&h1)[M::D], double (&h2)[M::D], double (&E)[M::D]) {
  constexpr int D = M::D;
  if constexpr (F == kFamBdf12 || F == kFamBdf3) {
    for (int s = 0; s < S; ++s) {
      const StepCoef& c = sc[s];
      double xp[D], r[D], y[D];
      if (F == kFamBdf3 && c.kind == 3) {
        double fx[D];
        feval<M>(T, c.in0, x, fx);
#pragma unroll
        for (int i = 0; i < D; ++i) {
          xp[i] = fma(c.pi3, fx[i], fma(c.pi2, h2[i], fma(c.pi1, h1[i], c.pi0 * x[i])));
          r[i] = fma(c.rho3, h2[i], fma(c.rho2, h1[i], c.rho1 * x[i]));
          y[i] = xp[i];
        }
      } else if (F == kFamBdf12 && c.kind == 2) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
          xp[i] = fma(c.pi2, h2[i], fma(c.pi1, h1[i], c.pi0 * x[i]));
          r[i] = fma(c.rho2, h1[i], c.rho1 * x[i]);
          y[i] = xp[i];
        }
      } else {
        // BDF1 (cold start): r = x_n, Newton from x_n, error predictor x_n + h f(t_n, x_n)
#pragma unroll
        for (int i = 0; i < D; ++i) {
          r[i] = x[i];
          y[i] = x[i];
        }
        if (ERR) {
          double g[D];
          M::gf(T, c.h, x, g);
          if constexpr (M::kForced) g[0] = fma(c.h, c.in0, g[0]);
#pragma unroll
          for (int i = 0; i < D; ++i) xp[i] = x[i] + g[i];
        }
      }
      if constexpr (M::kForced) r[0] = fma(c.gamma, c.in1, r[0]);
      M::newton(T, c.gamma, r, y, K);
      if (ERR) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
          const double e = c.mu * (y[i] - xp[i]);
          E[i] = fma(e, e, E[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        h2[i] = h1[i];
        h1[i] = x[i];
        x[i] = y[i];
      }
    }
  } else {
    double f0[D], f1[D], f2[D];
    const int q0 = sc[0].kind % 10;
    feval<M>(T, sc[0].in0, x, f0);
    if (q0 >= 2) feval<M>(T, ep->in_hist[0], h1, f1);
    else
#pragma unroll
      for (int i = 0; i < D; ++i) f1[i] = f0[i];
    if (q0 >= 3) feval<M>(T, ep->in_hist[1], h2, f2);
    else
#pragma unroll
      for (int i = 0; i < D; ++i) f2[i] = f1[i];
    for (int s = 0; s < S; ++s) {
      const StepCoef& c = sc[s];
      double xp[D], r[D], y[D], fn[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        xp[i] = fma(c.pi2, f2[i], fma(c.pi1, f1[i], fma(c.pi0, f0[i], x[i])));
        r[i] = fma(c.rho2, f1[i], fma(c.rho1, f0[i], x[i]));
        y[i] = xp[i];
      }
      if constexpr (F == kFamAm) {
        double rr[D];
#pragma unroll
        for (int i = 0; i < D; ++i) rr[i] = r[i];
        if constexpr (M::kForced) rr[0] = fma(c.gamma, c.in1, rr[0]);
        M::newton(T, c.gamma, rr, y, K);
      }
      feval<M>(T, c.in1, y, fn);
      if (ERR) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
          // AM: corrector y against the AB predictor; AB: the AM value at y
          const double e = (F == kFamAm) ? c.mu * (y[i] - xp[i]) : c.mu * (fma(c.gamma, fn[i], r[i]) - y[i]);
          E[i] = fma(e, e, E[i]);
        }
      }
#pragma unroll
      for (int i = 0; i < D; ++i) {
        f2[i] = f1[i];
        f1[i] = f0[i];
        f0[i] = fn[i];
        h2[i] = h1[i];
        h1[i] = x[i];
        x[i] = y[i];
      }
    }
  }
}

// ------------------------------------------------------------------ init
// Step 1: phi drawn from the prior (uniform or log-uniform per component,
// Philox purpose INIT, epoch word 0), x = h1 = h2 = x0, unnormalised log
// weight 0 (w = 1/N after normalisation), into the pending buffer.
template <int D, int P>
__device__ __forceinline__ void init_body(const FilterDev& fd, int vb) {
  const Ctrl* ctrl = fd.ctrl;
  const Ensemble dst = pending(fd, ctrl->cur);
  const int64_t N = fd.N;
  const int64_t n = (int64_t)vb * blockDim.x + threadIdx.x;
  if (n >= N) return;
#pragma unroll
  for (int b = 0; b < (P + 1) / 2; ++b) {
    const U4 w = draw_block(fd, kRngInit, (uint32_t)n, 0u, (uint32_t)b);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * b + h;
      if (i >= P) break;
      const double u = h == 0 ? uniform53(w.x, w.y) : uniform53(w.z, w.w);
      double phi;
      if (fd.prior_kind[i] == PF_PRIOR_LOGUNIFORM) {
        const double lo = log(fd.prior_lo[i]), hi = log(fd.prior_hi[i]);
        const double lphi = lo + u * (hi - lo);
        phi = (fd.transform == PF_TRANSFORM_LOG) ? lphi : exp(lphi);
      } else {
        const double th = fd.prior_lo[i] + u * (fd.prior_hi[i] - fd.prior_lo[i]);
        phi = (fd.transform == PF_TRANSFORM_LOG) ? log(th) : th;
      }
      dst.phi[i * N + n] = phi;
    }
  }
  const int dd = D > 0 ? D : fd.d;  // D = 0: the state dimension is a runtime choice
  for (int i = 0; i < dd; ++i) {
    const double v = fd.x0[i];
    dst.x[i * N + n] = v;
    dst.h1[i * N + n] = v;
    dst.h2[i * N + n] = v;
  }
  dst.lw[n] = 0.0;
}

// ---------------------------------------------------------------- stage 1
template <class M, int F>
__device__ __forceinline__ void stage1_body(const FilterDev& fd, const EpochParams* __restrict__ ep,
                                            int vb, int vg, const StepCoef* s_sc, double* s_red,
                                            int* s_flag) {
  constexpr int D = M::D, P = M::P;
  const Ctrl* ctrl = fd.ctrl;
  const int S = ep->S;
  const Ensemble E = committed(fd, ctrl->cur);
  const int64_t N = fd.N;
  const int64_t n = (int64_t)vb * blockDim.x + threadIdx.x;
  double lg = -CUDART_INF;
  if (n < N) {
    double ph[P], th[P];
#pragma unroll
    for (int i = 0; i < P; ++i) ph[i] = fd.a * E.phi[i * N + n] + (1.0 - fd.a) * ctrl->phibar[i];
    to_theta<P>(fd, ph, th);
    const typename M::Th T = M::theta(th);
    double x[D], h1[D], h2[D], Eunused[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      x[i] = E.x[i * N + n];
      h1[i] = E.h1[i * N + n];
      h2[i] = E.h2[i * N + n];
    }
    propagate<M, false, F>(T, s_sc, S, fd.K, ep, x, h1, h2, Eunused);
    const double ll = loglik<D>(fd, ep, x);
    fd.ll1[n] = ll;
    lg = (E.lw[n] - ctrl->logW) + ll;
    if (!finite_bits(lg)) lg = -CUDART_INF;
    fd.lg[n] = lg;
  }
  pdl_trigger();
  stage1_tail(fd, ep->epoch, lg, vb, vg, s_red, s_flag);
}

// ------------------------------------------------------------------- scan
// Step 3a/3b's cumulative weights: scan_tile_core (pf_scan.cuh) on the
// filter's buffers; the shift M is lg_max.  c keeps the tile-local sums, and
// its readers apply the tile offsets and floors (CumTiles).
__device__ __forceinline__ ScanArgs scan_args(const FilterDev& fd) {
  Ctrl* ctrl = fd.ctrl;
  return ScanArgs{fd.lg, fd.N, fd.Ntile, fd.sms, ctrl->lg_max, fd.c, fd.blk, fd.boff, fd.pmax,
                  fd.ticket + 1, &ctrl->c_total};
}

__device__ __forceinline__ void scan_tile_body(const FilterDev& fd, int vb, int vg, double* s_warp,
                                               int* s_flag) {
  scan_tile_core(scan_args(fd), vb, vg, s_warp, s_flag);
}


// --------------------------------------------------------------- resample
// Step 3b: the epoch's u is Philox purpose RESAMPLE, slot 0; the search is
// resample_tile (pf_scan.cuh).
// The filter's cumulative weights as the tile pass leaves them: the offsets
// and floors are applied on read (no separate offset pass over c).
__device__ __forceinline__ CumTiles cum_tiles(const FilterDev& fd) {
  return CumTiles{fd.c, fd.boff, fd.pmax, (uint32_t)scan_tile_len(fd.Ntile, fd.sms)};
}

__device__ __forceinline__ double resample_u(const FilterDev& fd, const EpochParams* __restrict__ ep) {
  const U4 w = draw_block(fd, kRngResample, 0u, ep->epoch, 0u);
  return uniform53(w.x, w.y);
}

// corners: the filter's corner array (two-phase, in the per-block scratch,
// which holds nothing else between the scan and stage 2), or null
__device__ __forceinline__ void resample_body(const FilterDev& fd, const EpochParams* __restrict__ ep,
                                              int vb, RsShared& sh, double* s_chol,
                                              const int32_t* corners) {
  // warp 2 of the first block factors C for stage 2 (warps 0 and 1 search)
  if (vb == 0 && (threadIdx.x >> 5) == 2) factor_covariance(fd, fd.p, s_chol, threadIdx.x & 31);
  // u is drawn by the two warps that use it (resample_tile)
  const double u = threadIdx.x < 64 ? resample_u(fd, ep) : 0.0;
  resample_tile(cum_tiles(fd), fd.N, u, fd.idx,
                reinterpret_cast<unsigned long long*>(&fd.ctrl->n_unique), vb, sh, corners);
}

// ---------------------------------------------------------------- stage 2
template <class M, int F>
__device__ __forceinline__ void stage2_body(const FilterDev& fd, const EpochParams* __restrict__ ep,
                                            int vb, int vg, const StepCoef* s_sc, double* s_red,
                                            int* s_flag) {
  constexpr int D = M::D, P = M::P;
  const Ctrl* ctrl = fd.ctrl;
  const int S = ep->S;
  const int cur = ctrl->cur;
  const Ensemble src = committed(fd, cur);
  const Ensemble dst = pending(fd, cur);
  const int64_t N = fd.N;
  const uint32_t epoch = ep->epoch;
  const int64_t n = (int64_t)vb * blockDim.x + threadIdx.x;
  double lwn = -CUDART_INF;
  double bad = 0.0;
  if (n < N) {
    const int64_t l = fd.idx[n];
    // 4a: phi_{j+1} = (a phi^l + (1 - a) phibar) + s L z
    double z[P + 1];
#pragma unroll
    for (int b = 0; b < (P + 1) / 2; ++b) {
      const U4 w = draw_block(fd, kRngTheta, (uint32_t)n, epoch, (uint32_t)b);
      normal_pair(w, z[2 * b], z[2 * b + 1]);
    }
    double ph[P], th[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      double lz = 0.0;
#pragma unroll
      for (int k = 0; k <= i; ++k) lz = fma(ctrl->L[i * kPMax + k], z[k], lz);
      const double shr = fd.a * src.phi[i * N + l] + (1.0 - fd.a) * ctrl->phibar[i];
      ph[i] = fma(fd.s, lz, shr);
    }
    to_theta<P>(fd, ph, th);
    const typename M::Th T = M::theta(th);
    double x[D], h1[D], h2[D], Eacc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      x[i] = src.x[i * N + l];
      h1[i] = src.h1[i * N + l];
      h2[i] = src.h2[i * N + l];
      Eacc[i] = 0.0;
    }
    // 4b, 4d: repropagate, summing the squared Milne estimates
    propagate<M, true, F>(T, s_sc, S, fd.K, ep, x, h1, h2, Eacc);
    // 4c, 4d: v ~ N(0, kappa diag(E)), added to x and to the stored history
#pragma unroll
    for (int b = 0; b < (D + 1) / 2; ++b) {
      const U4 w = draw_block(fd, kRngInnov, (uint32_t)n, epoch, (uint32_t)b);
      double z0, z1;
      normal_pair(w, z0, z1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * b + h;
        if (i < D) {
          const double v = sqrt(fd.kappa * Eacc[i]) * (h == 0 ? z0 : z1);
          x[i] += v;
          h1[i] += v;
          h2[i] += v;
        }
      }
    }
    // 5: log w = log pi(y | x_{j+1}) - log pi(y | xbar^l)
    const double ll2 = loglik<D>(fd, ep, x);
    lwn = ll2 - fd.ll1[l];
    if (!finite_bits(lwn)) {
      lwn = -CUDART_INF;
      bad = 1.0;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
      dst.x[i * N + n] = x[i];
      dst.h1[i * N + n] = h1[i];
      dst.h2[i * N + n] = h2[i];
    }
#pragma unroll
    for (int i = 0; i < P; ++i) dst.phi[i * N + n] = ph[i];
    dst.lw[n] = lwn;
  }
  pdl_trigger();
  stage2_tail(fd, epoch, lwn, bad, vb, vg, s_red, s_flag);
}

// ---------------------------------------------------------------- moments
// Weighted sums of the pending buffer with e_n = exp(lw_n - max lw):
//   [S0 = sum e, Sw2 = sum e^2, S1 = sum e phi, S2 = sum e (phi - c)(phi - c)^T
//    (upper triangle, shift c = the committed mean), Sx = sum e x]
// Zero-weight particles are skipped (their state may be non-finite).  The
// filter's last block reduces the partial records and commits the epoch.
template <int D, int P>
struct MomentLayout {
  static constexpr int kS0 = 0, kW2 = 1, kS1 = 2, kS2 = 2 + P, kSx = kS2 + P * (P + 1) / 2,
                       kN = kSx + D;
};

// Warp sums of a vector of N values by reduce-scatter.  A butterfly per value
// costs 5 N FP64 adds a lane; here each exchange halves the vector instead (a
// lane keeps one half and adds the partner's copy of it), so the adds are
// about N + 5 a lane, which matters where FP64 instructions are scarce.  On
// the last exchange each lane holds the warp totals of positions [lo, lo + N)
// of the original vector, of which the first cnt are real (the rest padding);
// lanes that are copies of a partner (the vector had one value left) write
// nothing.  The order of additions depends only on the lane layout.
template <int N, int O>
struct WarpScatter {
  __device__ __forceinline__ static void run(const double (&v)[N], int lane, int lo, int cnt, bool dup,
                                             double* out) {
    if constexpr (O == 0) {
      if (!dup) {
#pragma unroll
        for (int k = 0; k < N; ++k)
          if (k < cnt) out[lo + k] = v[k];
      }
    } else if constexpr (N == 1) {
      const double a[1] = {v[0] + __shfl_xor_sync(0xffffffffu, v[0], O)};
      WarpScatter<1, O / 2>::run(a, lane, lo, cnt, dup || (lane & O) != 0, out);
    } else {
      constexpr int H = (N + 1) / 2;
      const bool up = (lane & O) != 0;
      double a[H];
#pragma unroll
      for (int k = 0; k < H; ++k) {
        const double lv = v[k];
        const double hv = (H + k < N) ? v[H + k] : 0.0;
        a[k] = (up ? hv : lv) + __shfl_xor_sync(0xffffffffu, up ? lv : hv, O);
      }
      // lower lanes keep positions [0, H), upper lanes [H, 2H)
      const int ncnt = up ? (cnt > H ? cnt - H : 0) : (cnt < H ? cnt : H);
      WarpScatter<H, O / 2>::run(a, lane, up ? lo + H : lo, ncnt, dup, out);
    }
  }
};

// shared scratch of the moment kernels: 8 warp rows of NV values, or the
// group sums of the last block (at most kMomentThreads values)
template <int NV>
constexpr int kMomentShared = (kMomentThreads / 32) * NV > kMomentThreads ? (kMomentThreads / 32) * NV
                                                                         : kMomentThreads;

// Sum each of NV per-thread values over the block: warp reduce-scatter into
// one row per warp in shared memory, then NV threads add the rows.  out[k]
// (shared or global) receives the totals; s_part needs 8 * NV doubles.
template <int NV>
__device__ __forceinline__ void block_sum_vec(double (&acc)[NV], double* s_part, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  WarpScatter<NV, 16>::run(acc, lane, 0, NV, false, s_part + wid * NV);
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += s_part[w * NV + k];
    out[k] = t;
  }
  __syncthreads();
}

template <int D, int P>
__device__ __forceinline__ void moments_commit(const FilterDev& fd, int is_init, const double* s_tot,
                                               double* s_part, int* s_flag);

template <int D, int P>
__device__ __forceinline__ void moments_body(const FilterDev& fd, int is_init, int vb, int vg,
                                             double* s_part, double* s_tot, int* s_flag) {
  using Lay = MomentLayout<D, P>;
  constexpr int NV = Lay::kN;
  Ctrl* ctrl = fd.ctrl;
  const int cur = ctrl->cur;
  const Ensemble nw = pending(fd, cur);
  const int64_t N = fd.N;
  const double M = ctrl->lw_max;
  double c[P];
#pragma unroll
  for (int i = 0; i < P; ++i) c[i] = ctrl->phibar[i];
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  for (int64_t n = (int64_t)vb * blockDim.x + threadIdx.x; n < N; n += (int64_t)vg * blockDim.x) {
    const double lw = nw.lw[n];
    if (is_neg_inf(lw)) {
      if constexpr (D == 0) fd.wk[n] = 0.0;
      continue;
    }
    const double e = exp(lw - M);
    if constexpr (D == 0) fd.wk[n] = e;  // the weights x-bar needs (k_xbar)
    acc[Lay::kS0] += e;
    acc[Lay::kW2] = fma(e, e, acc[Lay::kW2]);
    double dp[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
      dp[i] = nw.phi[i * N + n] - c[i];
      acc[Lay::kS1 + i] = fma(e, dp[i], acc[Lay::kS1 + i]);
    }
    int q = Lay::kS2;
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const double di = e * dp[i];
#pragma unroll
      for (int j = i; j < P; ++j) {
        acc[q] = fma(di, dp[j], acc[q]);
        ++q;
      }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) acc[Lay::kSx + i] = fma(e, nw.x[i * N + n], acc[Lay::kSx + i]);
  }
  block_sum_vec<NV>(acc, s_part, fd.part + (int64_t)vb * fd.nrec);
  pdl_trigger();
  if (!elect_last_block(fd.ticket + 3, s_flag, (unsigned)vg)) return;
  // the vg partial records: thread (j, k) adds value k of records j, j + G,
  // ... (G groups of NV threads; loads issued eight at a time), then NV
  // threads add the G group sums
  const int G = (int)blockDim.x / NV;
  if ((int)threadIdx.x < G * NV) {
    const int k = threadIdx.x % NV, j = threadIdx.x / NV;
    double t = 0.0;
    for (int b0 = j; b0 < vg; b0 += 8 * G) {
      double x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int b = b0 + q * G;
        x[q] = b < vg ? __ldcg(fd.part + (int64_t)b * fd.nrec + k) : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) t += x[q];
    }
    s_part[j * NV + k] = t;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NV; k += blockDim.x) {
    double t = 0.0;
    for (int j = 0; j < G; ++j) t += s_part[j * NV + k];
    s_tot[k] = t;
  }
  __syncthreads();
  if (fd.shard_sums) {
    // a shard: its sums are one part of the global ones, which the commit
    // takes (moments_commit, after the caller has added every shard's)
    for (int k = threadIdx.x; k < NV; k += blockDim.x) fd.shard_sums[k] = s_tot[k];
    return;
  }
  moments_commit<D, P>(fd, is_init, s_tot, s_part, s_flag);
}

// The commit of Step 6 from the weighted sums s_tot (shared memory) of the
// pending buffer: every thread of one block calls it.
template <int D, int P>
__device__ __forceinline__ void moments_commit(const FilterDev& fd, int is_init, const double* s_tot,
                                               double* s_part, int* s_flag) {
  using Lay = MomentLayout<D, P>;
  Ctrl* ctrl = fd.ctrl;
  const int cur = ctrl->cur;
  const double M = ctrl->lw_max;
  // The commit.  Moments about the shift c (the previous mean): the first
  // moment of the differences gives the mean's displacement to full relative
  // precision, so C = E[(phi - c)(phi - c)^T] - m m^T loses only
  // eps E[|phi - c|^2].  Warp 0 forms the mean and C a lane per entry and
  // checks them; then, at once, warp 0 stores them, warp 1 the weight
  // statistics and warp 2 the state mean.
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const double S0 = s_tot[Lay::kS0];
  double* s_m1 = s_part;                // P values
  double* s_C = s_part + kPMax;         // kPMax^2 values
  constexpr int NC = P * (P + 1) / 2;
  if (wid == 0) {
    const double inv = 1.0 / S0;
    bool bad = !(S0 > 0.0);
    if (lane < kPMax * kPMax) s_C[lane] = 0.0;
    if (lane < P) {
      const double m1 = s_tot[Lay::kS1 + lane] * inv;
      s_m1[lane] = m1;
      bad = bad || !finite_bits(ctrl->phibar[lane] + m1);
    }
    __syncwarp();
    if (lane < NC) {
      int i = 0, r = lane;
      while (r >= P - i) {
        r -= P - i;
        ++i;
      }
      const int j = i + r;
      const double v = s_tot[Lay::kS2 + lane] * inv - s_m1[i] * s_m1[j];
      s_C[i * kPMax + j] = v;
      s_C[j * kPMax + i] = v;
      bad = bad || !finite_bits(v);
    }
    bad = __any_sync(0xffffffffu, bad);
    if (lane == 0) *s_flag = bad ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag) {
    if (threadIdx.x == 0) {
      ctrl->status = PF_ERR_NUMERIC;
      ctrl->failed_epoch = ctrl->epochs_done;
    }
    return;
  }
  if (wid == 0) {
    // (L, the factor of C, is formed by the next resampling launch)
    if (lane < kPMax * kPMax) ctrl->C[lane] = s_C[lane];
    if (lane < P) ctrl->phibar[lane] += s_m1[lane];
  } else if (wid == 1) {
    if (lane == 0) {
      ctrl->wsum = S0;
      ctrl->ess = S0 * S0 / s_tot[Lay::kW2];
      ctrl->logW = M + log(S0);
      ctrl->cur = 1 - cur;
      if (!is_init) ctrl->epochs_done += 1;
    }
  } else if (wid == 2) {
    const double inv = 1.0 / S0;
    for (int i = lane; i < D; i += 32) fd.xbar[i] = s_tot[Lay::kSx + i] * inv;
  }
}

// ========================================================= single filter
template <int D, int P>
__global__ void __launch_bounds__(kInitThreads) k_init(const __grid_constant__ FilterDev fd) {
  init_body<D, P>(fd, blockIdx.x);
}

template <class M, int F>
__global__ void __launch_bounds__(kSmallThreads) k_stage1(const __grid_constant__ FilterDev fd,
                                                          const EpochParams* __restrict__ ep) {
  extern __shared__ double s_dyn[];
  __shared__ double s_red[32];
  __shared__ int s_flag;
  // the parameter block is written only by copies before the epoch's first
  // launch, so its substep table is staged before the wait
  StepCoef* s_sc = reinterpret_cast<StepCoef*>(s_dyn);
  load_steps(s_sc, ep, ep->S);
  pdl_wait();
  if (fd.ctrl->status != PF_OK) return;
  stage1_body<M, F>(fd, ep, blockIdx.x, gridDim.x, s_sc, s_red, &s_flag);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tile(const __grid_constant__ FilterDev fd) {
  __shared__ double s_warp[33];
  __shared__ int s_flag;
  pdl_wait();
  if (fd.ctrl->status != PF_OK) return;
  scan_tile_body(fd, blockIdx.x, gridDim.x, s_warp, &s_flag);
}

// Two-phase resampling of a large ensemble: every tile corner, one warp each,
// into the per-block scratch.
__global__ void __launch_bounds__(256) k_rs_corners(const __grid_constant__ FilterDev fd,
                                                   const EpochParams* __restrict__ ep) {
  pdl_wait();
  if (fd.ctrl->status != PF_OK) return;
  rs_corners_core(cum_tiles(fd), fd.N, resample_u(fd, ep),
                  ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, reinterpret_cast<int32_t*>(fd.blk));
}

__global__ void __launch_bounds__(kResampleThreads, 4) k_resample(const __grid_constant__ FilterDev fd,
                                                               const EpochParams* __restrict__ ep) {
  __shared__ RsShared sh;
  __shared__ double s_chol[kPMax * kPMax];
  pdl_wait();
  if (fd.ctrl->status != PF_OK) return;
  const int32_t* corners = rs_two_phase(fd.N, fd.sms) ? reinterpret_cast<const int32_t*>(fd.blk) : nullptr;
  resample_body(fd, ep, blockIdx.x, sh, s_chol, corners);
}

template <class M, int F>
__global__ void __launch_bounds__(kSmallThreads) k_stage2(const __grid_constant__ FilterDev fd,
                                                          const EpochParams* __restrict__ ep) {
  extern __shared__ double s_dyn[];
  __shared__ double s_red[32];
  __shared__ int s_flag;
  StepCoef* s_sc = reinterpret_cast<StepCoef*>(s_dyn);
  load_steps(s_sc, ep, ep->S);
  pdl_wait();
  if (fd.ctrl->status != PF_OK) return;
  stage2_body<M, F>(fd, ep, blockIdx.x, gridDim.x, s_sc, s_red, &s_flag);
}

template <int D, int P>
__global__ void __launch_bounds__(kMomentThreads) k_moments(const __grid_constant__ FilterDev fd,
                                                            int is_init) {
  constexpr int NV = MomentLayout<D, P>::kN;
  __shared__ double s_part[kMomentShared<NV>];
  __shared__ double s_tot[NV];
  __shared__ int s_flag;
  pdl_wait();
  if (fd.ctrl->status != PF_OK) return;
  moments_body<D, P>(fd, is_init, blockIdx.x, gridDim.x, s_part, s_tot, &s_flag);
}

// Weighted mean of theta = exp(phi) (or phi) of the committed ensemble, for
// pf_stats only: w_n = exp(lw_n - logW).  One block, off the epoch path.
template <int P>
__global__ void __launch_bounds__(kMomentThreads) k_theta_mean(const __grid_constant__ FilterDev fd) {
  __shared__ double s_part[(kMomentThreads / 32) * P];
  __shared__ double s_tot[P];
  Ctrl* ctrl = fd.ctrl;
  const Ensemble E = committed(fd, ctrl->cur);
  const int64_t N = fd.N;
  const double lW = ctrl->logW;
  double acc[P];
#pragma unroll
  for (int i = 0; i < P; ++i) acc[i] = 0.0;
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const double lw = E.lw[n];
    if (is_neg_inf(lw)) continue;
    const double w = exp(lw - lW);
#pragma unroll
    for (int i = 0; i < P; ++i) {
      const double ph = E.phi[i * N + n];
      acc[i] = fma(w, (fd.transform == PF_TRANSFORM_LOG) ? exp(ph) : ph, acc[i]);
    }
  }
  block_sum_vec<P>(acc, s_part, s_tot);
  if (threadIdx.x < P) ctrl->theta_mean[threadIdx.x] = s_tot[threadIdx.x];
}

// The ESS of the last epoch's first-stage weights for pf_stats (on demand,
// off the epoch): sum g^2 with g = exp(lg - lg_max) formed as the scan forms
// it, block partials into the per-block scratch, the last block adds them.
__global__ void __launch_bounds__(kMomentThreads) k_stage1_ess(const __grid_constant__ FilterDev fd) {
  __shared__ double s_red[32];
  __shared__ int s_flag;
  const double M = fd.ctrl->lg_max;
  double sq = 0.0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < fd.N;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double g = scan_weight(fd.lg[k], M);
    sq = fma(g, g, sq);
  }
  sq = block_sum(sq, s_red);
  if (threadIdx.x == 0) fd.tsq[blockIdx.x] = sq;
  if (elect_last_block(fd.ticket + 4, &s_flag, gridDim.x)) {
    double q = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) q += __ldcg(fd.tsq + b);
    q = block_sum(q, s_red);
    if (threadIdx.x == 0) fd.ctrl->g_sq = q;
  }
}

cudaError_t launch_stage1_ess(const FilterDev& fd, cudaStream_t st) {
  k_stage1_ess<<<moment_blocks(fd.N, fd.sms), kMomentThreads, 0, st>>>(fd);
  return cudaGetLastError();
}

__global__ void k_set_moments(const __grid_constant__ FilterDev fd) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double L[kPMax * kPMax];
  cholesky_psd(fd.p, fd.ctrl->C, L);
  for (int i = 0; i < kPMax * kPMax; ++i) fd.ctrl->L[i] = L[i];
}

// Weighted mean of x for states too large for the per-thread moment records
// (D = 0 moments): one block per component row of the newly committed
// ensemble, w_n = e_n / wsum with the weights e_n = exp(lw_n - lw_max) the
// moment kernel stored (zero-weight particles, whose state may be
// non-finite, are skipped by the bit pattern of their 0).
__global__ void __launch_bounds__(kMomentThreads) k_xbar(const __grid_constant__ FilterDev fd) {
  __shared__ double s_red[32];
  const Ctrl* ctrl = fd.ctrl;
  if (ctrl->status != PF_OK) return;
  const Ensemble E = committed(fd, ctrl->cur);
  const int64_t N = fd.N;
  const double* __restrict__ e = fd.wk;
  for (int i = blockIdx.x; i < fd.d; i += gridDim.x) {
    const double* xi = E.x + (int64_t)i * N;
    double acc = 0.0;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
      const double en = __ldg(e + n);
      if (__double_as_longlong(en) != 0) acc = fma(en, xi[n], acc);
    }
    acc = block_sum(acc, s_red);
    if (threadIdx.x == 0) fd.xbar[i] = acc / ctrl->wsum;
    __syncthreads();
  }
}

// ========================================================= batch of filters
// Every batched launch reads its block's (filter, virtual block) from a tile
// table and the filter's descriptor through a read-only pointer.  Tiles of
// different filters share a launch; the phases of one filter are ordered by
// the launches of the stream.  Stage kernels are per model, so each keeps the
// register budget of its own model.
__global__ void __launch_bounds__(kInitThreads) k_batch_init(const FilterDev* __restrict__ fds,
                                                           const BatchTile* __restrict__ tiles) {
  const BatchTile t = tiles[blockIdx.x];
  const FilterDev& fd = *(fds + t.f);
  switch (fd.ode) {
    case PF_ODE_LINEAR2: init_body<2, 2>(fd, t.vb); break;
    case PF_ODE_ROBERTSON: init_body<3, 3>(fd, t.vb); break;
    case PF_ODE_BRUSSELATOR1D: init_body<64, 3>(fd, t.vb); break;
    case PF_ODE_MICHAELIS3: init_body<3, 4>(fd, t.vb); break;
  }
}

template <class M, int STAGE, int F>
__global__ void __launch_bounds__(kSmallThreads) k_batch_stage(const FilterDev* __restrict__ fds,
                                                             const EpochParams* const* __restrict__ eps,
                                                             const BatchTile* __restrict__ tiles) {
  extern __shared__ double s_dyn[];
  __shared__ double s_red[32];
  __shared__ int s_flag;
  const BatchTile t = tiles[blockIdx.x];
  const FilterDev& fd = *(fds + t.f);
  if (fd.ctrl->status != PF_OK) return;
  const EpochParams* ep = eps[t.f];
  StepCoef* s_sc = reinterpret_cast<StepCoef*>(s_dyn);
  load_steps(s_sc, ep, ep->S);
  const int vg = (int)((fd.N + kSmallThreads - 1) / kSmallThreads);
  if (STAGE == 1) stage1_body<M, F>(fd, ep, t.vb, vg, s_sc, s_red, &s_flag);
  else stage2_body<M, F>(fd, ep, t.vb, vg, s_sc, s_red, &s_flag);
}

__global__ void __launch_bounds__(kScanThreads) k_batch_scan_tile(const FilterDev* __restrict__ fds,
                                                                const BatchTile* __restrict__ tiles) {
  __shared__ double s_warp[33];
  __shared__ int s_flag;
  const BatchTile t = tiles[blockIdx.x];
  const FilterDev& fd = *(fds + t.f);
  if (fd.ctrl->status != PF_OK) return;
  scan_tile_body(fd, t.vb, scan_tile_count(fd.N, fd.sms), s_warp, &s_flag);
}

__global__ void __launch_bounds__(kResampleThreads) k_batch_resample(
    const FilterDev* __restrict__ fds, const EpochParams* const* __restrict__ eps,
    const BatchTile* __restrict__ tiles) {
  __shared__ RsShared sh;
  __shared__ double s_chol[kPMax * kPMax];
  const BatchTile t = tiles[blockIdx.x];
  const FilterDev& fd = *(fds + t.f);
  if (fd.ctrl->status != PF_OK) return;
  resample_body(fd, eps[t.f], t.vb, sh, s_chol, nullptr);
}

template <int D, int P>
__global__ void __launch_bounds__(kMomentThreads) k_batch_moments(const FilterDev* __restrict__ fds,
                                                                const BatchTile* __restrict__ tiles,
                                                                int is_init) {
  constexpr int NV = MomentLayout<D, P>::kN;
  __shared__ double s_part[kMomentShared<NV>];
  __shared__ double s_tot[NV];
  __shared__ int s_flag;
  const BatchTile t = tiles[blockIdx.x];
  const FilterDev& fd = *(fds + t.f);
  if (fd.ctrl->status != PF_OK) return;
  const int vg = moment_blocks(fd.N, fd.sms);
  moments_body<D, P>(fd, is_init, t.vb, vg, s_part, s_tot, &s_flag);
}

// ----------------------------------------------------------------- launch
template <int D, int P>
static int moment_nrec() {
  return MomentLayout<D, P>::kN;
}

int moment_record_size(int ode) {
  switch (ode) {
    case PF_ODE_LINEAR2: return moment_nrec<2, 2>();
    case PF_ODE_ROBERTSON: return moment_nrec<3, 3>();
    case PF_ODE_BRUSSELATOR1D: return moment_nrec<64, 3>();
    case PF_ODE_ADVDIFF2D: return moment_nrec<0, 5>();
    case PF_ODE_MICHAELIS3: return moment_nrec<3, 4>();
  }
  return -1;
}

int max_grid_blocks(int64_t N, int sms) {
  const int64_t a = N;  // at least as many as any stage launch (one block per particle for M2)
  const int64_t b = scan_tile_count(N, sms);
  const int64_t c = (2 * N + kRsTile - 1) / kRsTile;
  int64_t m = a > b ? a : b;
  m = m > c ? m : c;
  const int mb = moment_blocks_max(sms);
  return (int)(m > mb ? m : mb);
}

int scan_tiles(int64_t N, int sms) { return scan_tile_count(N, sms); }

// Threads per block of a filter's own stage launches (a batch's tiles are
// always kSmallThreads): 128, halved (down to one warp) while the filter has
// fewer than 6 such blocks an SM.  The stage kernels are FP64-issue bound and
// their particles all cost the same, so a launch ends with the SMs that hold
// one block more than the others: 2.6 blocks of 128 an SM (M1, N = 50000) lose
// 1.7 % of the epoch against 10.3 blocks of 32.  The blocks only reduce a
// maximum and a count, so the results do not depend on the block size.
static int stage_threads(int64_t N, int sms) {
  int t = kSmallThreads;
  while (t > 32 && N < (int64_t)6 * t * sms) t >>= 1;
  return t;
}

static unsigned stage_grid(int64_t N, int sms) {
  const int t = stage_threads(N, sms);
  return (unsigned)((N + t - 1) / t);
}

int phase_blocks(int phase, int ode, int64_t N, int sms) {
  switch (phase) {
    case kPhaseInit: return (int)((N + kInitThreads - 1) / kInitThreads);
    case kPhaseStage1:
    case kPhaseStage2:
      if (ode == PF_ODE_ADVDIFF2D) return (int)N;
      return ode == PF_ODE_BRUSSELATOR1D ? bruss_stage_blocks(N)
                                         : (int)((N + kSmallThreads - 1) / kSmallThreads);
    case kPhaseScanTile: return scan_tiles(N, sms);
    case kPhaseResample: return (int)rs_tiles(N);
    case kPhaseMoments: return moment_blocks(N, sms);
  }
  return 0;
}

template <class M>
static cudaError_t launch_init_t(const FilterDev& fd, cudaStream_t st) {
  const int64_t N = fd.N;
  k_init<M::D, M::P><<<phase_blocks(kPhaseInit, M::ODE, N, fd.sms), kInitThreads, 0, st>>>(fd);
  k_moments<M::D, M::P><<<phase_blocks(kPhaseMoments, M::ODE, N, fd.sms), kMomentThreads, 0, st>>>(fd, 1);
  return cudaGetLastError();
}

using StageKernel = void (*)(const FilterDev, const EpochParams*);

// the stage kernels of model M for the filter's LMM family
template <class M>
static void stage_kernels(int lmm, StageKernel& k1, StageKernel& k2) {
  switch (lmm_family(lmm)) {
    case kFamBdf3: k1 = k_stage1<M, kFamBdf3>; k2 = k_stage2<M, kFamBdf3>; return;
    case kFamAm: k1 = k_stage1<M, kFamAm>; k2 = k_stage2<M, kFamAm>; return;
    case kFamAb: k1 = k_stage1<M, kFamAb>; k2 = k_stage2<M, kFamAb>; return;
  }
  k1 = k_stage1<M, kFamBdf12>;
  k2 = k_stage2<M, kFamBdf12>;
}

using BatchStageKernel = void (*)(const FilterDev*, const EpochParams* const*, const BatchTile*);

// the batched stage kernels of model M for an LMM family
template <class M>
static void batch_stage_kernels(int lmm, BatchStageKernel& k1, BatchStageKernel& k2) {
  switch (lmm_family(lmm)) {
    case kFamBdf3: k1 = k_batch_stage<M, 1, kFamBdf3>; k2 = k_batch_stage<M, 2, kFamBdf3>; return;
    case kFamAm: k1 = k_batch_stage<M, 1, kFamAm>; k2 = k_batch_stage<M, 2, kFamAm>; return;
    case kFamAb: k1 = k_batch_stage<M, 1, kFamAb>; k2 = k_batch_stage<M, 2, kFamAb>; return;
  }
  k1 = k_batch_stage<M, 1, kFamBdf12>;
  k2 = k_batch_stage<M, 2, kFamBdf12>;
}

// Launch kernel k on st with programmatic stream serialization: its blocks may
// be scheduled while the stream's previous kernel drains, and the kernel's
// pdl_wait() orders its accesses after that kernel's.
template <typename... P, typename... A>
static cudaError_t launch_pdl(void (*k)(P...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t st, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

template <class M>
static cudaError_t launch_epoch_t(const FilterDev& fd, const EpochParams* ep, int S,
                                  cudaStream_t st, cudaEvent_t* marks) {
  const int64_t N = fd.N;
  const size_t smem = (size_t)S * sizeof(StepCoef);
  StageKernel k1, k2;
  stage_kernels<M>(fd.lmm, k1, k2);
  const unsigned g_small = stage_grid(N, fd.sms);
  const int t_small = stage_threads(N, fd.sms);
  auto mark = [&](int i) {
    if (marks && marks[i]) cudaEventRecord(marks[i], st);
  };
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  mark(0);
  ok(launch_pdl(k1, g_small, t_small, smem, st, fd, ep));
  mark(1);
  ok(launch_pdl(k_scan_tile, (unsigned)phase_blocks(kPhaseScanTile, M::ODE, N, fd.sms), kScanThreads, 0,
                st, fd));
  mark(2);  // (marks[3] is not recorded: the scan_add slot is empty)
  if (rs_two_phase(N, fd.sms)) ok(launch_pdl(k_rs_corners, (unsigned)rs_corner_blocks(N), 256, 0, st, fd, ep));
  ok(launch_pdl(k_resample, (unsigned)phase_blocks(kPhaseResample, M::ODE, N, fd.sms), kResampleThreads, 0,
                st, fd, ep));
  mark(4);
  ok(launch_pdl(k2, g_small, t_small, smem, st, fd, ep));
  mark(5);
  ok(launch_pdl(k_moments<M::D, M::P>, (unsigned)phase_blocks(kPhaseMoments, M::ODE, N, fd.sms),
                kMomentThreads, 0, st, fd, 0));
  mark(6);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// the Brusselator's stage kernels live in pf_bruss.cu; the rest is shared
static cudaError_t launch_epoch_bruss(const FilterDev& fd, const EpochParams* ep, int S,
                                      cudaStream_t st, cudaEvent_t* marks) {
  const int64_t N = fd.N;
  const int ode = PF_ODE_BRUSSELATOR1D;
  auto mark = [&](int i) {
    if (marks && marks[i]) cudaEventRecord(marks[i], st);
  };
  cudaError_t e;
  mark(0);
  if ((e = launch_bruss_stage(1, fd, ep, S, st)) != cudaSuccess) return e;
  mark(1);
  k_scan_tile<<<(unsigned)phase_blocks(kPhaseScanTile, ode, N, fd.sms), kScanThreads, 0, st>>>(fd);
  mark(2);  // (marks[3] is not recorded: the scan_add slot is empty)
  if (rs_two_phase(N, fd.sms)) k_rs_corners<<<rs_corner_blocks(N), 256, 0, st>>>(fd, ep);
  k_resample<<<(unsigned)phase_blocks(kPhaseResample, ode, N, fd.sms), kResampleThreads, 0, st>>>(fd, ep);
  mark(4);
  if ((e = launch_bruss_stage(2, fd, ep, S, st)) != cudaSuccess) return e;
  mark(5);
  k_moments<64, 3><<<phase_blocks(kPhaseMoments, ode, N, fd.sms), kMomentThreads, 0, st>>>(fd, 0);
  mark(6);
  return cudaGetLastError();
}

// M2: the stage kernels live in pf_advdiff.cu; the moments take the D = 0
// record and x-bar its own kernel
static int xbar_blocks(const FilterDev& fd) { return fd.d < 1024 ? fd.d : 1024; }

static cudaError_t launch_epoch_ad(const FilterDev& fd, const EpochParams* ep, int S,
                                   cudaStream_t st, cudaEvent_t* marks) {
  const int64_t N = fd.N;
  const int ode = PF_ODE_ADVDIFF2D;
  auto mark = [&](int i) {
    if (marks && marks[i]) cudaEventRecord(marks[i], st);
  };
  cudaError_t e;
  mark(0);
  if ((e = launch_ad_stage(1, fd, ep, S, st)) != cudaSuccess) return e;
  mark(1);
  k_scan_tile<<<(unsigned)phase_blocks(kPhaseScanTile, ode, N, fd.sms), kScanThreads, 0, st>>>(fd);
  mark(2);  // (marks[3] is not recorded: the scan_add slot is empty)
  if (rs_two_phase(N, fd.sms)) k_rs_corners<<<rs_corner_blocks(N), 256, 0, st>>>(fd, ep);
  k_resample<<<(unsigned)phase_blocks(kPhaseResample, ode, N, fd.sms), kResampleThreads, 0, st>>>(fd, ep);
  mark(4);
  if ((e = launch_ad_stage(2, fd, ep, S, st)) != cudaSuccess) return e;
  mark(5);
  k_moments<0, 5><<<phase_blocks(kPhaseMoments, ode, N, fd.sms), kMomentThreads, 0, st>>>(fd, 0);
  k_xbar<<<xbar_blocks(fd), kMomentThreads, 0, st>>>(fd);
  mark(6);
  return cudaGetLastError();
}

cudaError_t launch_init(int ode, const FilterDev& fd, cudaStream_t st) {
  switch (ode) {
    case PF_ODE_ADVDIFF2D: {
      const int64_t N = fd.N;
      k_init<0, 5><<<phase_blocks(kPhaseInit, ode, N, fd.sms), kInitThreads, 0, st>>>(fd);
      k_moments<0, 5><<<phase_blocks(kPhaseMoments, ode, N, fd.sms), kMomentThreads, 0, st>>>(fd, 1);
      k_xbar<<<xbar_blocks(fd), kMomentThreads, 0, st>>>(fd);
      return cudaGetLastError();
    }
    case PF_ODE_LINEAR2: return launch_init_t<Linear2>(fd, st);
    case PF_ODE_ROBERTSON: return launch_init_t<Robertson>(fd, st);
    case PF_ODE_MICHAELIS3: return launch_init_t<Michaelis>(fd, st);
    case PF_ODE_BRUSSELATOR1D: {
      const int64_t N = fd.N;
      k_init<64, 3><<<phase_blocks(kPhaseInit, ode, N, fd.sms), kInitThreads, 0, st>>>(fd);
      k_moments<64, 3><<<phase_blocks(kPhaseMoments, ode, N, fd.sms), kMomentThreads, 0, st>>>(fd, 1);
      return cudaGetLastError();
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_epoch(int ode, const FilterDev& fd, const EpochParams* ep, int S, cudaStream_t st,
                         cudaEvent_t* marks) {
  switch (ode) {
    case PF_ODE_LINEAR2: return launch_epoch_t<Linear2>(fd, ep, S, st, marks);
    case PF_ODE_ROBERTSON: return launch_epoch_t<Robertson>(fd, ep, S, st, marks);
    case PF_ODE_MICHAELIS3: return launch_epoch_t<Michaelis>(fd, ep, S, st, marks);
    case PF_ODE_BRUSSELATOR1D: return launch_epoch_bruss(fd, ep, S, st, marks);
    case PF_ODE_ADVDIFF2D: return launch_epoch_ad(fd, ep, S, st, marks);
  }
  return cudaErrorInvalidValue;
}

int kernels_per_epoch(int ode) {
  (void)ode;
  return kEpochKernels;
}

cudaError_t launch_theta_mean(const FilterDev& fd, cudaStream_t st) {
  if (fd.p == 2) k_theta_mean<2><<<1, kMomentThreads, 0, st>>>(fd);
  else if (fd.p == 4) k_theta_mean<4><<<1, kMomentThreads, 0, st>>>(fd);
  else if (fd.p == 5) k_theta_mean<5><<<1, kMomentThreads, 0, st>>>(fd);
  else k_theta_mean<3><<<1, kMomentThreads, 0, st>>>(fd);
  return cudaGetLastError();
}

// Kernels are loaded lazily at their first launch, and a first launch may wait
// for the device to drain.  Querying a kernel's attributes loads it, so this
// loads every kernel of the library up front (once per process and device).
namespace {
template <class K>
cudaError_t touch(K* k) {
  cudaFuncAttributes a;
  return cudaFuncGetAttributes(&a, reinterpret_cast<const void*>(k));
}
}  // namespace

// A kernel that stages the substep table in dynamic shared memory may need
// more than the default 48 KB (PF_MAX_SUBSTEPS entries); loads it as well.
cudaError_t allow_step_table(const void* k) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(sizeof(StepCoef) * (size_t)kSMax));
}

struct UploadBlob {
  unsigned char b[kUploadBytes];
};

__global__ void k_upload(unsigned char* __restrict__ dst, int n, const __grid_constant__ UploadBlob blob) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = blob.b[i];
}

cudaError_t upload_small(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes > (size_t)kUploadBytes) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  if (bytes == 0) return cudaSuccess;
  UploadBlob blob;
  std::memcpy(blob.b, src, bytes);
  k_upload<<<1, 128, 0, st>>>(static_cast<unsigned char*>(dst), (int)bytes, blob);
  return cudaGetLastError();
}

cudaError_t preload_main_kernels() {
  const void* ks[] = {
      (const void*)k_init<2, 2>, (const void*)k_init<3, 3>, (const void*)k_init<64, 3>,
      (const void*)k_init<3, 4>, (const void*)k_moments<3, 4>, (const void*)k_theta_mean<4>,
      (const void*)k_moments<2, 2>, (const void*)k_moments<3, 3>, (const void*)k_moments<64, 3>,
      (const void*)k_scan_tile, (const void*)k_resample,
      (const void*)k_theta_mean<2>, (const void*)k_theta_mean<3>, (const void*)k_theta_mean<5>,
      (const void*)k_set_moments, (const void*)k_init<0, 5>, (const void*)k_moments<0, 5>,
      (const void*)k_xbar, (const void*)k_upload, (const void*)k_rs_corners,
      (const void*)k_stage1_ess,
      (const void*)k_batch_init, (const void*)k_batch_scan_tile,
      (const void*)k_batch_resample,
      (const void*)k_batch_moments<2, 2>, (const void*)k_batch_moments<3, 3>,
      (const void*)k_batch_moments<64, 3>, (const void*)k_batch_moments<3, 4>};
  for (const void* k : ks) {
    const cudaError_t e = touch(k);
    if (e != cudaSuccess) return e;
  }
  static const int lmms[] = {PF_LMM_BDF2, PF_LMM_BDF3, PF_LMM_AM2, PF_LMM_AB2};
  for (int lmm : lmms) {
    StageKernel k[6];
    BatchStageKernel kb[6];
    stage_kernels<Linear2>(lmm, k[0], k[1]);
    stage_kernels<Robertson>(lmm, k[2], k[3]);
    stage_kernels<Michaelis>(lmm, k[4], k[5]);
    batch_stage_kernels<Linear2>(lmm, kb[0], kb[1]);
    batch_stage_kernels<Robertson>(lmm, kb[2], kb[3]);
    batch_stage_kernels<Michaelis>(lmm, kb[4], kb[5]);
    for (int i = 0; i < 6; ++i) {
      cudaError_t e = allow_step_table(reinterpret_cast<const void*>(k[i]));
      if (e == cudaSuccess) e = allow_step_table(reinterpret_cast<const void*>(kb[i]));
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// ================================================ shard of a sharded filter
// Algorithm 1 over a global ensemble split into contiguous shards, one per GPU
// (the particle-parallel layout of Sec. 3.1): each shard runs the phases above
// on its own particles, and the host exchanges what couples them -- the
// log-sum-exp shift, the tile totals of the cumulative weights, the parents
// of the resampled slots and the moment sums.  A shard starts on a tile
// boundary of the global scan tiling, so its tile totals are those of a
// filter of the whole ensemble, and so are the offsets below.

// The global tile offsets and floors from every tile's total (all shards',
// in slot order): the block of scan_offsets_core a filter of the whole
// ensemble runs, so they are bit-identical to its.  out[t] = c at the last
// slot of tile t (a full tile: boff + T), out[nb] = c_{N-1} from the last
// tile's last tile-local value cl_last, out[nb + 1] = the epoch's resampling
// uniform.
__global__ void __launch_bounds__(kScanThreads) k_shard_offsets(const __grid_constant__ FilterDev fd,
                                                              const EpochParams* __restrict__ ep,
                                                              const double* __restrict__ tiles, int nb,
                                                              double cl_last, double* boff_all,
                                                              double* pmax_all, double* out) {
  __shared__ double s_warp[33];
  scan_offsets_core(tiles, nb, boff_all, pmax_all, s_warp, nullptr);
  __syncthreads();
  for (int t = threadIdx.x; t < nb; t += blockDim.x)
    out[t] = max_nonneg(boff_all[t] + tiles[t], pmax_all[t]);
  if (threadIdx.x == 0) {
    const double total = max_nonneg(boff_all[nb - 1] + cl_last, pmax_all[nb - 1]);
    out[nb] = total;
    out[nb + 1] = resample_u(fd, ep);
    fd.ctrl->c_total = total;
  }
}

// Step 3b for the outputs i in [i_lo, i_lo + cnt) whose parent lies in this
// shard: l_i = min{k : c_k > tau_i} over the shard's cumulative weights (the
// first k with c_k = c_{N-1} for i >= i_fb, where tau_i reaches the total),
// tau_i = ((i + u)/N) c_{N-1} over the whole ensemble.  Each output's parent
// record -- x, h1, h2 (d each), phi (p), ll1, the global parent slot -- goes to
// send[j * R], j = i - i_lo, R = 3d + p + 2.
__global__ void __launch_bounds__(256) k_shard_resample(const __grid_constant__ FilterDev fd, int64_t i_lo,
                                                       int64_t cnt, int64_t i_fb, double u, double total,
                                                       int64_t n_all, double* __restrict__ send) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= cnt) return;
  const int64_t i = i_lo + j;
  const CumTiles c = cum_tiles(fd);
  const int64_t N = fd.N;
  int64_t l;
  if (i >= i_fb) {
    l = lower_bound_bits(c, N, __double_as_longlong(total));
  } else {
    const double tau = ((double)i + u) / (double)n_all * total;
    l = upper_bound_bits(c, N, __double_as_longlong(tau));
  }
  // the host plans only outputs whose parent lies here, so l < N; the clamp
  // keeps a wrong plan from reading past the shard
  if (l >= N) l = N - 1;
  const Ensemble E = committed(fd, fd.ctrl->cur);
  const int d = fd.d, p = fd.p;
  double* r = send + j * (int64_t)(3 * d + p + 2);
  for (int k = 0; k < d; ++k) {
    r[k] = E.x[k * N + l];
    r[d + k] = E.h1[k * N + l];
    r[2 * d + k] = E.h2[k * N + l];
  }
  for (int k = 0; k < p; ++k) r[3 * d + k] = E.phi[k * N + l];
  r[3 * d + p] = fd.ll1[l];
  r[3 * d + p + 1] = (double)(l + (int64_t)fd.slot0);
}

// The received parent records of this shard's slots (in slot order) into the
// parent buffers stage 2 gathers from (x, h1, h2, phi: SoA; ll1), the slot's
// own index as its gather index, and the global parent slot.
__global__ void __launch_bounds__(256) k_shard_unpack(const __grid_constant__ FilterDev fd,
                                                     const double* __restrict__ recv, Ensemble par,
                                                     double* __restrict__ par_ll1,
                                                     int32_t* __restrict__ gparent) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t N = fd.N;
  if (n >= N) return;
  const int d = fd.d, p = fd.p;
  const double* r = recv + n * (int64_t)(3 * d + p + 2);
  for (int k = 0; k < d; ++k) {
    par.x[k * N + n] = r[k];
    par.h1[k * N + n] = r[d + k];
    par.h2[k * N + n] = r[2 * d + k];
  }
  for (int k = 0; k < p; ++k) par.phi[k * N + n] = r[3 * d + k];
  par_ll1[n] = r[3 * d + p];
  gparent[n] = (int32_t)r[3 * d + p + 1];
  fd.idx[n] = (int32_t)n;
}

// Step 6's commit from the global moment sums (every shard's, added in shard
// order by the host), then the factor L of the new C for the next epoch's
// Step 4a (cholesky_psd, as the resampling launch of a filter forms it).
template <int D, int P>
__global__ void __launch_bounds__(kMomentThreads) k_shard_commit(const __grid_constant__ FilterDev fd,
                                                               const double* __restrict__ sums,
                                                               int is_init) {
  constexpr int NV = MomentLayout<D, P>::kN;
  __shared__ double s_part[kMomentShared<NV>];
  __shared__ double s_tot[NV];
  __shared__ int s_flag;
  if (fd.ctrl->status != PF_OK) return;
  for (int k = threadIdx.x; k < NV; k += blockDim.x) s_tot[k] = sums[k];
  __syncthreads();
  moments_commit<D, P>(fd, is_init, s_tot, s_part, &s_flag);
  __syncthreads();
  if (threadIdx.x == 0 && fd.ctrl->status == PF_OK) {
    double L[kPMax * kPMax];
    cholesky_psd(fd.p, fd.ctrl->C, L);
    for (int i = 0; i < kPMax * kPMax; ++i) fd.ctrl->L[i] = L[i];
  }
}

// Step 1's draws alone (a shard's moments are committed from the global sums)
cudaError_t launch_init_draws(int ode, const FilterDev& fd, cudaStream_t st) {
  const unsigned g = (unsigned)phase_blocks(kPhaseInit, ode, fd.N, fd.sms);
  switch (ode) {
    case PF_ODE_LINEAR2: k_init<2, 2><<<g, kInitThreads, 0, st>>>(fd); break;
    case PF_ODE_ROBERTSON: k_init<3, 3><<<g, kInitThreads, 0, st>>>(fd); break;
    case PF_ODE_MICHAELIS3: k_init<3, 4><<<g, kInitThreads, 0, st>>>(fd); break;
    case PF_ODE_BRUSSELATOR1D: k_init<64, 3><<<g, kInitThreads, 0, st>>>(fd); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Stage 1 or 2 of one epoch of a filter whose moments and ensemble are set
// (a shard: for stage 2 the caller passes the descriptor whose committed
// buffers are the received parents)
cudaError_t launch_stage(int stage, const FilterDev& fd, const EpochParams* ep, int S,
                         cudaStream_t st) {
  if (fd.ode == PF_ODE_BRUSSELATOR1D) return launch_bruss_stage(stage, fd, ep, S, st);
  StageKernel k1, k2;
  switch (fd.ode) {
    case PF_ODE_LINEAR2: stage_kernels<Linear2>(fd.lmm, k1, k2); break;
    case PF_ODE_ROBERTSON: stage_kernels<Robertson>(fd.lmm, k1, k2); break;
    case PF_ODE_MICHAELIS3: stage_kernels<Michaelis>(fd.lmm, k1, k2); break;
    default: return cudaErrorInvalidValue;
  }
  const unsigned g = stage_grid(fd.N, fd.sms);
  (stage == 1 ? k1 : k2)<<<g, stage_threads(fd.N, fd.sms), (size_t)S * sizeof(StepCoef), st>>>(fd, ep);
  return cudaGetLastError();
}

cudaError_t launch_scan_tiles(const FilterDev& fd, int ntiles, cudaStream_t st) {
  k_scan_tile<<<(unsigned)ntiles, kScanThreads, 0, st>>>(fd);
  return cudaGetLastError();
}

cudaError_t launch_shard_offsets(const FilterDev& fd, const EpochParams* ep, const double* tiles,
                                 int nb, double cl_last, double* boff_all, double* pmax_all,
                                 double* out, cudaStream_t st) {
  k_shard_offsets<<<1, kScanThreads, 0, st>>>(fd, ep, tiles, nb, cl_last, boff_all, pmax_all, out);
  return cudaGetLastError();
}

cudaError_t launch_shard_resample(const FilterDev& fd, int64_t i_lo, int64_t cnt, int64_t i_fb,
                                  double u, double total, int64_t n_all, double* send,
                                  cudaStream_t st) {
  if (cnt <= 0) return cudaSuccess;
  k_shard_resample<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(fd, i_lo, cnt, i_fb, u, total,
                                                                   n_all, send);
  return cudaGetLastError();
}

cudaError_t launch_shard_unpack(const FilterDev& fd, const double* recv, const Ensemble& par,
                                double* par_ll1, int32_t* gparent, cudaStream_t st) {
  k_shard_unpack<<<(unsigned)((fd.N + 255) / 256), 256, 0, st>>>(fd, recv, par, par_ll1, gparent);
  return cudaGetLastError();
}

// The moment sums of the pending buffer (fd.shard_sums set) with the shift
// lw_max already in the control block.
cudaError_t launch_shard_moments(const FilterDev& fd, cudaStream_t st) {
  const unsigned g = (unsigned)phase_blocks(kPhaseMoments, fd.ode, fd.N, fd.sms);
  switch (fd.ode) {
    case PF_ODE_LINEAR2: k_moments<2, 2><<<g, kMomentThreads, 0, st>>>(fd, 0); break;
    case PF_ODE_ROBERTSON: k_moments<3, 3><<<g, kMomentThreads, 0, st>>>(fd, 0); break;
    case PF_ODE_MICHAELIS3: k_moments<3, 4><<<g, kMomentThreads, 0, st>>>(fd, 0); break;
    case PF_ODE_BRUSSELATOR1D: k_moments<64, 3><<<g, kMomentThreads, 0, st>>>(fd, 0); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_shard_commit(const FilterDev& fd, const double* sums, int is_init, cudaStream_t st) {
  switch (fd.ode) {
    case PF_ODE_LINEAR2: k_shard_commit<2, 2><<<1, kMomentThreads, 0, st>>>(fd, sums, is_init); break;
    case PF_ODE_ROBERTSON: k_shard_commit<3, 3><<<1, kMomentThreads, 0, st>>>(fd, sums, is_init); break;
    case PF_ODE_MICHAELIS3: k_shard_commit<3, 4><<<1, kMomentThreads, 0, st>>>(fd, sums, is_init); break;
    case PF_ODE_BRUSSELATOR1D: k_shard_commit<64, 3><<<1, kMomentThreads, 0, st>>>(fd, sums, is_init); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

bool ode_supported(int ode) {
  return ode == PF_ODE_LINEAR2 || ode == PF_ODE_ROBERTSON || ode == PF_ODE_BRUSSELATOR1D ||
         ode == PF_ODE_ADVDIFF2D || ode == PF_ODE_MICHAELIS3;
}

cudaError_t launch_set_moments(const FilterDev& fd, cudaStream_t st) {
  k_set_moments<<<1, 32, 0, st>>>(fd);
  return cudaGetLastError();
}

// One batched phase over the device tile table tiles[0..ntiles).  Stage and
// moment phases need tiles of one model only (ode); the other phases take any
// mix.
// smem is the step-table size of the largest interval among the filters.
cudaError_t launch_batch_phase(int phase, int ode, int lmm, const FilterDev* fds,
                               const EpochParams* const* eps, const BatchTile* tiles, int ntiles,
                               size_t smem, int is_init, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  switch (phase) {
    case kPhaseInit: k_batch_init<<<ntiles, kInitThreads, 0, st>>>(fds, tiles); break;
    case kPhaseStage1:
    case kPhaseStage2: {
      const int stage = phase == kPhaseStage1 ? 1 : 2;
      if (ode == PF_ODE_BRUSSELATOR1D)
        return launch_batch_bruss_stage(stage, fds, eps, tiles, ntiles, smem, st);
      BatchStageKernel k1, k2;
      if (ode == PF_ODE_ROBERTSON) batch_stage_kernels<Robertson>(lmm, k1, k2);
      else if (ode == PF_ODE_LINEAR2) batch_stage_kernels<Linear2>(lmm, k1, k2);
      else if (ode == PF_ODE_MICHAELIS3) batch_stage_kernels<Michaelis>(lmm, k1, k2);
      else return cudaErrorInvalidValue;
      (stage == 1 ? k1 : k2)<<<ntiles, kSmallThreads, smem, st>>>(fds, eps, tiles);
      break;
    }
    case kPhaseScanTile: k_batch_scan_tile<<<ntiles, kScanThreads, 0, st>>>(fds, tiles); break;
    case kPhaseResample: k_batch_resample<<<ntiles, kResampleThreads, 0, st>>>(fds, eps, tiles); break;
    case kPhaseMoments:
      if (ode == PF_ODE_LINEAR2) k_batch_moments<2, 2><<<ntiles, kMomentThreads, 0, st>>>(fds, tiles, is_init);
      else if (ode == PF_ODE_ROBERTSON) k_batch_moments<3, 3><<<ntiles, kMomentThreads, 0, st>>>(fds, tiles, is_init);
      else if (ode == PF_ODE_BRUSSELATOR1D) k_batch_moments<64, 3><<<ntiles, kMomentThreads, 0, st>>>(fds, tiles, is_init);
      else if (ode == PF_ODE_MICHAELIS3) k_batch_moments<3, 4><<<ntiles, kMomentThreads, 0, st>>>(fds, tiles, is_init);
      else return cudaErrorInvalidValue;
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pfg
