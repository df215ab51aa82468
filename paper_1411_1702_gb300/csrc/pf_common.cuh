// pf_common.cuh -- device data layout and primitives shared by the kernels of
// the GB300 LMM PF-SMC sampler (Algorithm 1 of Arnold, Calvetti, Somersalo).
//
// Layout in HBM (one filter):
//   two ensemble buffers (ping-pong, the committed one is Ctrl::cur), each SoA:
//     x[i*N + n], h1[i*N + n], h2[i*N + n]   i < d   (x_n, x_{n-1}, x_{n-2})
//     phi[i*N + n]                           i < p   (working-space parameter)
//     lw[n]                                          (unnormalised log weight)
//   work arrays: ll1[N], lg[N], c[N] (FP64), idx[N] (int32)
//   x0[d] (the fixed initial state) and xbar[d] (the committed weighted mean)
//   per-block scratch, the control block and the epoch parameter block.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "../../include/pf.h"
#include "pf_math.cuh"

namespace pfg {

constexpr int kDMax = 64;            // largest state kept in registers (small models)
constexpr int kPMax = 5;
constexpr int kMMax = PF_MAX_OBS;
constexpr int kSMax = PF_MAX_SUBSTEPS;
constexpr int kScanItemsMax = 4;     // elements per thread in the scan, at most
constexpr int kScanThreads = 256;
constexpr int kScanTilesPerSm = 4;    // scan tiles that fill one wave: 4 blocks on each SM
constexpr int kMomentBlocksPerSm = 2;
constexpr int kMomentThreads = 256;
// the most SMs a device may have for the fixed-size scratch of the no-alloc call
constexpr int kMaxSms = 1024;

// Blocks of the moment kernels for N particles on a device of sms SMs: one
// per 256 particles up to one block per SM, then one per SM (grid-stride, so
// no SM holds two blocks while another holds one) until two per SM pay, then
// two per SM.
__host__ __device__ inline int moment_blocks(int64_t N, int sms) {
  const int64_t b = (N + kMomentThreads - 1) / kMomentThreads;
  if (b <= sms) return (int)b;
  return b < (int64_t)kMomentBlocksPerSm * sms ? sms : kMomentBlocksPerSm * sms;
}
__host__ __device__ inline int moment_blocks_max(int sms) { return kMomentBlocksPerSm * sms; }

// Random-stream purposes (Philox counter word 2, low byte).
enum : uint32_t { kRngInit = 1, kRngTheta = 2, kRngInnov = 3, kRngResample = 4 };

// One substep of the shared grid.
// BDF kinds 1, 2 (BDF1 and BDF2):
//   x_{n+1} - rho1 x_n - rho2 x_{n-1} = gamma f(t_{n+1}, x_{n+1}),
//   predictor x_p = pi0 x_n + pi1 x_{n-1} + pi2 x_{n-2} (kind 2),
//   Milne local error e = mu (x_{n+1} - x_p).
//   Kind 1 (cold start): Newton starts at x_n and the error predictor is the
//   explicit-Euler step x_n + h f(t_n, x_n).
// BDF kind 3: x_{n+1} - rho1 x_n - rho2 x_{n-1} - rho3 x_{n-2} = gamma f_{n+1},
//   predictor pi0 x_n + pi1 x_{n-1} + pi2 x_{n-2} + pi3 f(t_n, x_n).
// Adams kinds 10 + q (Moulton, implicit) and 20 + q (Bashforth, explicit), q
// the order, with f_j = f(t_j, x_j):
//   predictor AB_q:  x_p = x_n + pi0 f_n + pi1 f_{n-1} + pi2 f_{n-2};
//   corrector AM_q:  x_c = x_n + gamma f_{n+1} + rho1 f_n + rho2 f_{n-1}
//   (weights include h and are zero beyond the order).
// in0, in1: the problem's time-dependent input at t_n and t_{n+1} (M1's Phi;
// zero for autonomous problems).
struct StepCoef {
  double h, gamma, rho1, rho2, pi0, pi1, pi2, mu;
  int kind;
  int pad;
  double rho3, pi3;
  double in0, in1;
};

// Per-epoch parameters (one observation).  Only the header and the first S
// entries of sc are copied to the device.
struct EpochParams {
  double t;
  double y[kMMax];
  double inv_sigma[kMMax];
  int S;
  uint32_t epoch;   // Philox epoch word = committed epoch count before this one
  int64_t pad;
  double in_hist[2]; // the input at t_n - h and t_n - 2h (h = the first
                     // substep): rebuilds the Adams derivative history
  StepCoef sc[kSMax];
};
constexpr size_t kEpochHeaderBytes = offsetof(EpochParams, sc);

// Control block: committed moments and the commit flag (device-resident).
struct Ctrl {
  int cur;              // committed ensemble buffer (0/1)
  int status;           // sticky error of the enqueued epochs (pf_status)
  int64_t failed_epoch; // epoch word of the first failed epoch
  int64_t epochs_done;  // committed epochs
  double phibar[kPMax];
  double C[kPMax * kPMax];
  double L[kPMax * kPMax];   // lower Cholesky factor of C (PSD rule)
  double logW;          // log sum exp(lw) of the committed weights
  double ess;
  double theta_mean[kPMax];
  double wsum;          // sum of exp(lw - lw_max) of the committed weights
  double lg_max;        // max log fitness weight of the running epoch
  double lw_max;        // max new log weight of the running epoch
  double c_total;       // total of the cumulative fitness weights
  double g_sq;          // sum of the squared fitness weights g (pf_stats, on demand)
  int64_t n_unique;
  int64_t n_nonfinite;
};

struct Ensemble {
  double* x;
  double* h1;
  double* h2;
  double* phi;
  double* lw;
};

// Everything a kernel needs about one filter (passed by value).
struct FilterDev {
  int64_t N;
  int ode;
  int lmm;          // pf_lmm (selects the propagation kernels)
  int d, p, m, K;
  int transform;
  int obs[kMMax];
  double a, s, kappa;
  uint64_t seed;
  uint32_t stream_id;
  Ensemble ens[2];
  double* ll1;
  double* lg;
  double* c;
  int32_t* idx;
  double* blk;      // per-block scratch (max or sums), >= max grid size
  double* boff;     // per-tile offsets of the scan
  double* pmax;     // per-tile running maximum of the earlier tiles' last c
  double* tsq;      // per-block sums of g^2 (first-stage ESS, moment_blocks_max(sms))
  double* part;     // moment partial records, moment_blocks_max(sms) * nrec
  double* wk;       // model work arrays (Brusselator: r, predictor, error sums; 2D system: weights)
  unsigned* ticket; // 4 counters for the last-block pattern
  Ctrl* ctrl;
  int nrec;
  int prior_kind[kPMax];
  double prior_lo[kPMax], prior_hi[kPMax];
  const double* x0; // fixed initial state (d)
  double* xbar;     // committed weighted mean of x (d)
  // A shard of a particle-sharded filter holds the global slots
  // [slot0, slot0 + N) of an ensemble of Ntile particles: its random streams
  // are keyed by the global slot, and its cumulative weights use the tiling of
  // the global ensemble.  A filter of its own has slot0 = 0 and Ntile = N.
  uint32_t slot0;
  int64_t Ntile;
  int sms;          // SMs of the device the filter lives on (grid shapes)
  // if set, the moments kernel stores its weighted sums here instead of
  // committing (a shard's part of the global sums)
  double* shard_sums;
};

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 32x32
// products of counter words 0 and 2 with the round multipliers; the new words
// are (hi1^c1^k0, lo1, hi0^c3^k1, lo0); the key is bumped by the Weyl
// constants between rounds.  Counter = (slot n, epoch, purpose | block<<8,
// filter id), key = seed halves.
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// n is the particle's slot in its filter (a shard adds its first global
// slot); the epoch's resampling uniform is keyed by slot 0 of the whole filter.
__device__ __forceinline__ U4 draw_block(const FilterDev& fd, uint32_t purpose, uint32_t n,
                                         uint32_t epoch, uint32_t block) {
  const uint32_t slot = purpose == kRngResample ? n : n + fd.slot0;
  return philox4x32_10(U4{slot, epoch, purpose | (block << 8), fd.stream_id},
                       (uint32_t)(fd.seed & 0xffffffffu), (uint32_t)(fd.seed >> 32));
}

// 53-bit uniform in [0,1): 27 high bits of a, 26 high bits of b, times 2^-53.
__device__ __forceinline__ double uniform53(uint32_t a, uint32_t b) {
  const uint64_t bits = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return (double)bits * 0x1.0p-53;
}

// Two standard normals from one Philox block by Box-Muller (Box & Muller
// 1958): r = sqrt(-2 log(1 - u1)), (z0, z1) = r (cos 2 pi u2, sin 2 pi u2)
// for the 53-bit uniforms u1 = k1 2^-53, u2 = k2 2^-53 of uniform53.  1 - u1
// = (2^53 - k1) 2^-53 is exact; the logarithm and the angle's sine and cosine
// are the table-driven ones of pf_math.cuh (about 28 FP64 instructions fewer
// a pair than the library routines).
__device__ __forceinline__ void normal_pair(const U4& w, double& z0, double& z1) {
  const uint64_t k1 = ((uint64_t)(w.x >> 5) << 26) | (uint64_t)(w.y >> 6);
  const uint64_t k2 = ((uint64_t)(w.z >> 5) << 26) | (uint64_t)(w.w >> 6);
  const double v = (double)((1ULL << 53) - k1) * 0x1.0p-53;
  const double r = sqrt(-2.0 * pfm::log_pos(v));
  double sn, cs;
  pfm::sincospi_k52(k2, sn, cs);
  z0 = r * cs;
  z1 = r * sn;
}

// ------------------------------------------------------------ arithmetic
// Reciprocal: the hardware approximation (rcp.approx.ftz.f64) refined by one
// Newton-Raphson step r <- r + r (1 - x r) (the textbook iteration for 1/x,
// e.g. Markstein 1990), which roughly doubles the correct bits.  Used only
// inside the Newton solves, whose own iteration absorbs the residual error.
__device__ __forceinline__ double rcp_hw(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}

__device__ __forceinline__ double rcp_nr(double x) {
  const double r = rcp_hw(x);
  const double e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// The reciprocal of a Newton correction's pivot.  Before the last iteration
// it is the hardware approximation alone: the following iteration evaluates
// the exact residual and so corrects that step's error (an inexact Newton
// step).  In the last iteration, whose correction is final, it is refined.
__device__ __forceinline__ double rcp_newton(double x, bool last) {
  return last ? rcp_nr(x) : rcp_hw(x);
}

__device__ __forceinline__ double rcp_nr2(double x) {
  const double r = rcp_nr(x);
  const double e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// the programmatic-stream-serialization attribute may be scheduled while the
// stream's previous kernel is still running.  pdl_wait() returns once that
// kernel has completed and its memory operations are visible (at once when
// the launch had no such dependency), so every access of the epoch's state
// comes after it.  pdl_trigger() lets the next such kernel be scheduled once
// every block of this one has called it or exited; it orders nothing.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Finite test on the bit pattern (integer pipe, no FP64 compare).
__device__ __forceinline__ bool finite_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return ((b >> 52) & 0x7ffull) != 0x7ffull;
}

__device__ __forceinline__ bool is_neg_inf(double v) {
  return (unsigned long long)__double_as_longlong(v) == 0xfff0000000000000ull;
}

// ------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum/max; every thread gets the result.  s needs 32 doubles.
// Deterministic: the tree depends only on the block size.
__device__ __forceinline__ double block_sum(double v, double* s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) s[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? s[threadIdx.x] : 0.0;
  if (wid == 0) {
    t = warp_sum(t);
    if (lane == 0) s[0] = t;
  }
  __syncthreads();
  return s[0];
}

__device__ __forceinline__ double block_max(double v, double* s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) s[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? s[threadIdx.x] : -CUDART_INF;
  if (wid == 0) {
    t = warp_max(t);
    if (lane == 0) s[0] = t;
  }
  __syncthreads();
  return s[0];
}

// Last-block election among the vg blocks that work on one filter (vg =
// gridDim.x for a single-filter launch): after every block has written its
// partial result, the block that increments the ticket last sees all of them.
// No waiting.
__device__ __forceinline__ bool elect_last_block(unsigned* ticket, int* s_flag, unsigned vg) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(ticket, 1u);
    *s_flag = (t == vg - 1) ? 1 : 0;
  }
  __syncthreads();
  if (*s_flag) {
    __threadfence();
    if (threadIdx.x == 0) *ticket = 0u;  // ready for the next launch
    return true;
  }
  return false;
}

}  // namespace pfg
