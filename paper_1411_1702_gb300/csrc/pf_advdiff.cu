// pf_advdiff.cu -- stage kernels of the epoch for the paper's 2D
// advection-diffusion system (Sec. 4): U' = L U on the periodic nt x nt grid,
//   L = -{k1^2 B1'B1 + k1 k3 (B1'B2 + B2'B1) + (k2^2 + k3^2) B2'B2} + c1 B1 + c2 B2,
// B1 = I (x) ell, B2 = ell (x) I, (ell u)_j = u_j - u_{j-1} (periodic), state
// U[iy*nt + ix], theta = (k1, k2, k3, c1, c2).
//
// The system is linear, so Newton's method (Sec. 2.1) with the exact Jacobian
// L solves each BDF step in one iteration; the work is the linear solve with
// I - gamma L, which differs per particle (theta) and per step size.  L is
// built from circulant difference matrices, so the 2D DFT diagonalises it:
// with a(m) = 1 - exp(-2 pi i m / nt) the symbol of ell,
//   lambda(mx, my) = -(k1^2 |a_x|^2 + 2 k1 k3 Re(conj(a_x) a_y) + (k2^2 + k3^2) |a_y|^2)
//                    + c1 a_x + c2 a_y,
// and (I - gamma L)^{-1} is a division by 1 - gamma lambda mode by mode.  One
// Newton iteration therefore costs a 7-point stencil for the residual
// G = x - r - gamma L x, a forward real 2D DFT, one complex multiply per mode
// and an inverse DFT -- O(d nt) flops instead of a sparse or banded LU.
//
// One block per particle: its history ring (x_n, x_{n-1}, x_{n-2}, iterate),
// the half spectrum (nt odd, so modes mx = 0..(nt-1)/2 and Hermitian symmetry
// give the rest), the per-mode multipliers, and in stage 2 the Milne predictor
// and error sums all live in shared memory; the DFTs are direct sums over a
// cos/sin table (nt is small and prime or nearly so), split over the block's
// threads by output.  Global memory is touched once per particle per stage.
#include "pf_epoch.cuh"
#include "pf_kernels.h"

namespace pfg {

constexpr int kAdMaxSide = 45;
constexpr int kAdScDoubles = (int)(sizeof(StepCoef) / sizeof(double));

__host__ __device__ inline int ad_side(int d) {
  for (int nt = 3; nt <= kAdMaxSide; nt += 2)
    if (nt * nt == d) return nt;
  return 0;
}

// Shared-memory layout of one particle's block, in doubles.
struct AdLayout {
  int nt, d, H;
  int sc;    // step table, S entries
  int tw;    // cos(2 pi k / nt), then sin(2 pi k / nt), k < nt
  int X[4];  // x_n, x_{n-1}, x_{n-2} and the iterate (roles rotate)
  int s1;    // half spectrum [row][mx] (complex), also the inverse column output
  int s2;    // half spectrum [my][mx] (complex); the residual G (real, d) before it
  int wi;    // -1 / (nt^2 (1 - gamma lambda)) per mode (complex)
  int xp;    // stage 2: Milne predictor
  int ee;    // stage 2: error sums
  int total;
};

__host__ __device__ inline AdLayout ad_layout(int d, int S, bool err) {
  AdLayout L;
  L.nt = ad_side(d);
  L.d = d;
  L.H = (L.nt + 1) / 2;
  int off = 0;
  L.sc = off;
  off += S * kAdScDoubles;
  L.tw = off;
  off += 2 * L.nt;
  for (int k = 0; k < 4; ++k) {
    L.X[k] = off;
    off += d;
  }
  const int spec = 2 * L.nt * L.H;  // >= d
  L.s1 = off;
  off += spec;
  L.s2 = off;
  off += spec;
  L.wi = off;
  off += spec;
  L.xp = off;
  off += err ? d : 0;
  L.ee = off;
  off += err ? d : 0;
  L.total = off;
  return L;
}

// The operator for one parameter vector: the 7-point stencil of L (derived
// from the products of the difference matrices) and the symbol's weights.
struct AdOp {
  double c0, xm, xp, ym, yp, pm, mp;  // u(x,y), u(x-1,y), u(x+1,y), u(x,y-1), u(x,y+1), u(x+1,y-1), u(x-1,y+1)
  double kxx, kxy, kyy, c1, c2;       // k1^2, k1 k3, k2^2 + k3^2, c1, c2
};

__device__ __forceinline__ AdOp ad_op(const double* th) {
  const double k1 = th[0], k2 = th[1], k3 = th[2], c1 = th[3], c2 = th[4];
  AdOp o;
  o.kxx = k1 * k1;
  o.kxy = k1 * k3;
  o.kyy = k2 * k2 + k3 * k3;
  o.c1 = c1;
  o.c2 = c2;
  o.c0 = -2.0 * (o.kxx + o.kxy + o.kyy) + c1 + c2;
  o.xm = o.kxx + o.kxy - c1;
  o.xp = o.kxx + o.kxy;
  o.ym = o.kxy + o.kyy - c2;
  o.yp = o.kxy + o.kyy;
  o.pm = -o.kxy;
  o.mp = -o.kxy;
  return o;
}

__device__ __forceinline__ double ad_apply(const AdOp& o, const double* u, int nt, int ix, int iy) {
  const int xm = ix == 0 ? nt - 1 : ix - 1, xp = ix == nt - 1 ? 0 : ix + 1;
  const int rm = (iy == 0 ? nt - 1 : iy - 1) * nt, rp = (iy == nt - 1 ? 0 : iy + 1) * nt;
  const int r = iy * nt;
  double s = o.c0 * u[r + ix];
  s = fma(o.xm, u[r + xm], s);
  s = fma(o.xp, u[r + xp], s);
  s = fma(o.ym, u[rm + ix], s);
  s = fma(o.yp, u[rp + ix], s);
  s = fma(o.pm, u[rm + xp], s);
  s = fma(o.mp, u[rp + xm], s);
  return s;
}

// wi(my, mx) = -1 / (nt^2 (1 - gamma lambda(mx, my))): the inverse of the
// Newton matrix per mode, with the inverse DFT's 1/nt^2 and the sign of -G.
__device__ void ad_multipliers(const AdLayout& L, const AdOp& o, double gamma, const double* tw,
                               double* wi) {
  const int nt = L.nt, H = L.H;
  const double inv = 1.0 / (double)(nt * nt);
  for (int t = threadIdx.x; t < nt * H; t += blockDim.x) {
    const int my = t / H, mx = t - my * H;
    const double axr = 1.0 - tw[mx], axi = tw[nt + mx];
    const double ayr = 1.0 - tw[my], ayi = tw[nt + my];
    const double ax2 = fma(axr, axr, axi * axi), ay2 = fma(ayr, ayr, ayi * ayi);
    const double cr = fma(axr, ayr, axi * ayi);
    const double lr = fma(o.c1, axr, o.c2 * ayr) - fma(o.kxx, ax2, fma(2.0 * o.kxy, cr, o.kyy * ay2));
    const double li = fma(o.c1, axi, o.c2 * ayi);
    const double p = fma(-gamma, lr, 1.0), q = -gamma * li;
    const double s = -inv / fma(p, p, q * q);
    wi[2 * t] = s * p;
    wi[2 * t + 1] = -s * q;
  }
}

// One Newton iteration on the iterate XI: G = XI - (rho1 X0 + rho2 X1) -
// gamma L XI, then XI += -(I - gamma L)^{-1} G through the DFT.
__device__ void ad_newton(const AdLayout& L, const AdOp& o, const StepCoef& c, const double* tw,
                          const double* X0, const double* X1, double* XI, double* S1, double* S2,
                          const double* WI) {
  const int nt = L.nt, H = L.H, d = L.d, T = blockDim.x, tid = threadIdx.x;
  double* G = S2;
  for (int i = tid; i < d; i += T) {
    const int iy = i / nt, ix = i - iy * nt;
    const double lx = ad_apply(o, XI, nt, ix, iy);
    const double r = fma(c.rho1, X0[i], c.rho2 * X1[i]);
    G[i] = fma(-c.gamma, lx, XI[i] - r);
  }
  __syncthreads();
  // rows: S1[iy][mx] = sum_ix G[iy][ix] exp(-i phi mx ix)
  for (int t = tid; t < nt * H; t += T) {
    const int iy = t / H, mx = t - iy * H;
    const double* g = G + iy * nt;
    double re = 0.0, im = 0.0;
    int k = 0;
    for (int ix = 0; ix < nt; ++ix) {
      re = fma(g[ix], tw[k], re);
      im = fma(-g[ix], tw[nt + k], im);
      k += mx;
      if (k >= nt) k -= nt;
    }
    S1[2 * t] = re;
    S1[2 * t + 1] = im;
  }
  __syncthreads();
  // columns and the per-mode solve: S2[my][mx] = WI * sum_iy S1[iy][mx] exp(-i phi my iy)
  for (int t = tid; t < nt * H; t += T) {
    const int my = t / H, mx = t - my * H;
    double re = 0.0, im = 0.0;
    int k = 0;
    for (int iy = 0; iy < nt; ++iy) {
      const double ar = S1[2 * (iy * H + mx)], ai = S1[2 * (iy * H + mx) + 1];
      const double cs = tw[k], sn = tw[nt + k];
      re = fma(ar, cs, fma(ai, sn, re));
      im = fma(ai, cs, fma(-ar, sn, im));
      k += my;
      if (k >= nt) k -= nt;
    }
    const double wr = WI[2 * t], wm = WI[2 * t + 1];
    S2[2 * t] = fma(re, wr, -im * wm);
    S2[2 * t + 1] = fma(re, wm, im * wr);
  }
  __syncthreads();
  // inverse columns: S1[iy][mx] = sum_my S2[my][mx] exp(+i phi my iy)
  for (int t = tid; t < nt * H; t += T) {
    const int iy = t / H, mx = t - iy * H;
    double re = 0.0, im = 0.0;
    int k = 0;
    for (int my = 0; my < nt; ++my) {
      const double ar = S2[2 * (my * H + mx)], ai = S2[2 * (my * H + mx) + 1];
      const double cs = tw[k], sn = tw[nt + k];
      re = fma(ar, cs, fma(-ai, sn, re));
      im = fma(ai, cs, fma(ar, sn, im));
      k += iy;
      if (k >= nt) k -= nt;
    }
    S1[2 * t] = re;
    S1[2 * t + 1] = im;
  }
  __syncthreads();
  // inverse rows (Hermitian in mx): dx = Re z0 + 2 sum_{mx>0} Re(z_mx exp(+i phi mx ix))
  for (int i = tid; i < d; i += T) {
    const int iy = i / nt, ix = i - iy * nt;
    const double* z = S1 + 2 * iy * H;
    double acc = 0.0;
    int k = ix;
    for (int mx = 1; mx < H; ++mx) {
      acc = fma(z[2 * mx], tw[k], fma(-z[2 * mx + 1], tw[nt + k], acc));
      k += ix;
      if (k >= nt) k -= nt;
    }
    XI[i] += fma(2.0, acc, z[0]);
  }
  __syncthreads();
}

// Psi over the S substeps on the block's shared history ring (Steps 2 and
// 4b/4d).  On exit X[0], X[1], X[2] (after rotation, see ring) hold x_n,
// x_{n-1}, x_{n-2}; with ERR the squared Milne estimates are summed into EE.
template <bool ERR>
__device__ void ad_propagate(const AdLayout& L, const AdOp& o, const StepCoef* sc, int S, int K,
                             double* sm, int (&ring)[4]) {
  const int nt = L.nt, d = L.d, T = blockDim.x, tid = threadIdx.x;
  const double* tw = sm + L.tw;
  double* S1 = sm + L.s1;
  double* S2 = sm + L.s2;
  double* WI = sm + L.wi;
  double* XP = sm + L.xp;
  double* EE = sm + L.ee;
  double gamma_wi = CUDART_NAN;
  for (int s = 0; s < S; ++s) {
    const StepCoef c = sc[s];
    double* X0 = sm + ring[0];
    double* X1 = sm + ring[1];
    double* X2 = sm + ring[2];
    double* XI = sm + ring[3];
    for (int i = tid; i < d; i += T) {
      double xp;
      if (c.kind == 2) {
        xp = fma(c.pi0, X0[i], fma(c.pi1, X1[i], c.pi2 * X2[i]));
        if (ERR) XP[i] = xp;
      } else {
        xp = X0[i];
        if (ERR) {  // explicit-Euler error predictor of a cold-start step
          const int iy = i / nt, ix = i - iy * nt;
          XP[i] = fma(c.h, ad_apply(o, X0, nt, ix, iy), X0[i]);
        }
      }
      XI[i] = xp;
    }
    if (!(c.gamma == gamma_wi)) {
      ad_multipliers(L, o, c.gamma, tw, WI);
      gamma_wi = c.gamma;
    }
    __syncthreads();
    for (int it = 0; it < K; ++it) ad_newton(L, o, c, tw, X0, X1, XI, S1, S2, WI);
    if (ERR) {
      for (int i = tid; i < d; i += T) {
        const double e = c.mu * (XI[i] - XP[i]);
        EE[i] = fma(e, e, EE[i]);
      }
    }
    const int r3 = ring[3];
    ring[3] = ring[2];
    ring[2] = ring[1];
    ring[1] = ring[0];
    ring[0] = r3;
    // the next substep reads neighbours of the new x_n written by other threads;
    // ad_newton ended with a barrier, and EE/XP are per-thread indices
  }
}

__device__ __forceinline__ double ad_loglik(const FilterDev& fd, const EpochParams* __restrict__ ep,
                                            const double* X) {
  double s = 0.0;
  for (int i = 0; i < fd.m; ++i) {
    const double z = (ep->y[i] - X[fd.obs[i]]) * ep->inv_sigma[i];
    s = fma(z, z, s);
  }
  return -0.5 * s;
}

__device__ __forceinline__ void ad_tables(const AdLayout& L, double* sm) {
  double* tw = sm + L.tw;
  for (int k = threadIdx.x; k < L.nt; k += blockDim.x) {
    double sn, cs;
    sincospi(2.0 * (double)k / (double)L.nt, &sn, &cs);
    tw[k] = cs;
    tw[L.nt + k] = sn;
  }
}

template <int STAGE>
__global__ void __launch_bounds__(512) k_adstage(const __grid_constant__ FilterDev fd,
                                                 const EpochParams* __restrict__ ep) {
  extern __shared__ double s_dyn[];
  __shared__ double s_red[32];
  __shared__ double s_th[kPMax];
  __shared__ int s_flag;
  const Ctrl* ctrl = fd.ctrl;
  if (ctrl->status != PF_OK) return;
  const int S = ep->S;
  const AdLayout L = ad_layout(fd.d, S, STAGE == 2);
  double* sm = s_dyn;
  load_steps(reinterpret_cast<StepCoef*>(sm + L.sc), ep, S);  // ends with a barrier
  const int cur = ctrl->cur;
  const Ensemble src = committed(fd, cur);
  const Ensemble dst = pending(fd, cur);
  const int64_t N = fd.N;
  const int64_t n = blockIdx.x;
  const uint32_t epoch = ep->epoch;
  const int d = L.d, T = blockDim.x, tid = threadIdx.x;
  int64_t l = n;
  if (STAGE == 2) l = fd.idx[n];
  if (tid == 0) {
    double ph[5];
    if (STAGE == 1) {
      // Step 2: phibar^n = a phi^n + (1 - a) phibar
      for (int i = 0; i < 5; ++i) ph[i] = fd.a * src.phi[i * N + n] + (1.0 - fd.a) * ctrl->phibar[i];
    } else {
      // Step 4a: phi_{j+1}^n = phibar^l + s L z
      double z[6];
      for (int b = 0; b < 3; ++b) {
        const U4 w = draw_block(fd, kRngTheta, (uint32_t)n, epoch, (uint32_t)b);
        normal_pair(w, z[2 * b], z[2 * b + 1]);
      }
      for (int i = 0; i < 5; ++i) {
        double lz = 0.0;
        for (int k = 0; k <= i; ++k) lz = fma(ctrl->L[i * kPMax + k], z[k], lz);
        const double shr = fd.a * src.phi[i * N + l] + (1.0 - fd.a) * ctrl->phibar[i];
        ph[i] = fma(fd.s, lz, shr);
        dst.phi[i * N + n] = ph[i];
      }
    }
    for (int i = 0; i < 5; ++i) s_th[i] = (fd.transform == PF_TRANSFORM_LOG) ? exp(ph[i]) : ph[i];
  }
  ad_tables(L, sm);
  for (int i = tid; i < d; i += T) {
    const int64_t o = (int64_t)i * N + l;
    sm[L.X[0] + i] = src.x[o];
    sm[L.X[1] + i] = src.h1[o];
    sm[L.X[2] + i] = src.h2[o];
    if (STAGE == 2) sm[L.ee + i] = 0.0;
  }
  __syncthreads();
  double th[5];
  for (int i = 0; i < 5; ++i) th[i] = s_th[i];
  const AdOp op = ad_op(th);
  int ring[4] = {L.X[0], L.X[1], L.X[2], L.X[3]};
  ad_propagate<STAGE == 2>(L, op, reinterpret_cast<const StepCoef*>(sm + L.sc), S, fd.K, sm, ring);
  double* X0 = sm + ring[0];
  if (STAGE == 1) {
    double lg = -CUDART_INF;
    if (tid == 0) {
      const double ll = ad_loglik(fd, ep, X0);
      fd.ll1[n] = ll;
      lg = (src.lw[n] - ctrl->logW) + ll;
      if (!finite_bits(lg)) lg = -CUDART_INF;
      fd.lg[n] = lg;
    }
    stage1_tail(fd, epoch, lg, (int)blockIdx.x, (int)gridDim.x, s_red, &s_flag);
  } else {
    // Steps 4c, 4d: innovation v = sqrt(kappa E) z', written in (x, h1, h2) order
    const double* X1 = sm + ring[1];
    const double* X2 = sm + ring[2];
    const double* EE = sm + L.ee;
    for (int b = tid; b < (d + 1) / 2; b += T) {
      const U4 w = draw_block(fd, kRngInnov, (uint32_t)n, epoch, (uint32_t)b);
      double z0, z1;
      normal_pair(w, z0, z1);
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * b + h;
        if (i >= d) break;
        const double v = sqrt(fd.kappa * EE[i]) * (h == 0 ? z0 : z1);
        const int64_t o = (int64_t)i * N + n;
        const double xv = X0[i] + v;
        X0[i] = xv;
        dst.x[o] = xv;
        dst.h1[o] = X1[i] + v;
        dst.h2[o] = X2[i] + v;
      }
    }
    __syncthreads();
    double lwn = -CUDART_INF, bad = 0.0;
    if (tid == 0) {
      // Step 5: new log weight
      lwn = ad_loglik(fd, ep, X0) - fd.ll1[l];
      if (!finite_bits(lwn)) {
        lwn = -CUDART_INF;
        bad = 1.0;
      }
      dst.lw[n] = lwn;
    }
    stage2_tail(fd, epoch, lwn, bad, (int)blockIdx.x, (int)gridDim.x, s_red, &s_flag);
  }
}

// Threads per block for a grid side: the DFT passes have nt*H outputs and the
// pointwise passes d; pick the multiple of 32 (64..512) with the fewest idle
// lane-cycles, counting the ~10 nt-long sums of a spectral output against the
// ~(2H + 9) of a pointwise one, and one barrier round each.
int ad_threads(int nt) {
  const int H = (nt + 1) / 2, d = nt * nt, spec = nt * H;
  int best = 64;
  double best_cost = 1e300;
  for (int T = 64; T <= 512; T += 32) {
    const int rs = (spec + T - 1) / T, rp = (d + T - 1) / T;
    const double cost = (double)rs * T * (10.0 * nt) + (double)rp * T * (2.0 * H + 9.0) +
                        (double)(3 * rs + 2 * rp) * 32.0 * 40.0;
    if (cost < best_cost) {
      best_cost = cost;
      best = T;
    }
  }
  return best;
}

size_t ad_stage_smem(int d, int S, int stage) {
  return sizeof(double) * (size_t)ad_layout(d, S, stage == 2).total;
}

cudaError_t launch_ad_stage(int stage, const FilterDev& fd, const EpochParams* ep, int S,
                            cudaStream_t st) {
  const int nt = ad_side(fd.d);
  if (nt == 0) return cudaErrorInvalidValue;
  const size_t smem = ad_stage_smem(fd.d, S, stage);
  const int T = ad_threads(nt);
  const void* k = stage == 1 ? (const void*)k_adstage<1> : (const void*)k_adstage<2>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (stage == 1) k_adstage<1><<<(unsigned)fd.N, T, smem, st>>>(fd, ep);
  else k_adstage<2><<<(unsigned)fd.N, T, smem, st>>>(fd, ep);
  return cudaGetLastError();
}

cudaError_t preload_ad_kernels() {
  const void* ks[] = {(const void*)k_adstage<1>, (const void*)k_adstage<2>};
  for (const void* k : ks) {
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pfg
