// pf_advdiff.cu -- stage kernels of the epoch for the paper's 2D
// advection-diffusion system (Sec. 4): U' = L U on the periodic nt x nt grid,
//   L = -{k1^2 B1'B1 + k1 k3 (B1'B2 + B2'B1) + (k2^2 + k3^2) B2'B2} + c1 B1 + c2 B2,
// B1 = I (x) ell, B2 = ell (x) I, (ell u)_j = u_j - u_{j-1} (periodic), state
// U[iy*nt + ix], theta = (k1, k2, k3, c1, c2).
//
// L is built from circulant difference matrices, so the 2D DFT diagonalises
// it: with a(m) = 1 - exp(-2 pi i m / nt) the symbol of ell,
//   lambda(mx, my) = -(k1^2 |a_x|^2 + 2 k1 k3 Re(conj(a_x) a_y) + (k2^2 + k3^2) |a_y|^2)
//                    + c1 a_x + c2 a_y.
// The system is linear, so Newton's method with the exact Jacobian L solves
// each implicit BDF step in one iteration (Sec. 2.1), and the solution of
//   x_{n+1} - rho1 x_n - rho2 x_{n-1} = gamma L x_{n+1}
// is, mode by mode, X_{n+1} = (rho1 X_n + rho2 X_{n-1}) / (1 - gamma lambda).
// Every quantity of an interval's S substeps is a fixed linear combination of
// the modes of (x_n, x_{n-1}, x_{n-2}): the predictor pi0 X_n + pi1 X_{n-1} +
// pi2 X_{n-2}, the explicit-Euler predictor (1 + h lambda) X_n of a cold
// start, the corrector, and Milne's estimate mu (X_{n+1} - X_p).  So each
// particle's history is transformed once at the interval's start and stays in
// the Fourier basis, each thread stepping its own modes in registers through
// all S substeps; only what is needed in physical space is transformed back:
// the final states, and in stage 2 each substep's local error, whose squares
// are summed per grid point (Step 4b: Gamma = kappa diag(sum_s e_s^2)).
//
// Transforms.  nt is odd and the state real, so the half spectrum mx =
// 0..H-1, H = (nt+1)/2, carries everything.  The transforms are direct sums
// over a cos/sin table (nt is small and prime or nearly so), organised by
// the symmetry of the twiddles: the DFT terms of indices m and nt - m share
// their cosine and have opposite sines, so
//   sum_m z_m e^{+i phi m k} = z_0 + sum_{m=1}^{H-1} [(z_m + z_{nt-m}) cos(phi m k)
//                                              + i (z_m - z_{nt-m}) sin(phi m k)],
// and the outputs k and nt - k differ only in the sign of the sine part.
// One work unit computes such an output pair from the sum and difference
// of an input pair: 4 (H-1) FMAs for two complex outputs instead of 8 nt.
// A thread owns the mode pairs (my, mx) and (nt - my, mx) of its units, in
// registers, so the forward transform ends and the inverse begins in the
// owning thread.
//
// A block advances PB particles (1, 2 or 4: on small grids several
// particles fill the block's warps), all in step through the same substeps.
// Shared memory holds the substep table and the twiddle table, and per
// particle the physical states, the pair buffers of the transforms and in
// stage 2 the error sums.  Global memory is touched once per particle per
// stage.
#include "pf_epoch.cuh"
#include "pf_kernels.h"

namespace pfg {

constexpr int kAdMaxSide = 45;
constexpr int kAdScDoubles = (int)(sizeof(StepCoef) / sizeof(double));
constexpr int kAdMaxUnitsPerThread = 2;  // mode-pair units a thread steps in registers

__host__ __device__ inline int ad_side(int d) {
  for (int nt = 3; nt <= kAdMaxSide; nt += 2)
    if (nt * nt == d) return nt;
  return 0;
}

// Shared-memory layout of one block, in doubles: the substep table and the
// twiddle table, then one region per particle of the block.
struct AdLayout {
  int nt, d, H, PB;
  int sc;    // step table, S entries
  int tw;    // cos(2 pi k / nt), then sin(2 pi k / nt), k < nt
  int base;  // particle 0's region; particle q's is at base + q * per
  int per;   // doubles per particle region
  // offsets within a particle's region:
  int X[3];  // physical x_n, x_{n-1}, x_{n-2}
  int ps;    // pair sums [p][mx] (complex), p < H; p = 0 holds the unpaired entry
  int pd;    // pair differences [p][mx] (complex)
  int cy;    // inverse columns [iy][mx] (complex), iy < nt
  int ee;    // stage 2: error sums per grid point
  int total;
};

__host__ __device__ inline AdLayout ad_layout(int d, int S, bool err, int PB) {
  AdLayout L;
  L.nt = ad_side(d);
  L.d = d;
  L.H = (L.nt + 1) / 2;
  L.PB = PB;
  int off = 0;
  L.sc = off;
  off += S * kAdScDoubles;
  L.tw = off;
  off += 2 * L.nt;
  L.base = off;
  int r = 0;
  for (int k = 0; k < 3; ++k) {
    L.X[k] = r;
    r += d;
  }
  L.ps = r;
  r += 2 * L.H * L.H;
  L.pd = r;
  r += 2 * L.H * L.H;
  L.cy = r;
  r += 2 * L.nt * L.H;
  L.ee = r;
  r += err ? d : 0;
  L.per = r;
  L.total = off + PB * r;
  return L;
}

// The operator's Fourier symbol for one parameter vector.
struct AdOp {
  double kxx, kxy, kyy, c1, c2;  // k1^2, k1 k3, k2^2 + k3^2, c1, c2
};

__device__ __forceinline__ AdOp ad_op(const double* th) {
  const double k1 = th[0], k2 = th[1], k3 = th[2];
  AdOp o;
  o.kxx = k1 * k1;
  o.kxy = k1 * k3;
  o.kyy = fma(k2, k2, k3 * k3);
  o.c1 = th[3];
  o.c2 = th[4];
  return o;
}

// lambda(mx, my)
__device__ __forceinline__ void ad_lambda(const AdLayout& L, const AdOp& o, const double* tw, int my,
                                          int mx, double& lr, double& li) {
  const int nt = L.nt;
  const double axr = 1.0 - tw[mx], axi = tw[nt + mx];
  const double ayr = 1.0 - tw[my], ayi = tw[nt + my];
  const double ax2 = fma(axr, axr, axi * axi), ay2 = fma(ayr, ayr, ayi * ayi);
  const double cr = fma(axr, ayr, axi * ayi);
  lr = fma(o.c1, axr, o.c2 * ayr) - fma(o.kxx, ax2, fma(2.0 * o.kxy, cr, o.kyy * ay2));
  li = fma(o.c1, axi, o.c2 * ayi);
}

// A thread's modes: work item t = q * H^2 + p * H + mx (particle q of the
// block) holds mode A = (my = p, mx) and, for p >= 1, mode B = (my = nt - p,
// mx).  Index [j][0] is A, [j][1] is B, for the items t = tid + j T.
template <int U>
struct Modes {
  double re[U][2], im[U][2];
};

// Forward real 2D DFT of state k of every particle of the block (physical,
// shared) into the calling thread's own modes:
// X(my, mx) = sum_{iy,ix} u[iy][ix] exp(-i phi (mx ix + my iy)).
// Ends with a barrier.
template <int U>
__device__ void ad_forward(const AdLayout& L, const double* tw, double* sm, int k_state,
                           Modes<U>& out) {
  const int nt = L.nt, H = L.H, T = blockDim.x, tid = threadIdx.x, units = H * H;
  const int items = L.PB * units;
  // rows py and nt - py at column mx, stored as their sum and difference
  for (int t = tid; t < items; t += T) {
    const int q = t / units, v = t - q * units;
    double* R = sm + L.base + q * L.per;
    const double* u = R + L.X[k_state];
    double* ps = R + L.ps;
    double* pd = R + L.pd;
    const int py = v / H, mx = v - py * H;
    const double* g1 = u + py * nt;
    const double* g2 = u + (py == 0 ? 0 : nt - py) * nt;
    double r1 = 0.0, i1 = 0.0, r2 = 0.0, i2 = 0.0;
    int k = 0;
    for (int ix = 0; ix < nt; ++ix) {
      const double cs = tw[k], sn = tw[nt + k];
      r1 = fma(g1[ix], cs, r1);
      i1 = fma(-g1[ix], sn, i1);
      r2 = fma(g2[ix], cs, r2);
      i2 = fma(-g2[ix], sn, i2);
      k += mx;
      if (k >= nt) k -= nt;
    }
    if (py == 0) {
      ps[2 * v] = r1;
      ps[2 * v + 1] = i1;
    } else {
      ps[2 * v] = r1 + r2;
      ps[2 * v + 1] = i1 + i2;
      pd[2 * v] = r1 - r2;
      pd[2 * v + 1] = i1 - i2;
    }
  }
  __syncthreads();
  // columns: X(my) = R0 + sum_{iy=1}^{H-1} [s_iy cos(phi my iy) - i d_iy sin(phi my iy)]
  // for my = p, and the conjugate sine part for my = nt - p
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int t = tid + j * T;
    double cr = 0.0, ci = 0.0, dr = 0.0, di = 0.0;
    if (t < items) {
      const int q = t / units, v = t - q * units;
      const double* R = sm + L.base + q * L.per;
      const double* ps = R + L.ps;
      const double* pd = R + L.pd;
      const int p = v / H, mx = v - p * H;
      cr = ps[2 * mx];
      ci = ps[2 * mx + 1];
      int k = p;
      for (int iy = 1; iy < H; ++iy) {
        const int o = 2 * (iy * H + mx);
        const double cs = tw[k], sn = tw[nt + k];
        cr = fma(ps[o], cs, cr);
        ci = fma(ps[o + 1], cs, ci);
        dr = fma(pd[o], sn, dr);
        di = fma(pd[o + 1], sn, di);
        k += p;
        if (k >= nt) k -= nt;
      }
    }
    // A: C - i D, B: C + i D
    out.re[j][0] = cr + di;
    out.im[j][0] = ci - dr;
    out.re[j][1] = cr - di;
    out.im[j][1] = ci + dr;
  }
  __syncthreads();
}

// Inverse: the threads' modes z (already scaled) give, per particle q,
//   u[iy][ix] = sum over all modes z exp(+i phi (mx ix + my iy))
// (Hermitian in mx), delivered per grid point to `out(q, i, value)`.  Ends
// with a barrier.
template <int U, class Out>
__device__ void ad_inverse(const AdLayout& L, const double* tw, double* sm, const Modes<U>& z, Out out) {
  const int nt = L.nt, H = L.H, T = blockDim.x, tid = threadIdx.x, units = H * H;
  const int items = L.PB * units;
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int t = tid + j * T;
    if (t < items) {
      const int q = t / units, v = t - q * units;
      double* R = sm + L.base + q * L.per;
      double* ps = R + L.ps;
      double* pd = R + L.pd;
      if (v < H) {  // p = 0: the unpaired my = 0
        ps[2 * v] = z.re[j][0];
        ps[2 * v + 1] = z.im[j][0];
      } else {
        ps[2 * v] = z.re[j][0] + z.re[j][1];
        ps[2 * v + 1] = z.im[j][0] + z.im[j][1];
        pd[2 * v] = z.re[j][0] - z.re[j][1];
        pd[2 * v + 1] = z.im[j][0] - z.im[j][1];
      }
    }
  }
  __syncthreads();
  // columns: Y(iy) = Z0 + sum_{m=1}^{H-1} [s_m cos(phi m iy) + i d_m sin(phi m iy)]
  // for iy = py, and the conjugate sine part for iy = nt - py
  for (int t = tid; t < items; t += T) {
    const int q = t / units, v = t - q * units;
    double* R = sm + L.base + q * L.per;
    const double* ps = R + L.ps;
    const double* pd = R + L.pd;
    double* cy = R + L.cy;
    const int py = v / H, mx = v - py * H;
    double cr = ps[2 * mx], ci = ps[2 * mx + 1], dr = 0.0, di = 0.0;
    int k = py;
    for (int m = 1; m < H; ++m) {
      const int o = 2 * (m * H + mx);
      const double cs = tw[k], sn = tw[nt + k];
      cr = fma(ps[o], cs, cr);
      ci = fma(ps[o + 1], cs, ci);
      dr = fma(pd[o], sn, dr);
      di = fma(pd[o + 1], sn, di);
      k += py;
      if (k >= nt) k -= nt;
    }
    cy[2 * (py * H + mx)] = cr - di;
    cy[2 * (py * H + mx) + 1] = ci + dr;
    if (py > 0) {
      cy[2 * ((nt - py) * H + mx)] = cr + di;
      cy[2 * ((nt - py) * H + mx) + 1] = ci - dr;
    }
  }
  __syncthreads();
  // rows (Hermitian in mx): u[px] = Re Y0 + 2 (A - B), u[nt - px] = Re Y0 + 2 (A + B),
  // A = sum_{mx>=1} Re Y cos(phi mx px), B = sum_{mx>=1} Im Y sin(phi mx px)
  const int rows = nt * H;
  for (int t = tid; t < L.PB * rows; t += T) {
    const int q = t / rows, v = t - q * rows;
    const double* cy = sm + L.base + q * L.per + L.cy;
    const int iy = v / H, px = v - iy * H;
    const double* y = cy + 2 * iy * H;
    double a = 0.0, b = 0.0;
    int k = px;
    for (int mx = 1; mx < H; ++mx) {
      a = fma(y[2 * mx], tw[k], a);
      b = fma(y[2 * mx + 1], tw[nt + k], b);
      k += px;
      if (k >= nt) k -= nt;
    }
    out(q, iy * nt + px, fma(2.0, a - b, y[0]));
    if (px > 0) out(q, iy * nt + nt - px, fma(2.0, a + b, y[0]));
  }
  __syncthreads();
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

// complex a * b
__device__ __forceinline__ void cmul(double ar, double ai, double br, double bi, double& r, double& i) {
  r = fma(ar, br, -ai * bi);
  i = fma(ar, bi, ai * br);
}

// One block advances PB particles (PB > 1 fills the warps on small grids);
// U = 2 serves grids of more than 512 units (nt = 45), at most 288 threads.
template <int STAGE, int U, int PB>
__global__ void __launch_bounds__(U == 1 ? 512 : 384, 1) k_adstage(const __grid_constant__ FilterDev fd,
                                                                   const EpochParams* __restrict__ ep) {
  extern __shared__ double s_dyn[];
  __shared__ double s_red[32];
  __shared__ double s_th[PB][kPMax];
  __shared__ int s_flag;
  const Ctrl* ctrl = fd.ctrl;
  if (ctrl->status != PF_OK) return;
  const int S = ep->S;
  const AdLayout L = ad_layout(fd.d, S, STAGE == 2, PB);
  double* sm = s_dyn;
  load_steps(reinterpret_cast<StepCoef*>(sm + L.sc), ep, S);  // ends with a barrier
  const StepCoef* sc = reinterpret_cast<const StepCoef*>(sm + L.sc);
  const int cur = ctrl->cur;
  const Ensemble src = committed(fd, cur);
  const Ensemble dst = pending(fd, cur);
  const int64_t N = fd.N;
  const int64_t n0 = (int64_t)blockIdx.x * PB;  // the block's first particle
  const uint32_t epoch = ep->epoch;
  const int d = L.d, nt = L.nt, H = L.H, T = blockDim.x, tid = threadIdx.x, units = H * H;
  const double inv_d = 1.0 / (double)d;
  // particle q of the block is n0 + q, gathered from slot l (stage 2: the
  // resampled parent); slots past N are idle and stay zero
  auto slot_of = [&](int q) -> int64_t { return STAGE == 2 ? (int64_t)fd.idx[n0 + q] : n0 + q; };
  if (tid < PB) {
    const int q = tid;
    const int64_t n = n0 + q;
    double ph[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (n < N) {
      const int64_t l = slot_of(q);
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
    }
    for (int i = 0; i < 5; ++i) s_th[q][i] = (fd.transform == PF_TRANSFORM_LOG) ? exp(ph[i]) : ph[i];
  }
  ad_tables(L, sm);
  for (int t = tid; t < PB * d; t += T) {
    const int q = t / d, i = t - q * d;
    double* R = sm + L.base + q * L.per;
    double x0 = 0.0, x1 = 0.0, x2 = 0.0;
    if (n0 + q < N) {
      const int64_t o = (int64_t)i * N + slot_of(q);
      x0 = src.x[o];
      x1 = src.h1[o];
      x2 = src.h2[o];
    }
    R[L.X[0] + i] = x0;
    R[L.X[1] + i] = x1;
    R[L.X[2] + i] = x2;
    if (STAGE == 2) R[L.ee + i] = 0.0;
  }
  __syncthreads();
  const double* tw = sm + L.tw;

  // the history in the Fourier basis, each thread holding its own mode pairs
  Modes<U> x0, x1, x2;
  ad_forward<U>(L, tw, sm, 0, x0);
  ad_forward<U>(L, tw, sm, 1, x1);
  ad_forward<U>(L, tw, sm, 2, x2);
  double lr[U][2], li[U][2];
#pragma unroll
  for (int j = 0; j < U; ++j) {
    const int t = tid + j * T;
    lr[j][0] = li[j][0] = lr[j][1] = li[j][1] = 0.0;
    if (t < PB * units) {
      const int q = t / units, v = t - q * units;
      const int p = v / H, mx = v - p * H;
      const AdOp op = ad_op(s_th[q]);
      ad_lambda(L, op, tw, p, mx, lr[j][0], li[j][0]);
      if (p > 0) ad_lambda(L, op, tw, nt - p, mx, lr[j][1], li[j][1]);
    }
  }

  // Psi over the S substeps (Steps 2 and 4b/4d), mode by mode
  double wr[U][2], wi[U][2];
  double gamma_w = CUDART_NAN;
  for (int s = 0; s < S; ++s) {
    const StepCoef c = sc[s];
    if (!(c.gamma == gamma_w)) {
      // w = 1 / (1 - gamma lambda) per mode
#pragma unroll
      for (int j = 0; j < U; ++j)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const double p = fma(-c.gamma, lr[j][b], 1.0), q = -c.gamma * li[j][b];
          const double inv = 1.0 / fma(p, p, q * q);
          wr[j][b] = p * inv;
          wi[j][b] = -q * inv;
        }
      gamma_w = c.gamma;
    }
    Modes<U> e;
#pragma unroll
    for (int j = 0; j < U; ++j)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        double rr, ri, pr = 0.0, pi = 0.0;
        if (c.kind == 2) {
          rr = fma(c.rho2, x1.re[j][b], c.rho1 * x0.re[j][b]);
          ri = fma(c.rho2, x1.im[j][b], c.rho1 * x0.im[j][b]);
          if (STAGE == 2) {
            pr = fma(c.pi2, x2.re[j][b], fma(c.pi1, x1.re[j][b], c.pi0 * x0.re[j][b]));
            pi = fma(c.pi2, x2.im[j][b], fma(c.pi1, x1.im[j][b], c.pi0 * x0.im[j][b]));
          }
        } else {
          // BDF1 (cold start): r = x_n; error predictor x_n + h L x_n
          rr = x0.re[j][b];
          ri = x0.im[j][b];
          if (STAGE == 2) {
            double gr, gi;
            cmul(c.h * lr[j][b], c.h * li[j][b], x0.re[j][b], x0.im[j][b], gr, gi);
            pr = x0.re[j][b] + gr;
            pi = x0.im[j][b] + gi;
          }
        }
        double yr, yi;
        cmul(rr, ri, wr[j][b], wi[j][b], yr, yi);
        if (STAGE == 2) {
          // Milne's estimate, with the inverse transform's 1/d
          const double f = c.mu * inv_d;
          e.re[j][b] = f * (yr - pr);
          e.im[j][b] = f * (yi - pi);
        }
        x2.re[j][b] = x1.re[j][b];
        x2.im[j][b] = x1.im[j][b];
        x1.re[j][b] = x0.re[j][b];
        x1.im[j][b] = x0.im[j][b];
        x0.re[j][b] = yr;
        x0.im[j][b] = yi;
      }
    if (STAGE == 2) {
      ad_inverse<U>(L, tw, sm, e, [&](int q, int i, double v) {
        double* EE = sm + L.base + q * L.per + L.ee;
        EE[i] = fma(v, v, EE[i]);
      });
    }
  }

  // back to physical space (scaled by 1/d)
  auto back = [&](Modes<U>& z, int k_state) {
#pragma unroll
    for (int j = 0; j < U; ++j)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        z.re[j][b] *= inv_d;
        z.im[j][b] *= inv_d;
      }
    ad_inverse<U>(L, tw, sm, z, [&](int q, int i, double v) {
      sm[L.base + q * L.per + L.X[k_state] + i] = v;
    });
  };
  back(x0, 0);
  if (STAGE == 1) {
    double lg = -CUDART_INF;
    if (tid < PB && n0 + tid < N) {
      const int64_t n = n0 + tid;
      const double ll = ad_loglik(fd, ep, sm + L.base + tid * L.per + L.X[0]);
      fd.ll1[n] = ll;
      lg = (src.lw[n] - ctrl->logW) + ll;
      if (!finite_bits(lg)) lg = -CUDART_INF;
      fd.lg[n] = lg;
    }
    stage1_tail(fd, epoch, lg, (int)blockIdx.x, (int)gridDim.x, s_red, &s_flag);
  } else {
    back(x1, 1);
    back(x2, 2);
    // Steps 4c, 4d: innovation v = sqrt(kappa E) z', written in (x, h1, h2) order
    const int halves = (d + 1) / 2;
    for (int t = tid; t < PB * halves; t += T) {
      const int q = t / halves, b = t - q * halves;
      const int64_t n = n0 + q;
      if (n >= N) continue;
      double* R = sm + L.base + q * L.per;
      const U4 w = draw_block(fd, kRngInnov, (uint32_t)n, epoch, (uint32_t)b);
      double z0, z1;
      normal_pair(w, z0, z1);
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * b + h;
        if (i >= d) break;
        const double v = sqrt(fd.kappa * R[L.ee + i]) * (h == 0 ? z0 : z1);
        const int64_t o = (int64_t)i * N + n;
        const double xv = R[L.X[0] + i] + v;
        R[L.X[0] + i] = xv;
        dst.x[o] = xv;
        dst.h1[o] = R[L.X[1] + i] + v;
        dst.h2[o] = R[L.X[2] + i] + v;
      }
    }
    __syncthreads();
    double lwn = -CUDART_INF, bad = 0.0;
    if (tid < PB && n0 + tid < N) {
      // Step 5: new log weight
      const int64_t n = n0 + tid;
      lwn = ad_loglik(fd, ep, sm + L.base + tid * L.per + L.X[0]) - fd.ll1[slot_of(tid)];
      if (!finite_bits(lwn)) {
        lwn = -CUDART_INF;
        bad = 1.0;
      }
      dst.lw[n] = lwn;
    }
    stage2_tail(fd, epoch, lwn, bad, (int)blockIdx.x, (int)gridDim.x, s_red, &s_flag);
  }
}

// Launch shape for a grid side and stage: particles per block PB and units
// (mode pairs) per thread U, and threads per block, a multiple of 32
// covering PB H^2 units.  PB (1, 2 or 4) wastes the fewest lanes in the unit
// and row passes while the block keeps at least two blocks per SM resident
// (stage 2 keeps more registers per thread: at most 288 threads); U = 2 only
// where one particle's units exceed 512.
static void ad_shape(int nt, int stage, int* threads, int* upt, int* pb) {
  const int H = (nt + 1) / 2, units = H * H;
  const int cap = stage == 2 ? 288 : 512;
  int u = 1;
  while (u < kAdMaxUnitsPerThread && (units + u - 1) / u > 512) u *= 2;
  int best_pb = 1, best_T = 0;
  double best_eff = -1.0;
  for (int p = 1; p <= 4; p *= 2) {
    if (u > 1 && p > 1) break;
    const int need = (p * units + u - 1) / u;
    const int T = ((need > 64 ? need : 64) + 31) / 32 * 32;
    if (p > 1 && T > cap) break;
    // lane efficiency of the unit passes and of the row passes
    const double e_units = (double)(p * units) / (double)(((p * units + T - 1) / T) * T);
    const double e_rows = (double)(p * nt * H) / (double)(((p * nt * H + T - 1) / T) * T);
    const double eff = 0.7 * e_units + 0.3 * e_rows;
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best_pb = p;
      best_T = T;
    }
  }
  *upt = u;
  *pb = best_pb;
  *threads = best_T;
}

int ad_threads(int nt) {
  int T, u, pb;
  ad_shape(nt, 2, &T, &u, &pb);
  return T;
}

size_t ad_stage_smem(int d, int S, int stage) {
  int T, u, pb;
  ad_shape(ad_side(d), stage, &T, &u, &pb);
  return sizeof(double) * (size_t)ad_layout(d, S, stage == 2, pb).total;
}

cudaError_t launch_ad_stage(int stage, const FilterDev& fd, const EpochParams* ep, int S,
                            cudaStream_t st) {
  const int nt = ad_side(fd.d);
  if (nt == 0) return cudaErrorInvalidValue;
  int T, upt, pb;
  ad_shape(nt, stage, &T, &upt, &pb);
  const size_t smem = sizeof(double) * (size_t)ad_layout(fd.d, S, stage == 2, pb).total;
  const int H = (nt + 1) / 2;
  if (T * upt < pb * H * H || T > (upt == 1 ? 512 : 384)) return cudaErrorInvalidValue;
  using K = void (*)(const FilterDev, const EpochParams*);
  K k;
  if (upt == 2) k = stage == 1 ? k_adstage<1, 2, 1> : k_adstage<2, 2, 1>;
  else if (pb == 4) k = stage == 1 ? k_adstage<1, 1, 4> : k_adstage<2, 1, 4>;
  else if (pb == 2) k = stage == 1 ? k_adstage<1, 1, 2> : k_adstage<2, 1, 2>;
  else k = stage == 1 ? k_adstage<1, 1, 1> : k_adstage<2, 1, 1>;
  cudaError_t e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((fd.N + pb - 1) / pb);
  k<<<blocks, T, smem, st>>>(fd, ep);
  return cudaGetLastError();
}

cudaError_t preload_ad_kernels() {
  const void* ks[] = {(const void*)k_adstage<1, 1, 1>, (const void*)k_adstage<2, 1, 1>,
                      (const void*)k_adstage<1, 1, 2>, (const void*)k_adstage<2, 1, 2>,
                      (const void*)k_adstage<1, 1, 4>, (const void*)k_adstage<2, 1, 4>,
                      (const void*)k_adstage<1, 2, 1>, (const void*)k_adstage<2, 2, 1>};
  for (const void* k : ks) {
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pfg
