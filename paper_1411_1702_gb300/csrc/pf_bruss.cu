// pf_bruss.cu -- stage kernels of the epoch for the 1D Brusselator (d = 64):
// 32 interior grid points xi_i = i/33, Dirichlet u = 1, v = 3 at both ends,
//   u_i' = A + u_i^2 v_i - (B+1) u_i + D (u_{i-1} - 2 u_i + u_{i+1}),
//   v_i' = B u_i - u_i^2 v_i + D (v_{i-1} - 2 v_i + v_{i+1}),  D = alpha 33^2,
// state interleaved (u_0, v_0, u_1, v_1, ...), theta = (A, B, alpha).
//
// One particle per thread, as for the small models: the FP64 pipe is the
// limit on GB300, so the Newton system is solved with the fewest FP64 operations
// -- an exact block Thomas sweep over the 2x2 blocks of the block-tridiagonal
// I - gamma J (off-diagonal blocks -gamma D I) -- rather than a warp-parallel
// cyclic reduction, which would multiply the arithmetic several times over.
// The particle's vectors live in HBM as structure-of-arrays (component-major,
// coalesced across the warp): the rotating history x_n, x_{n-1}, x_{n-2} in the
// pending ensemble buffer, and r, the error predictor, the error sums and the
// sweep's inverted pivot blocks and intermediate solutions (6 doubles per grid
// point, read back in reverse by the backward pass) in a work area.  Keeping
// the sweep out of shared memory lets registers, not shared memory, set the
// residency, so each SM sub-partition interleaves several particles' sweeps
// and hides the latency of the block recurrence.
#include "pf_epoch.cuh"
#include "pf_kernels.h"

namespace pfg {

constexpr int kBrPts = 32;
constexpr int kBrD = 64;
constexpr int kBrThreads = 64;
// work area per particle (doubles, each array component-major over N):
// r (64), error predictor (64), error sums (64), pivot inverses W (32 x 4),
// sweep solutions z (32 x 2)
constexpr int kBrWorkRows = 3 * kBrD + kBrPts * 6;

struct BrTheta {
  double A, B, D;
};

__device__ __forceinline__ BrTheta br_theta(const double* th) {
  return BrTheta{th[0], th[1], th[2] * 33.0 * 33.0};
}

// x_EE = x + h f(x) for the BDF1 error predictor
__device__ void br_euler_predictor(const double* __restrict__ X, double* __restrict__ XP, int64_t N,
                                   int64_t n, double h, const BrTheta& T) {
  double uL = 1.0, vL = 3.0, u = X[n], v = X[N + n];
  for (int i = 0; i < kBrPts; ++i) {
    double uR = 1.0, vR = 3.0;
    if (i < kBrPts - 1) {
      uR = X[(int64_t)(2 * i + 2) * N + n];
      vR = X[(int64_t)(2 * i + 3) * N + n];
    }
    const double uuv = u * u * v;
    const double fu = fma(T.D, (uL - 2.0 * u) + uR, fma(-(T.B + 1.0), u, T.A + uuv));
    const double fv = fma(T.D, (vL - 2.0 * v) + vR, fma(T.B, u, -uuv));
    XP[(int64_t)(2 * i) * N + n] = fma(h, fu, u);
    XP[(int64_t)(2 * i + 1) * N + n] = fma(h, fv, v);
    uL = u;
    vL = v;
    u = uR;
    v = vR;
  }
}

// K Newton iterations on y (in place): (I - g J(y)) dy = -G(y),
// G = y - r - g f(y), with M_i the 2x2 diagonal block of point i and e = g D:
//   forward  W_i = (M_i - e^2 W_{i-1})^{-1},  z_i = W_i (-G_i + e z_{i-1}),
//   backward dy_i = z_i + e W_i dy_{i+1}  (dy_32 = 0).
// R holds r with g A already added to the u rows (br_propagate), and the
// Laplacian's -2u, -2v terms are gathered into the diagonal coefficients, so
//   G_u = (1 + g(B+1) + 2gD) u - (r_u + gA) - g u^2 v - gD (u_L + u_R),
//   G_v = (1 + 2gD) v - r_v - gB u + g u^2 v - gD (v_L + v_R):
// the same residual in 9 FP64 instructions a point instead of 13.
__device__ void br_newton(double* __restrict__ Y, const double* __restrict__ R, int64_t N, int64_t n,
                          double g, int K, const BrTheta& T, double* __restrict__ Wg,
                          double* __restrict__ Zg) {
  const double gD = g * T.D, e2 = gD * gD, g2 = 2.0 * g, mg = -g;
  const double ca = 1.0 + g * (T.B + 1.0) + 2.0 * gD;  // 1 + g(B+1) + 2gD
  const double cd = 1.0 + 2.0 * gD;
  const double gB = g * T.B;
  // one iteration; the determinants' reciprocals are refined only in the last
  auto step = [&](const bool last) {
    double uL = 1.0, vL = 3.0;
    double u = Y[n], v = Y[N + n];
    double W00 = 0.0, W01 = 0.0, W10 = 0.0, W11 = 0.0, z0 = 0.0, z1 = 0.0;
    for (int i = 0; i < kBrPts; ++i) {
      double uR = 1.0, vR = 3.0;
      if (i < kBrPts - 1) {
        uR = Y[(int64_t)(2 * i + 2) * N + n];
        vR = Y[(int64_t)(2 * i + 3) * N + n];
      }
      const double ru = R[(int64_t)(2 * i) * N + n], rv = R[(int64_t)(2 * i + 1) * N + n];
      const double uu = u * u, uv = u * v, uuv = uu * v;
      const double Gu = fma(ca, u, fma(mg, uuv, fma(-gD, uL + uR, -ru)));
      const double Gv = fma(cd, v, fma(g, uuv, fma(-gB, u, fma(-gD, vL + vR, -rv))));
      double a = fma(-g2, uv, ca), b = mg * uu, c = fma(g2, uv, -gB), d = fma(g, uu, cd);
      a = fma(-e2, W00, a);
      b = fma(-e2, W01, b);
      c = fma(-e2, W10, c);
      d = fma(-e2, W11, d);
      const double rdet = rcp_newton(fma(a, d, -(b * c)), last);
      W00 = d * rdet;
      W01 = -b * rdet;
      W10 = -c * rdet;
      W11 = a * rdet;
      const double h0 = fma(gD, z0, -Gu), h1 = fma(gD, z1, -Gv);
      z0 = fma(W00, h0, W01 * h1);
      z1 = fma(W10, h0, W11 * h1);
      double* w = Wg + (int64_t)(i * 4) * N + n;
      w[0] = W00;
      w[N] = W01;
      w[2 * N] = W10;
      w[3 * N] = W11;
      double* zz = Zg + (int64_t)(i * 2) * N + n;
      zz[0] = z0;
      zz[N] = z1;
      uL = u;
      vL = v;
      u = uR;
      v = vR;
    }
    double du = 0.0, dv = 0.0;
    for (int i = kBrPts - 1; i >= 0; --i) {
      const double* w = Wg + (int64_t)(i * 4) * N + n;
      const double* zz = Zg + (int64_t)(i * 2) * N + n;
      const double t0 = fma(w[0], du, w[N] * dv);
      const double t1 = fma(w[2 * N], du, w[3 * N] * dv);
      du = fma(gD, t0, zz[0]);
      dv = fma(gD, t1, zz[N]);
      Y[(int64_t)(2 * i) * N + n] += du;
      Y[(int64_t)(2 * i + 1) * N + n] += dv;
    }
  };
  for (int it = 0; it + 1 < K; ++it) step(false);
  if (K > 0) step(true);
}

// Psi over the S substeps.  P0, P1, P2 hold x_n, x_{n-1}, x_{n-2}; each
// substep writes its iterate over x_{n-2} and the roles rotate.
template <bool ERR>
__device__ void br_propagate(const FilterDev& fd, int64_t n, const StepCoef* sc, int S, int K,
                             const BrTheta& T, double*& P0, double*& P1, double*& P2) {
  const int64_t N = fd.N;
  double* R = fd.wk;
  double* XP = fd.wk + (int64_t)kBrD * N;
  double* EE = fd.wk + 2 * (int64_t)kBrD * N;
  double* Wg = fd.wk + 3 * (int64_t)kBrD * N;
  double* Zg = Wg + 4 * (int64_t)kBrPts * N;
  for (int s = 0; s < S; ++s) {
    const StepCoef& c = sc[s];
    // r, with gamma A added to the u rows for br_newton's residual
    const double gA = c.gamma * T.A;
    if (c.kind == 2) {
      for (int k = 0; k < kBrD; ++k) {
        const int64_t o = (int64_t)k * N + n;
        const double xn = P0[o], x1 = P1[o], x2 = P2[o];
        const double xp = fma(c.pi2, x2, fma(c.pi1, x1, c.pi0 * xn));
        R[o] = fma(c.rho2, x1, fma(c.rho1, xn, (k & 1) ? 0.0 : gA));
        P2[o] = xp;
        if (ERR) XP[o] = xp;
      }
    } else {
      if (ERR) br_euler_predictor(P0, XP, N, n, c.h, T);
      for (int k = 0; k < kBrD; ++k) {
        const int64_t o = (int64_t)k * N + n;
        const double xn = P0[o];
        R[o] = (k & 1) ? xn : xn + gA;
        P2[o] = xn;
      }
    }
    br_newton(P2, R, N, n, c.gamma, K, T, Wg, Zg);
    if (ERR) {
      for (int k = 0; k < kBrD; ++k) {
        const int64_t o = (int64_t)k * N + n;
        const double e = c.mu * (P2[o] - XP[o]);
        EE[o] = fma(e, e, EE[o]);
      }
    }
    double* t = P2;
    P2 = P1;
    P1 = P0;
    P0 = t;
  }
}

__device__ __forceinline__ double br_loglik(const FilterDev& fd, const EpochParams* __restrict__ ep,
                                            const double* X, int64_t n) {
  double s = 0.0;
  for (int i = 0; i < fd.m; ++i) {
    const double z = (ep->y[i] - X[(int64_t)fd.obs[i] * fd.N + n]) * ep->inv_sigma[i];
    s = fma(z, z, s);
  }
  return -0.5 * s;
}

__device__ __forceinline__ void bstage1_body(const FilterDev& fd, const EpochParams* __restrict__ ep,
                                             int vb, int vg, const StepCoef* s_sc, double* s_red,
                                             int* s_flag) {
  const Ctrl* ctrl = fd.ctrl;
  const int S = ep->S;
  const int cur = ctrl->cur;
  const Ensemble src = committed(fd, cur);
  const Ensemble dst = pending(fd, cur);
  const int64_t N = fd.N;
  const int64_t n = (int64_t)vb * blockDim.x + threadIdx.x;
  double lg = -CUDART_INF;
  if (n < N) {
    double ph[3], th[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) ph[i] = fd.a * src.phi[i * N + n] + (1.0 - fd.a) * ctrl->phibar[i];
    to_theta<3>(fd, ph, th);
    const BrTheta T = br_theta(th);
    // the pending buffer is free until stage 2: it holds the evolving history
    for (int k = 0; k < kBrD; ++k) {
      const int64_t o = (int64_t)k * N + n;
      dst.x[o] = src.x[o];
      dst.h1[o] = src.h1[o];
      dst.h2[o] = src.h2[o];
    }
    double *P0 = dst.x, *P1 = dst.h1, *P2 = dst.h2;
    br_propagate<false>(fd, n, s_sc, S, fd.K, T, P0, P1, P2);
    const double ll = br_loglik(fd, ep, P0, n);
    fd.ll1[n] = ll;
    lg = (src.lw[n] - ctrl->logW) + ll;
    if (!finite_bits(lg)) lg = -CUDART_INF;
    fd.lg[n] = lg;
  }
  stage1_tail(fd, ep->epoch, lg, vb, vg, s_red, s_flag);
}

__device__ __forceinline__ void bstage2_body(const FilterDev& fd, const EpochParams* __restrict__ ep,
                                             int vb, int vg, const StepCoef* s_sc, double* s_red,
                                             int* s_flag) {
  const Ctrl* ctrl = fd.ctrl;
  const int S = ep->S;
  const int cur = ctrl->cur;
  const Ensemble src = committed(fd, cur);
  const Ensemble dst = pending(fd, cur);
  const int64_t N = fd.N;
  const uint32_t epoch = ep->epoch;
  const int64_t n = (int64_t)vb * blockDim.x + threadIdx.x;
  double lwn = -CUDART_INF, bad = 0.0;
  if (n < N) {
    const int64_t l = fd.idx[n];
    // 4a: proliferate phi
    double z[4];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const U4 w = draw_block(fd, kRngTheta, (uint32_t)n, epoch, (uint32_t)b);
      normal_pair(w, z[2 * b], z[2 * b + 1]);
    }
    double ph[3], th[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      double lz = 0.0;
#pragma unroll
      for (int k = 0; k <= i; ++k) lz = fma(ctrl->L[i * kPMax + k], z[k], lz);
      const double shr = fd.a * src.phi[i * N + l] + (1.0 - fd.a) * ctrl->phibar[i];
      ph[i] = fma(fd.s, lz, shr);
      dst.phi[i * N + n] = ph[i];
    }
    to_theta<3>(fd, ph, th);
    const BrTheta T = br_theta(th);
    double* EE = fd.wk + 2 * (int64_t)kBrD * N;
    for (int k = 0; k < kBrD; ++k) {
      const int64_t o = (int64_t)k * N + n, ol = (int64_t)k * N + l;
      dst.x[o] = src.x[ol];
      dst.h1[o] = src.h1[ol];
      dst.h2[o] = src.h2[ol];
      EE[o] = 0.0;
    }
    double *P0 = dst.x, *P1 = dst.h1, *P2 = dst.h2;
    // 4b, 4d: repropagate with the Milne error sums
    br_propagate<true>(fd, n, s_sc, S, fd.K, T, P0, P1, P2);
    // 4c, 4d: innovation, written back in the canonical (x, h1, h2) order
    for (int b = 0; b < kBrD / 2; ++b) {
      const U4 w = draw_block(fd, kRngInnov, (uint32_t)n, epoch, (uint32_t)b);
      double z0, z1;
      normal_pair(w, z0, z1);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t o = (int64_t)(2 * b + h) * N + n;
        const double v = sqrt(fd.kappa * EE[o]) * (h == 0 ? z0 : z1);
        const double a0 = P0[o], a1 = P1[o], a2 = P2[o];
        dst.x[o] = a0 + v;
        dst.h1[o] = a1 + v;
        dst.h2[o] = a2 + v;
      }
    }
    // 5: new log weight
    lwn = br_loglik(fd, ep, dst.x, n) - fd.ll1[l];
    if (!finite_bits(lwn)) {
      lwn = -CUDART_INF;
      bad = 1.0;
    }
    dst.lw[n] = lwn;
  }
  stage2_tail(fd, epoch, lwn, bad, vb, vg, s_red, s_flag);
}

template <int STAGE>
__global__ void __launch_bounds__(kBrThreads) k_bstage(const __grid_constant__ FilterDev fd,
                                                     const EpochParams* __restrict__ ep) {
  extern __shared__ double s_dyn[];
  __shared__ double s_red[32];
  __shared__ int s_flag;
  if (fd.ctrl->status != PF_OK) return;
  StepCoef* s_sc = reinterpret_cast<StepCoef*>(s_dyn);
  load_steps(s_sc, ep, ep->S);
  if (STAGE == 1) bstage1_body(fd, ep, blockIdx.x, gridDim.x, s_sc, s_red, &s_flag);
  else bstage2_body(fd, ep, blockIdx.x, gridDim.x, s_sc, s_red, &s_flag);
}

template <int STAGE>
__global__ void __launch_bounds__(kBrThreads) k_batch_bstage(const FilterDev* __restrict__ fds,
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
  const int vg = (int)((fd.N + kBrThreads - 1) / kBrThreads);
  if (STAGE == 1) bstage1_body(fd, ep, t.vb, vg, s_sc, s_red, &s_flag);
  else bstage2_body(fd, ep, t.vb, vg, s_sc, s_red, &s_flag);
}

int bruss_stage_blocks(int64_t N) { return (int)((N + kBrThreads - 1) / kBrThreads); }

cudaError_t launch_bruss_stage(int stage, const FilterDev& fd, const EpochParams* ep, int S,
                               cudaStream_t st) {
  const size_t smem = (size_t)S * sizeof(StepCoef);
  const unsigned grid = (unsigned)bruss_stage_blocks(fd.N);
  if (stage == 1) k_bstage<1><<<grid, kBrThreads, smem, st>>>(fd, ep);
  else k_bstage<2><<<grid, kBrThreads, smem, st>>>(fd, ep);
  return cudaGetLastError();
}

cudaError_t launch_batch_bruss_stage(int stage, const FilterDev* fds, const EpochParams* const* eps,
                                     const BatchTile* tiles, int ntiles, size_t smem,
                                     cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  if (stage == 1) k_batch_bstage<1><<<ntiles, kBrThreads, smem, st>>>(fds, eps, tiles);
  else k_batch_bstage<2><<<ntiles, kBrThreads, smem, st>>>(fds, eps, tiles);
  return cudaGetLastError();
}

size_t bruss_work_doubles(int64_t N) { return (size_t)kBrWorkRows * (size_t)N; }

cudaError_t preload_bruss_kernels() {
  const void* ks[] = {(const void*)k_bstage<1>, (const void*)k_bstage<2>,
                      (const void*)k_batch_bstage<1>, (const void*)k_batch_bstage<2>};
  for (const void* k : ks) {
    const cudaError_t e = allow_step_table(k);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pfg
