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
// One block per particle.  Shared memory holds the substep table, a cos/sin
// table of nt entries, the physical states, one half-spectrum transform
// buffer (nt odd: modes mx = 0..(nt-1)/2, Hermitian symmetry gives the rest)
// and in stage 2 the error sums.  The transforms are direct sums over the
// table (nt is small and prime or nearly so), split over the block's threads
// by output.  Global memory is touched once per particle per stage.
#include "pf_epoch.cuh"
#include "pf_kernels.h"

namespace pfg {

constexpr int kAdMaxSide = 45;
constexpr int kAdScDoubles = (int)(sizeof(StepCoef) / sizeof(double));
constexpr int kAdMaxModesPerThread = 4;  // modes a thread steps in registers (MPT <= this)

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
  int X[3];  // physical x_n, x_{n-1}, x_{n-2}
  int sp;    // half-spectrum transform buffer [row][mx] (complex)
  int ee;    // stage 2: error sums per grid point
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
  for (int k = 0; k < 3; ++k) {
    L.X[k] = off;
    off += d;
  }
  L.sp = off;
  off += 2 * L.nt * L.H;
  L.ee = off;
  off += err ? d : 0;
  L.total = off;
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

// lambda(mx, my) for mode index t = my * H + mx
__device__ __forceinline__ void ad_lambda(const AdLayout& L, const AdOp& o, const double* tw, int t,
                                          double& lr, double& li) {
  const int nt = L.nt, H = L.H;
  const int my = t / H, mx = t - my * H;
  const double axr = 1.0 - tw[mx], axi = tw[nt + mx];
  const double ayr = 1.0 - tw[my], ayi = tw[nt + my];
  const double ax2 = fma(axr, axr, axi * axi), ay2 = fma(ayr, ayr, ayi * ayi);
  const double cr = fma(axr, ayr, axi * ayi);
  lr = fma(o.c1, axr, o.c2 * ayr) - fma(o.kxx, ax2, fma(2.0 * o.kxy, cr, o.kyy * ay2));
  li = fma(o.c1, axi, o.c2 * ayi);
}

// Forward real 2D DFT of u (physical, shared) into the calling thread's own
// modes: spec[j] = sum_{iy,ix} u[iy][ix] exp(-i phi (mx ix + my iy)) for the
// modes t = tid + j T.  Uses the block's transform buffer; ends with a barrier.
template <int MPT>
__device__ void ad_forward(const AdLayout& L, const double* tw, const double* u, double* buf,
                           double (&re)[MPT], double (&im)[MPT]) {
  const int nt = L.nt, H = L.H, T = blockDim.x, tid = threadIdx.x;
  // rows: buf[iy][mx] = sum_ix u[iy][ix] exp(-i phi mx ix)
  for (int t = tid; t < nt * H; t += T) {
    const int iy = t / H, mx = t - iy * H;
    const double* g = u + iy * nt;
    double sr = 0.0, si = 0.0;
    int k = 0;
    for (int ix = 0; ix < nt; ++ix) {
      sr = fma(g[ix], tw[k], sr);
      si = fma(-g[ix], tw[nt + k], si);
      k += mx;
      if (k >= nt) k -= nt;
    }
    buf[2 * t] = sr;
    buf[2 * t + 1] = si;
  }
  __syncthreads();
  // columns: mode (my, mx) = sum_iy buf[iy][mx] exp(-i phi my iy)
#pragma unroll
  for (int j = 0; j < MPT; ++j) {
    const int t = tid + j * T;
    double sr = 0.0, si = 0.0;
    if (t < nt * H) {
      const int my = t / H, mx = t - my * H;
      int k = 0;
      for (int iy = 0; iy < nt; ++iy) {
        const double ar = buf[2 * (iy * H + mx)], ai = buf[2 * (iy * H + mx) + 1];
        const double cs = tw[k], sn = tw[nt + k];
        sr = fma(ar, cs, fma(ai, sn, sr));
        si = fma(ai, cs, fma(-ar, sn, si));
        k += my;
        if (k >= nt) k -= nt;
      }
    }
    re[j] = sr;
    im[j] = si;
  }
  __syncthreads();
}

// Inverse: the threads' modes (already scaled) are written to the transform
// buffer, then u[iy][ix] = sum over all modes of spec exp(+i phi (mx ix + my
// iy)) (Hermitian in mx), delivered per grid point to `out(i, value)`.
// Ends with a barrier.
template <int MPT, class Out>
__device__ void ad_inverse(const AdLayout& L, const double* tw, double* buf, const double (&re)[MPT],
                           const double (&im)[MPT], Out out) {
  const int nt = L.nt, H = L.H, d = L.d, T = blockDim.x, tid = threadIdx.x;
  double* spec = buf;
#pragma unroll
  for (int j = 0; j < MPT; ++j) {
    const int t = tid + j * T;
    if (t < nt * H) {
      spec[2 * t] = re[j];
      spec[2 * t + 1] = im[j];
    }
  }
  __syncthreads();
  // columns: col[iy][mx] = sum_my spec[my][mx] exp(+i phi my iy), computed
  // into registers and written back in place after a barrier
  double cr[MPT], ci[MPT];
#pragma unroll
  for (int j = 0; j < MPT; ++j) {
    const int t = tid + j * T;
    double sr = 0.0, si = 0.0;
    if (t < nt * H) {
      const int iy = t / H, mx = t - iy * H;
      int k = 0;
      for (int my = 0; my < nt; ++my) {
        const double ar = spec[2 * (my * H + mx)], ai = spec[2 * (my * H + mx) + 1];
        const double cs = tw[k], sn = tw[nt + k];
        sr = fma(ar, cs, fma(-ai, sn, sr));
        si = fma(ai, cs, fma(ar, sn, si));
        k += iy;
        if (k >= nt) k -= nt;
      }
    }
    cr[j] = sr;
    ci[j] = si;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < MPT; ++j) {
    const int t = tid + j * T;
    if (t < nt * H) {
      spec[2 * t] = cr[j];
      spec[2 * t + 1] = ci[j];
    }
  }
  __syncthreads();
  // rows (Hermitian in mx): u = Re z0 + 2 sum_{mx>0} Re(z_mx exp(+i phi mx ix))
  for (int i = tid; i < d; i += T) {
    const int iy = i / nt, ix = i - iy * nt;
    const double* z = spec + 2 * iy * H;
    double acc = 0.0;
    int k = ix;
    for (int mx = 1; mx < H; ++mx) {
      acc = fma(z[2 * mx], tw[k], fma(-z[2 * mx + 1], tw[nt + k], acc));
      k += ix;
      if (k >= nt) k -= nt;
    }
    out(i, fma(2.0, acc, z[0]));
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

template <int STAGE, int MPT>
__global__ void __launch_bounds__(512, 1) k_adstage(const __grid_constant__ FilterDev fd,
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
  const StepCoef* sc = reinterpret_cast<const StepCoef*>(sm + L.sc);
  const int cur = ctrl->cur;
  const Ensemble src = committed(fd, cur);
  const Ensemble dst = pending(fd, cur);
  const int64_t N = fd.N;
  const int64_t n = blockIdx.x;
  const uint32_t epoch = ep->epoch;
  const int d = L.d, T = blockDim.x, tid = threadIdx.x, modes = L.nt * L.H;
  const double inv_d = 1.0 / (double)d;
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
  const double* tw = sm + L.tw;
  double* buf = sm + L.sp;

  // the history in the Fourier basis, each thread holding its own modes
  double x0r[MPT], x0i[MPT];
  double x1r[MPT], x1i[MPT];
  double x2r[MPT], x2i[MPT];
  ad_forward<MPT>(L, tw, sm + L.X[0], buf, x0r, x0i);
  ad_forward<MPT>(L, tw, sm + L.X[1], buf, x1r, x1i);
  ad_forward<MPT>(L, tw, sm + L.X[2], buf, x2r, x2i);
  double lr[MPT], li[MPT];
#pragma unroll
  for (int j = 0; j < MPT; ++j) {
    lr[j] = li[j] = 0.0;
    if (tid + j * T < modes) ad_lambda(L, op, tw, tid + j * T, lr[j], li[j]);
  }

  // Psi over the S substeps (Steps 2 and 4b/4d), mode by mode
  double wr[MPT], wi[MPT];
  double gamma_w = CUDART_NAN;
  for (int s = 0; s < S; ++s) {
    const StepCoef c = sc[s];
    if (!(c.gamma == gamma_w)) {
      // w = 1 / (1 - gamma lambda) per mode
#pragma unroll
      for (int j = 0; j < MPT; ++j) {
        const double p = fma(-c.gamma, lr[j], 1.0), q = -c.gamma * li[j];
        const double inv = 1.0 / fma(p, p, q * q);
        wr[j] = p * inv;
        wi[j] = -q * inv;
      }
      gamma_w = c.gamma;
    }
    double er[MPT], ei[MPT];
#pragma unroll
    for (int j = 0; j < MPT; ++j) {
      double rr, ri, pr = 0.0, pi = 0.0;
      if (c.kind == 2) {
        rr = fma(c.rho2, x1r[j], c.rho1 * x0r[j]);
        ri = fma(c.rho2, x1i[j], c.rho1 * x0i[j]);
        if (STAGE == 2) {
          pr = fma(c.pi2, x2r[j], fma(c.pi1, x1r[j], c.pi0 * x0r[j]));
          pi = fma(c.pi2, x2i[j], fma(c.pi1, x1i[j], c.pi0 * x0i[j]));
        }
      } else {
        // BDF1 (cold start): r = x_n; error predictor x_n + h L x_n
        rr = x0r[j];
        ri = x0i[j];
        if (STAGE == 2) {
          double gr, gi;
          cmul(c.h * lr[j], c.h * li[j], x0r[j], x0i[j], gr, gi);
          pr = x0r[j] + gr;
          pi = x0i[j] + gi;
        }
      }
      double yr, yi;
      cmul(rr, ri, wr[j], wi[j], yr, yi);
      if (STAGE == 2) {
        // Milne's estimate, with the inverse transform's 1/d
        const double f = c.mu * inv_d;
        er[j] = f * (yr - pr);
        ei[j] = f * (yi - pi);
      }
      x2r[j] = x1r[j];
      x2i[j] = x1i[j];
      x1r[j] = x0r[j];
      x1i[j] = x0i[j];
      x0r[j] = yr;
      x0i[j] = yi;
    }
    if (STAGE == 2) {
      double* EE = sm + L.ee;
      ad_inverse<MPT>(L, tw, buf, er, ei, [&](int i, double e) { EE[i] = fma(e, e, EE[i]); });
    }
  }

  // back to physical space (scaled by 1/d)
  auto back = [&](double (&re)[MPT], double (&im)[MPT], double* u) {
#pragma unroll
    for (int j = 0; j < MPT; ++j) {
      re[j] *= inv_d;
      im[j] *= inv_d;
    }
    ad_inverse<MPT>(L, tw, buf, re, im, [&](int i, double v) { u[i] = v; });
  };
  double* X0 = sm + L.X[0];
  back(x0r, x0i, X0);
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
    double* X1 = sm + L.X[1];
    double* X2 = sm + L.X[2];
    back(x1r, x1i, X1);
    back(x2r, x2i, X2);
    // Steps 4c, 4d: innovation v = sqrt(kappa E) z', written in (x, h1, h2) order
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

// Launch shape for a grid side: modes per thread MPT (1, 2 or 4: fewer modes
// per thread keep fewer registers, so more blocks fit an SM) and threads per
// block, a multiple of 32 covering the nt * H modes.
static void ad_shape(int nt, int* threads, int* mpt) {
  const int modes = nt * ((nt + 1) / 2);
  int m = 1;
  while (m < kAdMaxModesPerThread && (modes + m - 1) / m > 512) m *= 2;
  const int need = (modes + m - 1) / m;
  *mpt = m;
  *threads = ((need > 64 ? need : 64) + 31) / 32 * 32;
}

int ad_threads(int nt) {
  int T, m;
  ad_shape(nt, &T, &m);
  return T;
}

size_t ad_stage_smem(int d, int S, int stage) {
  return sizeof(double) * (size_t)ad_layout(d, S, stage == 2).total;
}

cudaError_t launch_ad_stage(int stage, const FilterDev& fd, const EpochParams* ep, int S,
                            cudaStream_t st) {
  const int nt = ad_side(fd.d);
  if (nt == 0) return cudaErrorInvalidValue;
  const size_t smem = ad_stage_smem(fd.d, S, stage);
  int T, mpt;
  ad_shape(nt, &T, &mpt);
  if (T * mpt < nt * ((nt + 1) / 2) || T > 512) return cudaErrorInvalidValue;
  using K = void (*)(const FilterDev, const EpochParams*);
  K k;
  if (mpt == 1) k = stage == 1 ? k_adstage<1, 1> : k_adstage<2, 1>;
  else if (mpt == 2) k = stage == 1 ? k_adstage<1, 2> : k_adstage<2, 2>;
  else k = stage == 1 ? k_adstage<1, 4> : k_adstage<2, 4>;
  cudaError_t e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)fd.N, T, smem, st>>>(fd, ep);
  return cudaGetLastError();
}

cudaError_t preload_ad_kernels() {
  const void* ks[] = {(const void*)k_adstage<1, 1>, (const void*)k_adstage<2, 1>,
                      (const void*)k_adstage<1, 2>, (const void*)k_adstage<2, 2>,
                      (const void*)k_adstage<1, 4>, (const void*)k_adstage<2, 4>};
  for (const void* k : ks) {
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace pfg
