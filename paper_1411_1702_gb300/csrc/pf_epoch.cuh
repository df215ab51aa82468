// pf_epoch.cuh -- device helpers shared by the epoch kernels of every model.
#pragma once
#include "pf_common.cuh"

namespace pfg {

__device__ __forceinline__ Ensemble committed(const FilterDev& fd, int cur) {
  return cur ? fd.ens[1] : fd.ens[0];
}
__device__ __forceinline__ Ensemble pending(const FilterDev& fd, int cur) {
  return cur ? fd.ens[0] : fd.ens[1];
}

template <int P>
__device__ __forceinline__ void to_theta(const FilterDev& fd, const double (&ph)[P], double (&th)[P]) {
#pragma unroll
  for (int i = 0; i < P; ++i) th[i] = (fd.transform == PF_TRANSFORM_LOG) ? exp(ph[i]) : ph[i];
}

__device__ __forceinline__ void load_steps(StepCoef* s_sc, const EpochParams* __restrict__ ep, int S) {
  const double* src = reinterpret_cast<const double*>(ep->sc);
  double* dst = reinterpret_cast<double*>(s_sc);
  const int nd = S * (int)(sizeof(StepCoef) / sizeof(double));
  for (int i = threadIdx.x; i < nd; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Cholesky factor of a PSD matrix; a non-positive pivot gives a zero column.
__device__ inline void cholesky_psd(int p, const double* C, double* L) {
  for (int i = 0; i < kPMax * kPMax; ++i) L[i] = 0.0;
  for (int j = 0; j < p; ++j) {
    double dsum = C[j * kPMax + j];
    for (int k = 0; k < j; ++k) dsum -= L[j * kPMax + k] * L[j * kPMax + k];
    if (!(dsum > 0.0)) continue;
    const double ljj = sqrt(dsum);
    L[j * kPMax + j] = ljj;
    for (int i = j + 1; i < p; ++i) {
      double s = C[i * kPMax + j];
      for (int k = 0; k < j; ++k) s -= L[i * kPMax + k] * L[j * kPMax + k];
      L[i * kPMax + j] = s / ljj;
    }
  }
}

// Step 4a's factor L of the committed covariance C, by one warp (lane = 0..31)
// of the filter's first resampling block: only stage 2 uses L, and that warp
// is idle while two others search the tile corners, so the factorisation is
// off the epoch's serial tails.  Lane i owns row i; the column order and the
// operations are those of cholesky_psd, so L is the same to the bit.  s needs
// kPMax * kPMax doubles of shared memory of the warp's own.
__device__ __forceinline__ void factor_covariance(const FilterDev& fd, int p, double* s, int lane) {
  Ctrl* ctrl = fd.ctrl;
  if (lane < kPMax * kPMax) s[lane] = 0.0;
  __syncwarp();
  for (int j = 0; j < p; ++j) {
    double dsum = ctrl->C[j * kPMax + j];
    for (int k = 0; k < j; ++k) dsum -= s[j * kPMax + k] * s[j * kPMax + k];
    if (dsum > 0.0) {
      const double ljj = sqrt(dsum);
      if (lane == j) s[j * kPMax + j] = ljj;
      if (lane > j && lane < p) {
        double sv = ctrl->C[lane * kPMax + j];
        for (int k = 0; k < j; ++k) sv -= s[lane * kPMax + k] * s[j * kPMax + k];
        s[lane * kPMax + j] = sv / ljj;
      }
    }
    __syncwarp();
  }
  if (lane < kPMax * kPMax) ctrl->L[lane] = s[lane];
}

// End of stage 1 (Step 3a): block maximum of the log fitness weights; the
// last of the filter's vg blocks stores the global maximum (the log-sum-exp
// shift) and flags a degenerate epoch.  Every thread of the block must call it.
__device__ __forceinline__ void stage1_tail(const FilterDev& fd, uint32_t epoch, double lg, int vb,
                                            int vg, double* s_red, int* s_flag) {
  Ctrl* ctrl = fd.ctrl;
  const double bm = block_max(lg, s_red);
  if (threadIdx.x == 0) fd.blk[vb] = bm;
  if (elect_last_block(fd.ticket + 0, s_flag, (unsigned)vg)) {
    double m = -CUDART_INF;
    for (int b = threadIdx.x; b < vg; b += blockDim.x) m = fmax(m, __ldcg(fd.blk + b));
    m = block_max(m, s_red);
    if (threadIdx.x == 0) {
      ctrl->lg_max = m;
      ctrl->n_unique = 0;
      ctrl->n_nonfinite = 0;
      if (!(m > -CUDART_INF)) {
        ctrl->status = PF_ERR_DEGENERATE;
        ctrl->failed_epoch = epoch;
      }
    }
  }
}

// End of stage 2 (Step 5): block maximum of the new log weights and the count
// of zero-weight particles; the last of the filter's vg blocks stores the
// maximum and flags a degenerate epoch.  Every thread of the block must call it.
__device__ __forceinline__ void stage2_tail(const FilterDev& fd, uint32_t epoch, double lwn,
                                            double bad, int vb, int vg, double* s_red, int* s_flag) {
  Ctrl* ctrl = fd.ctrl;
  const double bm = block_max(lwn, s_red);
  const double nb = block_sum(bad, s_red);
  if (threadIdx.x == 0) {
    fd.blk[vb] = bm;
    if (nb > 0.0)
      atomicAdd(reinterpret_cast<unsigned long long*>(&ctrl->n_nonfinite), (unsigned long long)nb);
  }
  if (elect_last_block(fd.ticket + 2, s_flag, (unsigned)vg)) {
    double m = -CUDART_INF;
    for (int b = threadIdx.x; b < vg; b += blockDim.x) m = fmax(m, __ldcg(fd.blk + b));
    m = block_max(m, s_red);
    if (threadIdx.x == 0) {
      ctrl->lw_max = m;
      if (!(m > -CUDART_INF)) {
        ctrl->status = PF_ERR_DEGENERATE;
        ctrl->failed_epoch = epoch;
      }
    }
  }
}

}  // namespace pfg
