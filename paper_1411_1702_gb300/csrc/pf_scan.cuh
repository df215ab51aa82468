// pf_scan.cuh -- block scans and the systematic-resampling search shared by
// the epoch kernels (pf_kernels.cu) and the stand-alone resampling call.
#pragma once
#include "pf_common.cuh"

namespace pfg {

struct SumOp {
  __device__ static double apply(double a, double b) { return a + b; }
};
struct MaxOp {
  __device__ static double apply(double a, double b) { return fmax(a, b); }
};

// Exclusive block scan with identity 0 (all inputs are >= 0); total gets the
// inclusive result of the last thread.  s_warp needs 33 doubles.
template <class Op>
__device__ __forceinline__ double block_exclusive_scan(double v, double* s_warp, double& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  double incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl = Op::apply(t, incl);
  }
  double excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if (lane == 0) excl = 0.0;
  __syncthreads();
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const double w = (lane < nw) ? s_warp[lane] : 0.0;
    double wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi = Op::apply(t, wi);
    }
    double we = __shfl_up_sync(0xffffffffu, wi, 1);
    if (lane == 0) we = 0.0;
    if (lane < nw) s_warp[lane] = we;
    if (lane == nw - 1) s_warp[32] = wi;
  }
  __syncthreads();
  total = s_warp[32];
  return Op::apply(s_warp[wid], excl);
}

__device__ __forceinline__ int64_t upper_bound_bits(const double* c, int64_t N, long long key) {
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__double_as_longlong(__ldg(c + mid)) > key) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ int64_t lower_bound_bits(const double* c, int64_t N, long long key) {
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__double_as_longlong(__ldg(c + mid)) >= key) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ int32_t systematic_index(const double* c, int64_t N, int64_t i, double u,
                                                    double total) {
  const double tau = ((double)i + u) / (double)N * total;
  int64_t k = upper_bound_bits(c, N, __double_as_longlong(tau));
  if (k == N) k = lower_bound_bits(c, N, __double_as_longlong(total));
  return (int32_t)k;
}

}  // namespace pfg
