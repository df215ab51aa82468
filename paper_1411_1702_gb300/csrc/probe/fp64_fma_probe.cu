// fp64_fma_probe.cu -- a measurement probe for the benchmark, built as its own
// library (libpf_fp64_probe.so), not part of the sampler's C ABI: the FP64 FMA
// throughput this GPU sustains, beside the nominal FP64 rate that the roofline
// of the propagation kernels (one particle per thread, bound by FP64 issue)
// divides by.
//
// Every thread runs kChains independent FMA recurrences acc <- acc * a + b
// (a < 1, so each converges to b / (1 - a) and never over- or underflows),
// enough warps per SM sub-partition to keep the FP64 pipe issuing every
// cycle it can.  The result is stored only under a condition that never
// holds, so the work is not removed.
#include <cuda_runtime.h>

#include <cmath>

namespace {

constexpr int kChains = 8;
constexpr int kDiagThreads = 256;
constexpr int kDiagBlocksPerSm = 4;

__global__ void __launch_bounds__(kDiagThreads) k_fp64_fma(int iters, double a, double b, double* sink) {
  double acc[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc[k] = (double)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = fma(acc[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += acc[k];
  if (s == -1.0) sink[blockIdx.x] = s;  // never true: keeps the chains alive
}

}  // namespace

// TFLOP/s (an FMA counts 2) of independent FMA chains over every SM for about
// ms milliseconds (best of three launches after a calibration) on `stream`
// (a cudaStream_t, NULL = the legacy default stream).  Synchronous.  Returns 0,
// -1 for bad arguments (tflops NULL, ms <= 0), or the CUDA error code.
extern "C" int fp64_fma_rate(void* stream, double ms, double* tflops) {
  if (!tflops || !(ms > 0.0) || !std::isfinite(ms)) return -1;
  *tflops = 0.0;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ev1);
  const int blocks = sms * kDiagBlocksPerSm;
  double* sink = nullptr;  // written only under a condition that never holds
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double) * (size_t)(blocks > 0 ? blocks : 1));
  auto timed = [&](int iters, float* out_ms) -> cudaError_t {
    cudaError_t r = cudaEventRecord(ev0, st);
    if (r == cudaSuccess) {
      k_fp64_fma<<<blocks, kDiagThreads, 0, st>>>(iters, 0.999999, 1e-7, sink);
      r = cudaGetLastError();
    }
    if (r == cudaSuccess) r = cudaEventRecord(ev1, st);
    if (r == cudaSuccess) r = cudaEventSynchronize(ev1);
    if (r == cudaSuccess) r = cudaEventElapsedTime(out_ms, ev0, ev1);
    return r;
  };
  // calibrate: after a warm-up, grow the iteration count until a launch takes
  // at least 2 ms, then scale it to about ms milliseconds; take the best of
  // three such launches
  int iters = 1 << 8;
  float t = 0.0f;
  if (e == cudaSuccess) e = timed(iters, &t);
  if (e == cudaSuccess) e = timed(iters, &t);
  while (e == cudaSuccess && t < 2.0f && iters < (1 << 24)) {
    iters *= 4;
    e = timed(iters, &t);
  }
  if (e == cudaSuccess && t > 0.0f) {
    const double scale = ms / (double)t;
    const double want = (double)iters * (scale > 1.0 ? scale : 1.0);
    iters = (int)(want < (double)(1 << 28) ? want : (double)(1 << 28));
  }
  double best = 0.0;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = timed(iters, &t);
    if (e == cudaSuccess && t > 0.0f) {
      const double flops = 2.0 * kChains * (double)iters * (double)kDiagThreads * (double)blocks;
      const double r = flops / ((double)t * 1e-3) / 1e12;
      best = r > best ? r : best;
    }
  }
  if (sink) cudaFree(sink);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  if (e != cudaSuccess) return (int)e;
  *tflops = best;
  return 0;
}
