// math_probe.cu -- the device side of the test of pf_math.cuh, in the probe
// library (libpf_fp64_probe.so, outside the sampler's C ABI): evaluates the
// table-driven logarithm and sine/cosine on the GPU for given inputs, so that
// a test can compare them bit for bit with a host build of the same header.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../pf_math.cuh"

namespace {

__global__ void k_math(const double* __restrict__ x, const uint64_t* __restrict__ k, int64_t n,
                       double* __restrict__ lg, double* __restrict__ s, double* __restrict__ c) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  lg[i] = pfm::log_pos(x[i]);
  double a, b;
  pfm::sincospi_k52(k[i], a, b);
  s[i] = a;
  c[i] = b;
}

}  // namespace

// x[n]: positive normal doubles; k[n]: integers below 2^53 (all device
// memory, checked by the caller).  Writes log x, sin(pi k 2^-52) and
// cos(pi k 2^-52) to the device arrays lg, s, c.  Synchronous.  Returns 0, -1
// for bad arguments (a NULL pointer, n < 0 or n >= 2^31), or the CUDA error code.
extern "C" int pf_probe_math(const double* x, const uint64_t* k, int64_t n, double* lg, double* s,
                             double* c) {
  if (!x || !k || !lg || !s || !c || n < 0 || n >= ((int64_t)1 << 31)) return -1;
  if (n == 0) return 0;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  k_math<<<blocks, threads>>>(x, k, n, lg, s, c);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return (int)e;
}
