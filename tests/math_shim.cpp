// A host build of the CUDA path's table-driven math routines (pf_math.cuh),
// for the tests: the routines use only additions, multiplications and fused
// multiply-adds, so this build gives the device's bits.
#include <stdint.h>

#include "pf_math.cuh"

extern "C" void shim_log(const double* x, double* y, long n) {
  for (long i = 0; i < n; ++i) y[i] = pfm::log_pos(x[i]);
}

extern "C" void shim_sincospi(const uint64_t* k, double* s, double* c, long n) {
  for (long i = 0; i < n; ++i) pfm::sincospi_k52(k[i], s[i], c[i]);
}
