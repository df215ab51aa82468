// pf_math.cuh -- the logarithm and the sine/cosine pair of the Box-Muller
// transform in fewer FP64 instructions than the general-purpose library
// routines (on this chip every FP64 instruction counts): each is one table
// value and a short Taylor polynomial.
//
//  log x, after Tang (Table-driven implementation of the logarithm function
//  in IEEE floating-point arithmetic, ACM TOMS 16(4), 1990): x = 2^e y with
//  y in [1, 2), F = 1 + j/128 the breakpoint nearest y, f = y - F (exact),
//  r = f / F (as f times the tabulated 1/F), |r| <= 2^-8, and
//      log x = e log 2 + log F + log1p(r),
//  log1p(r) = r - r^2/2 + ... + r^7/7 (the next term is below 2^-67).  For x
//  in [1/2, 1) the first two terms are one tabulated value, log(F/2): as a sum
//  of two rounded constants it would cancel as F nears 2 (x just below 1).
//
//  sin(pi x), cos(pi x) for x = k 2^-52, 0 <= k < 2^53: the Box-Muller angle
//  2 pi u of a 53-bit uniform u = k 2^-53.  The nearest multiple j/64 of x is
//  split off exactly in integer arithmetic, x = j/64 + t with |t| <= 2^-7,
//  r = pi t, and the angle-addition formulas combine the tabulated sin, cos
//  of pi j/64 with sin r = r - r^3/3! + r^5/5! - r^7/7! and
//  cos r = 1 - r^2/2! + r^4/4! - r^6/6! (|r| <= pi/128; the next terms are
//  below 2^-66 and 2^-58).
//
// Both use only additions, multiplications and fused multiply-adds, so a host
// build of this header (plain C++) gives the same bits as the device one.
#pragma once
#include <stdint.h>

#include <math.h>
#include <string.h>

#include "pf_mathtab.h"

#ifdef __CUDACC__
#define PF_MATH_FN __device__ __forceinline__
#else
#define PF_MATH_FN inline
#endif

namespace pfm {

PF_MATH_FN int64_t bits_of(double x) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(x);
#else
  int64_t b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}

PF_MATH_FN double from_bits(int64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(b);
#else
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}

// log x for a positive normal double x
PF_MATH_FN double log_pos(double x) {
  const int64_t b = bits_of(x);
  const int e = (int)(b >> 52) - 1023;
  const int64_t m = b & 0x000fffffffffffffLL;
  const int j = (int)((m + (1LL << 44)) >> 45);  // y's nearest j/128, 0..128
  const double y = from_bits(m | 0x3ff0000000000000LL);
  const double F = from_bits(0x3ff0000000000000LL + ((int64_t)j << 45));  // 1 + j/128
  const double r = (y - F) * kPfLogInvF[j];
  const double r2 = r * r;
  double p = fma(1.0 / 7.0, r, -1.0 / 6.0);
  p = fma(p, r, 1.0 / 5.0);
  p = fma(p, r, -1.0 / 4.0);
  p = fma(p, r, 1.0 / 3.0);
  p = fma(p, r, -0.5);
  const double l1p = fma(p, r2, r);
  const bool half = e == -1;
  return fma(half ? 0.0 : (double)e, 0x1.62e42fefa39efp-1, kPfLogF[j + (half ? 129 : 0)]) + l1p;
}

// sin(pi x) and cos(pi x), x = k 2^-52, k < 2^53
PF_MATH_FN void sincospi_k52(uint64_t k, double& s, double& c) {
  const int64_t j = (int64_t)((k + (1ULL << 45)) >> 46);  // x's nearest j/64, 0..128
  const int64_t rem = (int64_t)k - (j << 46);               // |rem| <= 2^45: exact as a double
  // r = pi rem 2^-52, with pi 2^-52 the double nearest pi times 2^-52
  const double r = (double)rem * 0x1.921fb54442d18p-51;
  const double r2 = r * r;
  double q = fma(r2, -1.0 / 5040.0, 1.0 / 120.0);
  q = fma(q, r2, -1.0 / 6.0);
  const double sr = fma(q, r2 * r, r);
  double u = fma(r2, -1.0 / 720.0, 1.0 / 24.0);
  u = fma(u, r2, -0.5);
  const double cr = fma(u, r2, 1.0);
  const double sa = kPfSinPi64[j], ca = kPfCosPi64[j];
  s = fma(sa, cr, ca * sr);
  c = fma(ca, cr, -(sa * sr));
}

}  // namespace pfm
