// opcount.cpp -- exact floating-point operation counts of the oracle's
// propagation Psi (Algorithm 1, Steps 2 and 4: the LMM substeps with their
// full Newton iterations and, for Step 4, the Milne local-error sums).
//
// TEST AND MEASUREMENT INFRASTRUCTURE ONLY, like the rest of oracle/.  The
// oracle's own source (pf_oracle.c) is compiled here a second time as C++
// with `double` replaced by a scalar type that counts every arithmetic
// operation applied to it, so the counts are those of exactly the code the
// oracle runs: dense Jacobian, I - gamma J, LU with partial pivoting, the
// predictor, the history combination and Milne's estimate.  A multiply-add
// counts 2 (the oracle has no fused operations: it is built with
// -ffp-contract=off); divisions, square roots and elementary functions are
// counted separately; comparisons are not flops.  These counts are the
// algorithmic work of one particle-substep that the benchmark's roofline
// divides by time.
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

namespace opc {
struct Counts {
  long long add, mul, div, sqrt_, elem;
};
static Counts g;
}  // namespace opc

struct Flop {
  double v;
  Flop() = default;
  Flop(double x) : v(x) {}                // NOLINT: literals and casts convert
  Flop(int x) : v((double)x) {}           // NOLINT
  Flop(long x) : v((double)x) {}          // NOLINT
  Flop(long long x) : v((double)x) {}     // NOLINT
  Flop(unsigned x) : v((double)x) {}      // NOLINT
  Flop(unsigned long x) : v((double)x) {} // NOLINT
  Flop(unsigned long long x) : v((double)x) {} // NOLINT
  explicit operator double() const { return v; }
  explicit operator int() const { return (int)v; }
  explicit operator long() const { return (long)v; }
  explicit operator long long() const { return (long long)v; }
  Flop& operator+=(Flop o) { ++opc::g.add; v += o.v; return *this; }
  Flop& operator-=(Flop o) { ++opc::g.add; v -= o.v; return *this; }
  Flop& operator*=(Flop o) { ++opc::g.mul; v *= o.v; return *this; }
  Flop& operator/=(Flop o) { ++opc::g.div; v /= o.v; return *this; }
};
static_assert(sizeof(Flop) == sizeof(double), "Flop must lay out like a double");

inline Flop operator+(Flop a, Flop b) { ++opc::g.add; return Flop(a.v + b.v); }
inline Flop operator-(Flop a, Flop b) { ++opc::g.add; return Flop(a.v - b.v); }
inline Flop operator*(Flop a, Flop b) { ++opc::g.mul; return Flop(a.v * b.v); }
inline Flop operator/(Flop a, Flop b) { ++opc::g.div; return Flop(a.v / b.v); }
inline Flop operator-(Flop a) { return Flop(-a.v); }   // a sign flip is not a flop
inline Flop operator+(Flop a) { return a; }
inline bool operator<(Flop a, Flop b) { return a.v < b.v; }
inline bool operator>(Flop a, Flop b) { return a.v > b.v; }
inline bool operator<=(Flop a, Flop b) { return a.v <= b.v; }
inline bool operator>=(Flop a, Flop b) { return a.v >= b.v; }
inline bool operator==(Flop a, Flop b) { return a.v == b.v; }
inline bool operator!=(Flop a, Flop b) { return a.v != b.v; }
inline Flop sqrt(Flop a) { ++opc::g.sqrt_; return Flop(::sqrt(a.v)); }
inline Flop exp(Flop a) { ++opc::g.elem; return Flop(::exp(a.v)); }
inline Flop log(Flop a) { ++opc::g.elem; return Flop(::log(a.v)); }
inline Flop sin(Flop a) { ++opc::g.elem; return Flop(::sin(a.v)); }
inline Flop cos(Flop a) { ++opc::g.elem; return Flop(::cos(a.v)); }
inline Flop pow(Flop a, Flop b) { ++opc::g.elem; return Flop(::pow(a.v, b.v)); }
inline Flop floor(Flop a) { return Flop(::floor(a.v)); }
inline Flop fabs(Flop a) { return Flop(::fabs(a.v)); }
inline Flop fmax(Flop a, Flop b) { return Flop(::fmax(a.v, b.v)); }
inline Flop fmin(Flop a, Flop b) { return Flop(::fmin(a.v, b.v)); }
inline bool isfinite(Flop a) { return ::isfinite(a.v); }

// the oracle's source, with every double a counted scalar
#define double Flop
#include "pf_oracle.c"
#undef double

// or_propagate's counts over the S substeps of tab for one particle (x, h1,
// h2: d values each, theta: p; with_error: Step 4's Milne sums).  out[0..4]:
// additions and subtractions, multiplications, divisions, square roots,
// elementary functions; x_out (if set, d values) the propagated state, which
// is the oracle's own to the bit (the same operations in the same order).
// Returns or_propagate's status.
extern "C" int or_count_propagate(int ode, int d, int K, const double* theta, const or_substep* tab,
                                  int S, const double* x, const double* h1, const double* h2,
                                  int with_error, long long* out, double* x_out) {
  Flop th[OR_PMAX], xx[OR_DMAX], a1[OR_DMAX], a2[OR_DMAX], E[OR_DMAX];
  int dd = 0, p = 0;
  if (or_ode_dims(ode, &dd, &p) != 0 || d < 1 || d > OR_DMAX) return -2;
  for (int i = 0; i < OR_PMAX; ++i) th[i] = Flop(i < p ? theta[i] : 0.0);
  for (int i = 0; i < d; ++i) {
    xx[i] = Flop(x[i]);
    a1[i] = Flop(h1[i]);
    a2[i] = Flop(h2[i]);
    E[i] = Flop(0.0);
  }
  opc::g = opc::Counts{0, 0, 0, 0, 0};
  const int rc = or_propagate(ode, d, K, th, tab, S, xx, a1, a2, with_error ? E : nullptr);
  out[0] = opc::g.add;
  out[1] = opc::g.mul;
  out[2] = opc::g.div;
  out[3] = opc::g.sqrt_;
  out[4] = opc::g.elem;
  if (x_out)
    for (int i = 0; i < d; ++i) x_out[i] = xx[i].v;
  return rc;
}
