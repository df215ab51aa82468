// pf_scan.cuh -- block scans and the systematic-resampling searches shared by
// the epoch kernels (pf_kernels.cu) and the stand-alone resampling calls
// (pf_noalloc.cu).
#pragma once
#include "pf_common.cuh"

namespace pfg {

struct SumOp {
  __device__ static double apply(double a, double b) { return a + b; }
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

// Binary searches and the per-output systematic index over a view c(k) of
// the cumulative weights (CumFinal, CumTiles below), on bit patterns.
template <class V>
__device__ __forceinline__ int64_t upper_bound_bits(const V& c, int64_t N, long long key) {
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__double_as_longlong(c(mid)) > key) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <class V>
__device__ __forceinline__ int64_t lower_bound_bits(const V& c, int64_t N, long long key) {
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (__double_as_longlong(c(mid)) >= key) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <class V>
__device__ __forceinline__ int32_t systematic_index(const V& c, int64_t N, int64_t i, double u,
                                                    double total) {
  const double tau = ((double)i + u) / (double)N * total;
  int64_t k = upper_bound_bits(c, N, __double_as_longlong(tau));
  if (k == N) k = lower_bound_bits(c, N, __double_as_longlong(total));
  return (int32_t)k;
}

// --------------------------------------------------- cumulative weights
// g_k = exp(lg_k - M) and their cumulative sums c_k (Algorithm 1, Step 3a).
// The N values are cut into tiles of kScanThreads * items consecutive values;
// each thread sums `items` of them sequentially, threads are combined by a
// block scan and tiles by the tile offsets of the last block.  A parallel FP64
// scan may dip by an ulp where partial sums meet, so two exact prefix-maximum
// passes (thread level and tile level) make c non-decreasing; the maximum is
// exact and associative, so c is a deterministic function of the log weights
// for a given N.
//
// The exponentials are the scan's cost and FP64 issue is scarce, so the tile
// length follows N and the device's SM count: of 1 to kScanItemsMax values a
// thread, the one whose busiest SM has the least to do -- ceil(tiles / sms)
// tiles of (items + 0.3) units, the 0.3 standing for a thread's share of the
// block scan -- among those that keep the tile count at most
// max(kScanTilesPerSm * sms, ceil(N / (kScanThreads * kScanItemsMax))); ties
// go to more values a thread.
__host__ __device__ constexpr int scan_items(int64_t N, int sms) {
  const int64_t cap_long = (N + kScanThreads * kScanItemsMax - 1) / (kScanThreads * kScanItemsMax);
  const int64_t target = (int64_t)kScanTilesPerSm * sms;
  const int64_t cap = cap_long > target ? cap_long : target;
  int best = kScanItemsMax;
  int64_t best_cost = -1;
  for (int it = kScanItemsMax; it >= 1; --it) {
    const int64_t tiles = (N + (int64_t)kScanThreads * it - 1) / ((int64_t)kScanThreads * it);
    if (tiles > cap) break;
    const int64_t cost = (tiles + sms - 1) / sms * (10 * it + 3);
    if (best_cost < 0 || cost < best_cost) {
      best = it;
      best_cost = cost;
    }
  }
  return best;
}
__host__ __device__ constexpr int64_t scan_tile_len(int64_t N, int sms) {
  return (int64_t)kScanThreads * scan_items(N, sms);
}
__host__ __device__ constexpr int scan_tile_count(int64_t N, int sms) {
  const int64_t L = scan_tile_len(N, sms);
  return (int)((N + L - 1) / L);
}

// g = exp(lg - M) for a finite log weight, 0 for anything else (-inf, and any
// other non-finite value, is a zero weight; the filter's own log weights are
// finite or -inf).  A zero weight stays 0 whatever M is, so all-zero weights
// give c = 0.
__device__ __forceinline__ double scan_weight(double lg, double M) {
  return finite_bits(lg) ? exp(lg - M) : 0.0;
}

// The maximum of two doubles >= +0 (every partial sum here is): their order is
// that of their bit patterns as integers, so this runs on the integer units.
__device__ __forceinline__ double max_nonneg(double a, double b) {
  const long long x = __double_as_longlong(a), y = __double_as_longlong(b);
  return __longlong_as_double(x > y ? x : y);
}
struct MaxNonnegOp {
  __device__ static double apply(double a, double b) { return max_nonneg(a, b); }
};

struct ScanArgs {
  const double* lg;  // N log weights
  int64_t N;
  int64_t Ntile;     // the ensemble size whose tile length applies (N, or the
                     // whole ensemble's size for a shard of it)
  int sms;           // the device's SM count (the tile length depends on it)
  double M;          // their maximum (the log-sum-exp shift)
  double* c;         // N cumulative weights (tile-local after the tile pass)
  double* tile;      // per-tile totals
  double* boff;      // per-tile offsets (sum of the earlier tiles)
  double* pmax;      // per-tile floor (running maximum of the earlier tiles' last values)
  unsigned* ticket;  // completion counter of the tile pass
  double* c_total;   // optional: c_{N-1}
};

// Tile offsets boff_b = sum of the earlier tile totals, and the running
// maximum pmax_b of the earlier tiles' last values boff_b' + T_b', from the nb
// tile totals, by one block; c_total (if set) gets the largest last value,
// c_{N-1}.  The order of additions depends only on nb and the block size.
__device__ __forceinline__ void scan_offsets_core(const double* tile, int nb, double* boff,
                                                  double* pmax, double* s_warp, double* c_total) {
  const int chunk = (nb + blockDim.x - 1) / blockDim.x;
  const int b0 = threadIdx.x * chunk;
  double acc = 0.0;
  for (int b = b0; b < b0 + chunk && b < nb; ++b) acc += __ldcg(tile + b);
  double grand;
  double off = block_exclusive_scan<SumOp>(acc, s_warp, grand);
  double lmax = 0.0;
  for (int b = b0; b < b0 + chunk && b < nb; ++b) {
    boff[b] = off;
    const double T = __ldcg(tile + b);
    lmax = max_nonneg(lmax, off + T);
    off += T;
  }
  double gmax;
  double pm = block_exclusive_scan<MaxNonnegOp>(lmax, s_warp, gmax);
  for (int b = b0; b < b0 + chunk && b < nb; ++b) {
    pmax[b] = pm;
    pm = max_nonneg(pm, boff[b] + __ldcg(tile + b));
  }
  if (threadIdx.x == 0 && c_total) *c_total = gmax;
}

// Tile vb of vg: tile-local cumulative sums; the last tile to finish turns the
// tile totals into offsets and floors.
__device__ __forceinline__ void scan_tile_core(const ScanArgs& a, int vb, int vg, double* s_warp,
                                               int* s_flag) {
  const int items = scan_items(a.Ntile, a.sms);
  const int64_t base = (int64_t)vb * kScanThreads * items + (int64_t)threadIdx.x * items;
  double v[kScanItemsMax];
  double run = 0.0;
#pragma unroll
  for (int j = 0; j < kScanItemsMax; ++j) {
    if (j < items) {
      const int64_t k = base + j;
      run += (k < a.N) ? scan_weight(a.lg[k], a.M) : 0.0;
    }
    v[j] = run;
  }
  double total;
  const double excl = block_exclusive_scan<SumOp>(run, s_warp, total);
#pragma unroll
  for (int j = 0; j < kScanItemsMax; ++j) v[j] = excl + v[j];
  double tile_last;
  const double floor_prev = block_exclusive_scan<MaxNonnegOp>(v[kScanItemsMax - 1], s_warp, tile_last);
#pragma unroll
  for (int j = 0; j < kScanItemsMax; ++j) {
    const int64_t k = base + j;
    if (j < items && k < a.N) a.c[k] = max_nonneg(v[j], floor_prev);
  }
  if (threadIdx.x == 0) a.tile[vb] = tile_last;
  pdl_trigger();
  if (elect_last_block(a.ticket, s_flag, (unsigned)vg))
    scan_offsets_core(a.tile, vg, a.boff, a.pmax, s_warp, a.c_total);
}

// c_k = max(tile offset + tile-local sum, tile floor)
__device__ __forceinline__ void scan_add_core(const ScanArgs& a, int64_t k) {
  if (k < a.N) {
    const int64_t b = k / scan_tile_len(a.Ntile, a.sms);
    a.c[k] = max_nonneg(__ldcg(a.boff + b) + a.c[k], __ldcg(a.pmax + b));
  }
}

// ------------------------------------------------- views of the weights
// CumFinal: c as stored.  CumTiles: c as the tile pass leaves it (tile-local
// sums) read through the per-tile offsets and floors, c_k = max(boff_t + cl_k,
// pmax_t) for the tile t holding k: the offset pass (scan_add_core) folded
// into the reads, bit for bit the values it would store.
struct CumFinal {
  const double* c;
  __device__ __forceinline__ double operator()(int64_t k) const { return __ldg(c + k); }
};

struct CumTiles {
  const double* cl;
  const double* boff;
  const double* pmax;
  uint32_t len;  // tile length, scan_tile_len(N, sms)
  __device__ __forceinline__ double operator()(int64_t k) const {
    const uint32_t t = (uint32_t)k / len;
    return max_nonneg(__ldg(boff + t) + __ldg(cl + k), __ldg(pmax + t));
  }
};

// ------------------------------------------------------ merge-path search
// Systematic resampling (Step 3b): tau_i = ((i + u)/N) c_{N-1} with one
// u per epoch; l_i = min{k : c_k > tau_i},
// else the first k with c_k = c_{N-1}.
//
// Both tau and c are sorted, so l is read off their merge: merging with c_k
// first on ties (c_k <= tau_i), tau_i is taken at the position where exactly
// the c_k <= tau_i have gone before it, i.e. at k = l_i.  The merged sequence
// (2N items) is cut into equal diagonal tiles (merge path): one warp per
// diagonal finds the block's two corners, the block stages its c segment and
// its tau estimates in shared memory with coalesced accesses, and each thread
// walks kRsItems items from its own corner, found by a search in shared
// memory.  Every block does the same work whatever the weights.
//
// FP64 instructions are scarce on this chip (two lanes a clock per SM), so
// the search compares bit patterns: for non-negative doubles their order as
// integers is their numeric order.  Each test tau_i < c_k is first decided
// from the estimate fma(i, s, u s) with s = c_{N-1} / N and u s both rounded:
// it lies within three roundings of the real (i + u) c_{N-1} / N (the rounding
// of u s is at most u / (i + u) <= 1 of a rounding of the whole), tau_i within
// two, so for a normal estimate they are under 3 ulps apart and their bit
// patterns at most 6; a c_k more than kRsUlps patterns away lies on the same
// side of both, and only closer calls (or tiny estimates) compute tau_i
// itself.  The one FP64 operation per output is the estimate's FMA.
constexpr int kResampleThreads = 256;
constexpr int kRsItems = 4;
constexpr int kRsTile = kResampleThreads * kRsItems;
constexpr long long kRsUlps = 64;
constexpr long long kRsTiny = 0x0170000000000000LL;  // bit pattern of 2^-1000

struct RsTau {
  double u, total, step;  // step = total / N, rounded
  double ustep;           // u * step, rounded
  int64_t N;
};

struct RsShared {
  long long c[kRsTile];  // the tile's c segment, as bit patterns
  long long t[kRsTile];  // the tile's tau estimates, as bit patterns
  RsTau tau;
  int64_t corner[2];
  unsigned fresh;
};

__device__ __forceinline__ double rs_tau(int64_t i, const RsTau& t) {
  return ((double)i + t.u) / (double)t.N * t.total;
}

__device__ __forceinline__ long long rs_estimate(int64_t i, const RsTau& t) {
  return __double_as_longlong(__fma_rn((double)i, t.step, t.ustep));
}

// tau_i < c, exactly, given e = rs_estimate(i); e and c are bit patterns
__device__ __forceinline__ bool rs_before(int64_t i, long long e, long long c, const RsTau& t) {
  if (e >= kRsTiny) {
    if (c - e > kRsUlps) return true;
    if (e - c > kRsUlps) return false;
  }
  return __double_as_longlong(rs_tau(i, t)) < c;
}

// Taus among the first dg items of the merge: the largest a with
// tau_{a-1} < c_{dg-a} (or dg - a = N).  One full warp; each round spreads 32
// probes over (lo, hi], and the first failing probe bounds the next range.
template <class V>
__device__ __forceinline__ int64_t rs_corner(const V& c, int64_t dg, const RsTau& t) {
  const int lane = threadIdx.x & 31;
  const int64_t N = t.N;
  int64_t lo = dg > N ? dg - N : 0, hi = dg < N ? dg : N;
  while (lo < hi) {
    const int64_t span = hi - lo;
    const int64_t a = lo + (span * (lane + 1) + 31) / 32;  // in (lo, hi]
    const int64_t b = dg - a;
    const bool ok = b >= N || rs_before(a - 1, rs_estimate(a - 1, t), __double_as_longlong(c(b)), t);
    const unsigned fail = __ballot_sync(0xffffffffu, !ok);
    const int k = fail ? __ffs(fail) - 1 : 32;  // probes 0 .. k-1 hold
    const int64_t nlo = lo + (span * k + 31) / 32;
    if (k < 32) hi = lo + (span * (k + 1) + 31) / 32 - 1;
    lo = nlo;
  }
  return lo;
}

// Tiles of the merge of N taus with N cumulative weights.  Above one wave of
// tiles (kRsTwoPhaseTilesPerSm on each SM) the corners are found first, by a
// launch of one thread per tile boundary (rs_corners_core), so that the
// dependent loads of all the corner searches overlap instead of heading every
// tile; below it each block finds its own two (rs_corner), which saves the
// launch.
constexpr int kRsTwoPhaseTilesPerSm = 4;
__host__ __device__ constexpr int64_t rs_tiles(int64_t N) { return (2 * N + kRsTile - 1) / kRsTile; }
__host__ __device__ inline bool rs_two_phase(int64_t N, int sms) {
  return rs_tiles(N) > (int64_t)kRsTwoPhaseTilesPerSm * sms;
}
// blocks of 256 threads (8 warps) for the corner pass: one warp per corner
__host__ __device__ inline unsigned rs_corner_blocks(int64_t N) {
  return (unsigned)((rs_tiles(N) + 1 + 7) / 8);
}

// Corner v (0 <= v <= rs_tiles(N)) of the merge, taus among its first
// min(v * kRsTile, 2N) items, by one full warp (rs_corner's 32-probe rounds:
// a handful of dependent loads instead of a binary search's twenty-odd).
// Every lane of the warp calls it with the same v.
template <class V>
__device__ __forceinline__ void rs_corners_core(const V& c, int64_t N, double u, int64_t v,
                                                int32_t* __restrict__ corners) {
  if (v > rs_tiles(N)) return;
  RsTau t;
  t.u = u;
  t.total = c(N - 1);
  t.N = N;
  t.step = t.total / (double)N;
  t.ustep = u * t.step;
  const int64_t dg = v * kRsTile < 2 * N ? v * kRsTile : 2 * N;
  const int64_t a = rs_corner(c, dg, t);
  if ((threadIdx.x & 31) == 0) corners[v] = (int32_t)a;
}

// One block's tile of the merge (blockDim.x == kResampleThreads): writes
// idx over the tile's taus and, if n_unique is not null, adds the number of
// outputs whose index differs from the previous output's (the distinct
// parents) to it.
template <class V>
__device__ __forceinline__ void resample_tile(const V& c, int64_t N, double u,
                                              int32_t* __restrict__ idx,
                                              unsigned long long* n_unique, int vb, RsShared& sh,
                                              const int32_t* __restrict__ corners = nullptr) {
  // the block's tile of the merge: items [d0, d1), taus [a0, a1), c [b0, b1)
  const int64_t d0 = (int64_t)vb * kRsTile;
  const int64_t d1 = d0 + kRsTile < 2 * N ? d0 + kRsTile : 2 * N;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (wid < 2) {
    RsTau t;
    t.u = u;
    t.total = c(N - 1);
    t.N = N;
    t.step = t.total / (double)N;
    t.ustep = u * t.step;
    // the corners: given (two-phase), else a warp-wide search each
    const int64_t a = corners ? (int64_t)__ldg(corners + vb + wid) : rs_corner(c, wid == 0 ? d0 : d1, t);
    if (lane == 0) {
      sh.corner[wid] = a;
      if (wid == 0) {
        sh.tau = t;
        sh.fresh = 0u;
      }
    }
  }
  __syncthreads();
  const RsTau t = sh.tau;
  const int64_t a0 = sh.corner[0], a1 = sh.corner[1];
  const int64_t b0 = d0 - a0, b1 = d1 - a1;
  for (int64_t k = b0 + threadIdx.x; k < b1; k += blockDim.x)
    sh.c[k - b0] = __double_as_longlong(c(k));
  for (int64_t k = a0 + threadIdx.x; k < a1; k += blockDim.x) sh.t[k - a0] = rs_estimate(k, t);
  __syncthreads();
  // this thread's corner: a merge-path search in shared memory
  const int64_t ds = d0 + (int64_t)threadIdx.x * kRsItems;
  const int64_t de = ds + kRsItems < d1 ? ds + kRsItems : d1;
  unsigned fresh = 0u;
  if (ds < d1) {
    const int64_t dl = ds - d0, na = a1 - a0, nb = b1 - b0;
    int64_t lo = dl > nb ? dl - nb : 0, hi = dl < na ? dl : na;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      const int64_t bl = dl - mid;
      if (bl >= nb || rs_before(a0 + mid - 1, sh.t[mid - 1], sh.c[bl], t)) lo = mid;
      else hi = mid - 1;
    }
    int64_t a = a0 + lo, b = b0 + (dl - lo);
    // the previous output's index, for the count of distinct parents: if
    // the item just before this corner is tau_{a-1}, it was taken at b
    // (l = b), if it is c_{b-1}, l_{a-1} < b
    bool prev_tau_at_b = false;
    if (a > 0) {
      if (b == 0) {
        prev_tau_at_b = true;
      } else {
        const long long cp = b - 1 >= b0 ? sh.c[b - 1 - b0] : __double_as_longlong(c(b - 1));
        const long long tp = a - 1 >= a0 ? sh.t[a - 1 - a0] : rs_estimate(a - 1, t);
        prev_tau_at_b = !rs_before(a - 1, tp, cp, t);
      }
    }
    int64_t prev_l = -2;  // unknown until this thread's first output
    int64_t fallback = -1;
    for (int64_t dd = ds; dd < de; ++dd) {
      if (a < a1 && (b >= b1 || rs_before(a, sh.t[a - a0], sh.c[b - b0], t))) {
        // tau_a goes before c_b: l_a = b
        int64_t l = b;
        if (b >= N) {
          if (fallback < 0) fallback = lower_bound_bits(c, N, __double_as_longlong(t.total));
          l = fallback;
        }
        idx[a] = (int32_t)l;
        bool is_new;
        if (prev_l != -2) {
          is_new = l != prev_l;
        } else if (a == 0) {
          is_new = true;
        } else if (b < N) {
          is_new = !prev_tau_at_b;
        } else {
          // past the last c (tau rounded up to the total): compare directly
          is_new = l != systematic_index(c, N, a - 1, t.u, t.total);
        }
        fresh += is_new ? 1u : 0u;
        prev_l = l;
        ++a;
      } else {
        ++b;
        prev_tau_at_b = false;  // a c_k goes between the previous output and the next
      }
    }
  }
  fresh = __reduce_add_sync(0xffffffffu, fresh);
  if (lane == 0 && fresh) atomicAdd(&sh.fresh, fresh);
  __syncthreads();
  if (threadIdx.x == 0 && sh.fresh && n_unique) atomicAdd(n_unique, (unsigned long long)sh.fresh);
}

}  // namespace pfg
