// pf_noalloc.cu -- systematic resampling of caller-owned device buffers
// without allocating any memory (pf_resample_systematic_noalloc in pf.h).
//
// Some callers cannot allocate device memory at the point where they need to
// resample: applications whose own pool allocator owns all device memory and
// forbids other allocations, latency-critical loops in which cudaMalloc's
// implicit device-wide synchronisation would stall their other streams, and
// callers that must not fail with out-of-memory halfway through a step.  This
// call therefore uses only the caller's input and output buffers plus a
// fixed-size scratch array that is part of the library's device image.
//
// The scratch array lives at file scope below.  Host code may not use its name
// as an address (in host code the name is only a host-side stand-in), so the
// first call on each device looks up its device address with
// cudaGetSymbolAddress while that device is current, and caches it.
//
// The kernels repeat the filter's cumulative-weight scan (same tiles, same
// order of additions, same exact prefix-maximum fix-ups) and run its
// systematic search, so for the same log weights and u the results are
// bit-identical to the cumulative weights and indices of pf_assimilate.
// pf_systematic_indices runs that search alone on given cumulative weights;
// it needs no scratch at all.
#include <mutex>

#include "pf_filter.h"
#include "pf_scan.cuh"

namespace pfg {

constexpr int64_t kNaMaxParticles = PF_NOALLOC_MAX_PARTICLES;
constexpr int kNaMaxTiles = (int)((kNaMaxParticles + kScanTile - 1) / kScanTile);
constexpr int kNaMaxBlocks = 304;  // blocks of the maximum reduction
constexpr int kNaThreads = 256;
// byte layout of the scratch array
constexpr size_t kNaTicketOff = 0;                         // 4 unsigned counters
constexpr size_t kNaHeadOff = 256;                         // max log weight
constexpr size_t kNaBlockMaxOff = 512;                     // kNaMaxBlocks doubles
constexpr size_t kNaTileOff = kNaBlockMaxOff + 8 * 512;    // tile totals
constexpr size_t kNaBoffOff = kNaTileOff + 8 * (size_t)kNaMaxTiles;
constexpr size_t kNaPmaxOff = kNaBoffOff + 8 * (size_t)kNaMaxTiles;
constexpr size_t kNaBytes = kNaPmaxOff + 8 * (size_t)kNaMaxTiles;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

struct NaScratch {
  unsigned* ticket;
  double* head;
  double* blockmax;
  double* tile;
  double* boff;
  double* pmax;
};

static NaScratch carve(unsigned char* base) {
  return NaScratch{reinterpret_cast<unsigned*>(base + kNaTicketOff),
                   reinterpret_cast<double*>(base + kNaHeadOff),
                   reinterpret_cast<double*>(base + kNaBlockMaxOff),
                   reinterpret_cast<double*>(base + kNaTileOff),
                   reinterpret_cast<double*>(base + kNaBoffOff),
                   reinterpret_cast<double*>(base + kNaPmaxOff)};
}

// Only -inf and finite log weights are meaningful; anything else counts as a
// zero weight (for valid inputs this is the identity).
__device__ __forceinline__ double clean_logw(double v) {
  return finite_bits(v) ? v : -CUDART_INF;
}

__global__ void __launch_bounds__(kNaThreads) k_na_max(const double* __restrict__ lg, int64_t N,
                                                     NaScratch sc) {
  __shared__ double s_red[32];
  __shared__ int s_flag;
  double m = -CUDART_INF;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x)
    m = fmax(m, clean_logw(lg[k]));
  m = block_max(m, s_red);
  if (threadIdx.x == 0) sc.blockmax[blockIdx.x] = m;
  if (elect_last_block(sc.ticket + 0, &s_flag, gridDim.x)) {
    double t = -CUDART_INF;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t = fmax(t, __ldcg(sc.blockmax + b));
    t = block_max(t, s_red);
    if (threadIdx.x == 0) sc.head[0] = t;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_na_scan_tile(const double* __restrict__ lg,
                                                             int64_t N, double* c, NaScratch sc) {
  __shared__ double s_warp[33];
  __shared__ int s_flag;
  const double M = __ldcg(sc.head);
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  double v[kScanItems];
  double run = 0.0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t k = base + j;
    const double g = (k < N) ? exp(clean_logw(lg[k]) - M) : 0.0;
    run += g;
    v[j] = run;
  }
  double total;
  const double excl = block_exclusive_scan<SumOp>(run, s_warp, total);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) v[j] = excl + v[j];
  double tile_last;
  const double floor_prev = block_exclusive_scan<MaxOp>(v[kScanItems - 1], s_warp, tile_last);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t k = base + j;
    if (k < N) c[k] = fmax(v[j], floor_prev);
  }
  if (threadIdx.x == 0) sc.tile[blockIdx.x] = tile_last;
  if (elect_last_block(sc.ticket + 1, &s_flag, gridDim.x)) {
    const int nb = gridDim.x;
    const int chunk = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * chunk;
    double acc = 0.0;
    for (int b = b0; b < b0 + chunk && b < nb; ++b) acc += __ldcg(sc.tile + b);
    double grand;
    double off = block_exclusive_scan<SumOp>(acc, s_warp, grand);
    double lmax = 0.0;
    for (int b = b0; b < b0 + chunk && b < nb; ++b) {
      sc.boff[b] = off;
      const double T = __ldcg(sc.tile + b);
      lmax = fmax(lmax, off + T);
      off += T;
    }
    double gmax;
    double pm = block_exclusive_scan<MaxOp>(lmax, s_warp, gmax);
    for (int b = b0; b < b0 + chunk && b < nb; ++b) {
      sc.pmax[b] = pm;
      pm = fmax(pm, sc.boff[b] + __ldcg(sc.tile + b));
    }
  }
}

__global__ void __launch_bounds__(256) k_na_scan_add(int64_t N, double* c, NaScratch sc) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < N) {
    const int64_t b = k / kScanTile;
    c[k] = fmax(__ldcg(sc.boff + b) + c[k], __ldcg(sc.pmax + b));
  }
}

// the filter's merge-path search (resample_tile), one block per diagonal tile
__global__ void __launch_bounds__(kResampleThreads) k_na_resample(const double* __restrict__ c,
                                                                  int64_t N, double u,
                                                                  int32_t* __restrict__ idx) {
  __shared__ RsShared sh;
  resample_tile(c, N, u, idx, nullptr, blockIdx.x, sh);
}

static unsigned resample_blocks(int64_t N) { return (unsigned)((2 * N + kRsTile - 1) / kRsTile); }

// device address of the scratch array, looked up once per device
constexpr int kMaxDevices = 64;
static std::mutex g_na_mutex;
static unsigned char* g_na_ptr[kMaxDevices];

static cudaError_t scratch_address(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

}  // namespace pfg

extern "C" pf_status pf_resample_systematic_noalloc(const double* log_g, int64_t N, double u,
                                                    double* cumulative, int32_t* idx,
                                                    void* stream) {
  using namespace pfg;
  if (!log_g || !cumulative || !idx) {
    set_thread_error("pf_resample_systematic_noalloc: NULL buffer");
    return PF_ERR_INVALID_ARG;
  }
  if (N < 1) {
    set_thread_error("pf_resample_systematic_noalloc: need N >= 1");
    return PF_ERR_INVALID_ARG;
  }
  if (N > kNaMaxParticles) {
    set_thread_error("pf_resample_systematic_noalloc: N exceeds PF_NOALLOC_MAX_PARTICLES (2^24); "
                     "use a filter (pf_create) for larger ensembles");
    return PF_ERR_BUDGET;
  }
  if (!(u >= 0.0 && u < 1.0)) {
    set_thread_error("pf_resample_systematic_noalloc: need 0 <= u < 1");
    return PF_ERR_INVALID_ARG;
  }
  unsigned char* base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    set_thread_error(std::string("pf_resample_systematic_noalloc: scratch address lookup failed: ") +
                     cudaGetErrorString(e));
    return PF_ERR_CUDA;
  }
  const NaScratch sc = carve(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the completion counters must start at zero
  e = cudaMemsetAsync(sc.ticket, 0, 4 * sizeof(unsigned), st);
  if (e == cudaSuccess) {
    const int64_t mb = (N + kNaThreads - 1) / kNaThreads;
    const unsigned g_max = (unsigned)(mb < kNaMaxBlocks ? mb : kNaMaxBlocks);
    k_na_max<<<g_max, kNaThreads, 0, st>>>(log_g, N, sc);
    k_na_scan_tile<<<(unsigned)((N + kScanTile - 1) / kScanTile), kScanThreads, 0, st>>>(
        log_g, N, cumulative, sc);
    k_na_scan_add<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, cumulative, sc);
    k_na_resample<<<resample_blocks(N), kResampleThreads, 0, st>>>(cumulative, N, u, idx);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_thread_error(std::string("pf_resample_systematic_noalloc: launch failed: ") +
                     cudaGetErrorString(e));
    return PF_ERR_CUDA;
  }
  return PF_OK;
}

extern "C" pf_status pf_systematic_indices(const double* cumulative, int64_t N, double u,
                                           int32_t* idx, void* stream) {
  using namespace pfg;
  if (!cumulative || !idx) {
    set_thread_error("pf_systematic_indices: NULL buffer");
    return PF_ERR_INVALID_ARG;
  }
  if (N < 1 || N > (int64_t)INT32_MAX) {
    set_thread_error("pf_systematic_indices: need 1 <= N <= 2^31 - 1");
    return PF_ERR_INVALID_ARG;
  }
  if (!(u >= 0.0 && u < 1.0)) {
    set_thread_error("pf_systematic_indices: need 0 <= u < 1");
    return PF_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_na_resample<<<resample_blocks(N), kResampleThreads, 0, st>>>(cumulative, N, u, idx);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_thread_error(std::string("pf_systematic_indices: launch failed: ") + cudaGetErrorString(e));
    return PF_ERR_CUDA;
  }
  return PF_OK;
}
