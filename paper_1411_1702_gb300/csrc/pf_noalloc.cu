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
// as an address (in host code the name is only a host-side stand-in), so every
// call looks up its device address with cudaGetSymbolAddress on the current
// device.
//
// The kernels repeat the filter's cumulative-weight scan (same tiles, same
// order of additions, same exact prefix-maximum fix-ups) and run its
// systematic search, so for the same log weights and u the results are
// bit-identical to the cumulative weights and indices of pf_assimilate.
// pf_systematic_indices runs that search alone on given cumulative weights;
// it needs no scratch at all.
#include "pf_filter.h"
#include "pf_scan.cuh"

namespace pfg {

constexpr int64_t kNaMaxParticles = PF_NOALLOC_MAX_PARTICLES;
// the most scan tiles of any N up to the maximum on a device of up to kMaxSms
// SMs (scan_tile_count)
constexpr int64_t kNaLongTiles = (kNaMaxParticles + kScanThreads * kScanItemsMax - 1) /
                                 (kScanThreads * kScanItemsMax);
constexpr int kNaMaxTiles = (int)(kNaLongTiles > (int64_t)kScanTilesPerSm * kMaxSms
                                      ? kNaLongTiles
                                      : (int64_t)kScanTilesPerSm * kMaxSms);
constexpr int kNaMaxBlocks = 304;  // blocks of the maximum reduction
constexpr int kNaThreads = 256;
// byte layout of the scratch array
constexpr size_t kNaTicketOff = 0;                         // 4 unsigned counters
constexpr size_t kNaHeadOff = 256;                         // max log weight
constexpr size_t kNaBlockMaxOff = 512;                     // kNaMaxBlocks doubles
constexpr size_t kNaTileOff = kNaBlockMaxOff + 8 * 512;    // tile totals
constexpr size_t kNaBoffOff = kNaTileOff + 8 * (size_t)kNaMaxTiles;
constexpr size_t kNaPmaxOff = kNaBoffOff + 8 * (size_t)kNaMaxTiles;
constexpr size_t kNaCornerOff = kNaPmaxOff + 8 * (size_t)kNaMaxTiles;  // merge-tile corners
constexpr int64_t kNaMaxCorners = (2 * kNaMaxParticles + kRsTile - 1) / kRsTile + 1;
constexpr size_t kNaBytes = kNaCornerOff + 4 * (size_t)kNaMaxCorners;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

struct NaScratch {
  unsigned* ticket;
  double* head;
  double* blockmax;
  double* tile;
  double* boff;
  double* pmax;
  int32_t* corners;
};

static NaScratch carve(unsigned char* base) {
  return NaScratch{reinterpret_cast<unsigned*>(base + kNaTicketOff),
                   reinterpret_cast<double*>(base + kNaHeadOff),
                   reinterpret_cast<double*>(base + kNaBlockMaxOff),
                   reinterpret_cast<double*>(base + kNaTileOff),
                   reinterpret_cast<double*>(base + kNaBoffOff),
                   reinterpret_cast<double*>(base + kNaPmaxOff),
                   reinterpret_cast<int32_t*>(base + kNaCornerOff)};
}

__global__ void __launch_bounds__(kNaThreads) k_na_max(const double* __restrict__ lg, int64_t N,
                                                     NaScratch sc) {
  __shared__ double s_red[32];
  __shared__ int s_flag;
  double m = -CUDART_INF;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
       k += (int64_t)gridDim.x * blockDim.x)
    if (finite_bits(lg[k])) m = fmax(m, lg[k]);
  m = block_max(m, s_red);
  if (threadIdx.x == 0) sc.blockmax[blockIdx.x] = m;
  if (elect_last_block(sc.ticket + 0, &s_flag, gridDim.x)) {
    double t = -CUDART_INF;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t = fmax(t, __ldcg(sc.blockmax + b));
    t = block_max(t, s_red);
    if (threadIdx.x == 0) sc.head[0] = t;
  }
}

// the filter's scan (scan_tile_core, scan_add_core) on the caller's buffers
__device__ __forceinline__ ScanArgs na_scan_args(const double* lg, int64_t N, int sms, double* c,
                                                 const NaScratch& sc) {
  return ScanArgs{lg, N, N, sms, __ldcg(sc.head), c, sc.tile, sc.boff, sc.pmax, sc.ticket + 1, nullptr};
}

__global__ void __launch_bounds__(kScanThreads) k_na_scan_tile(const double* __restrict__ lg,
                                                             int64_t N, int sms, double* c,
                                                             NaScratch sc) {
  __shared__ double s_warp[33];
  __shared__ int s_flag;
  scan_tile_core(na_scan_args(lg, N, sms, c, sc), blockIdx.x, gridDim.x, s_warp, &s_flag);
}

__global__ void __launch_bounds__(256) k_na_scan_add(int64_t N, int sms, double* c, NaScratch sc) {
  scan_add_core(na_scan_args(nullptr, N, sms, c, sc), (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// the filter's merge-path search (resample_tile), one block per diagonal tile;
// corners: found first by k_na_corners (two-phase), or null
__global__ void __launch_bounds__(kResampleThreads, 4) k_na_resample(const double* __restrict__ c,
                                                                  int64_t N, double u,
                                                                  int32_t* __restrict__ idx,
                                                                  const int32_t* __restrict__ corners) {
  __shared__ RsShared sh;
  resample_tile(CumFinal{c}, N, u, idx, nullptr, blockIdx.x, sh, corners);
}

__global__ void __launch_bounds__(256) k_na_corners(const double* __restrict__ c, int64_t N, double u,
                                                   int32_t* __restrict__ corners) {
  rs_corners_core(CumFinal{c}, N, u, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, corners);
}

static unsigned resample_blocks(int64_t N) { return (unsigned)((2 * N + kRsTile - 1) / kRsTile); }

// Device address of the scratch array on the current device.  It is looked up
// on every call (a table lookup once the module is loaded) rather than cached,
// so a device reset or a re-created primary context, after which the module is
// reloaded and the array may move, never leaves a stale address behind.
static cudaError_t scratch_address(unsigned char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<unsigned char*>(p);
  return cudaSuccess;
}

// The scratch layout holds every size up to the maximum: the scan's tile
// count is at most max(kScanTilesPerSm * sms, ceil(N / (kScanThreads *
// kScanItemsMax))) and the merge has rs_tiles(N) + 1 corners, both largest at
// the maximum N and SM count.
static_assert(scan_tile_count(kNaMaxParticles, kMaxSms) <= kNaMaxTiles, "scan tiles exceed the scratch");
static_assert(scan_tile_count(kScanThreads * kScanTilesPerSm * kMaxSms, kMaxSms) <= kNaMaxTiles,
              "scan tiles exceed the scratch");
static_assert(rs_tiles(kNaMaxParticles) + 1 <= kNaMaxCorners, "merge corners exceed the scratch");

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
  // a second line of defence behind the static_asserts: the layout must hold
  // this N's tiles and corners on this device
  const int sms = device_sms();
  if (scan_tile_count(N, sms) > kNaMaxTiles || rs_tiles(N) + 1 > kNaMaxCorners) {
    set_thread_error("pf_resample_systematic_noalloc: scratch layout too small for this N");
    return PF_ERR_BUDGET;
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
    k_na_scan_tile<<<(unsigned)scan_tile_count(N, sms), kScanThreads, 0, st>>>(
        log_g, N, sms, cumulative, sc);
    k_na_scan_add<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, sms, cumulative, sc);
    const bool two = rs_two_phase(N, sms);
    if (two) k_na_corners<<<rs_corner_blocks(N), 256, 0, st>>>(cumulative, N, u, sc.corners);
    k_na_resample<<<resample_blocks(N), kResampleThreads, 0, st>>>(cumulative, N, u, idx,
                                                                   two ? sc.corners : nullptr);
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
  k_na_resample<<<resample_blocks(N), kResampleThreads, 0, st>>>(cumulative, N, u, idx, nullptr);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_thread_error(std::string("pf_systematic_indices: launch failed: ") + cudaGetErrorString(e));
    return PF_ERR_CUDA;
  }
  return PF_OK;
}
