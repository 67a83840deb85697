// lbm_conservation_sums_static: the conservation totals of lbm_moments'
// diagnostics, computed without allocating any memory.
//
// Who needs it: callers that may not call cudaMalloc -- for example a host
// application or plugin whose device memory is owned by another allocator
// (a framework's caching allocator, a fixed arena sized at start-up), or a
// loop that must not allocate while it runs.  The regular path allocates its
// per-block partial sums inside lbm_moments on first use; this variant keeps
// them in a file-scope device array instead.
//
// The scratch array holds kStaticMaxBlocks x kNPartial doubles (192 KiB) on
// every GPU that loads the library, for the life of the process.  Host code
// must not pass the array's name to a kernel (on the host it is only a
// stand-in symbol); the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and passed to the kernels.
// That look-up, and a one-thread kernel that fills the inversion limits, run
// on the first call on each device, so that first call should come before any
// stream capture.  The looked-up addresses are cached per device index for
// the life of the process: after cudaDeviceReset they are stale, so a process
// that resets a device must not call this entry point on it again.
//
// Every call shares the array.  Each call writes every partial it later reads,
// so nothing needs clearing between calls, but calls whose kernels overlap on
// the GPU (different streams, or different host threads) race on the array:
// serialise them.
//
// The cell limit (kStaticMaxCells) is a policy, not a capacity: the kernel is
// a grid-stride loop over at most kStaticMaxBlocks blocks, so the scratch
// array would serve any size; the limit bounds the work of one call.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <mutex>

#include "fd_device.cuh"
#include "lbm.h"

namespace {

using namespace lbm;

constexpr int kNPartial = 6;  // sum n, jx, jy, E, clamped, nonfinite
constexpr int kStaticThreads = 256;
constexpr int kStaticMaxBlocks = 4096;
constexpr int kStaticCellsPerThread = 16;
constexpr int64_t kStaticMaxCells = (int64_t)kStaticMaxBlocks * kStaticThreads * kStaticCellsPerThread;
static_assert(kStaticMaxCells == LBM_STATIC_SUMS_MAX_CELLS, "header limit and kernel limit disagree");

static __device__ __align__(256) double g_static_partials[kStaticMaxBlocks * kNPartial];
static __device__ __align__(256) InvLimits g_static_limits;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
bool g_ready[kMaxDevices] = {};
double* g_partials_ptr[kMaxDevices] = {};
InvLimits* g_limits_ptr[kMaxDevices] = {};

// Per-cell sums of n, j, E, clamped inversions and non-finite states over the
// FP64 population array f[9][cells]; fixed-order block reduction into the
// partials (same order as the regular diagnostics).  Cells marked in solid
// (one byte per cell, same order as f; NULL: none) are obstacles and are left
// out, as lbm_moments leaves them out.  A cell counts as clamped when its
// finite J_2 lies outside the inversion's interval, the rule of lbm_moments
// (no inversion is needed for the count).
template <int STAT>
__global__ void __launch_bounds__(kStaticThreads) static_sums_kernel(const double* __restrict__ f, int64_t cells,
                                                                     const uint8_t* __restrict__ solid,
                                                                     const InvLimits* __restrict__ lim,
                                                                     double* __restrict__ partials) {
  double acc[kNPartial] = {0, 0, 0, 0, 0, 0};
  const InvLimits L = *lim;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += (int64_t)gridDim.x * blockDim.x) {
    if (solid != nullptr && solid[i] != 0) continue;
    double v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = f[a * cells + i];
    const double n = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
    const double jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
    const double jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
    const double E = ((v[1] + v[2]) + (v[3] + v[4])) + 2.0 * ((v[5] + v[6]) + (v[7] + v[8]));
    int cl = 0;
    if (STAT == LBM_STAT_FD) {
      const double ux = jx / n, uy = jy / n;
      const double J2 = 1.5 * (E / n - (ux * ux + uy * uy));
      cl = (isfinite(J2) && (J2 >= L.j2_hi || J2 <= L.j2_lo)) ? 1 : 0;
    }
    bool fin = isfinite(n) && isfinite(jx) && isfinite(jy) && isfinite(E);
#pragma unroll
    for (int a = 0; a < 9; ++a) fin = fin && isfinite(v[a]);
    acc[0] += n;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += E;
    acc[4] += cl;
    acc[5] += fin ? 0.0 : 1.0;
  }
  __shared__ double sh[kStaticThreads / 32][kNPartial];
#pragma unroll
  for (int k = 0; k < kNPartial; ++k) {
    double s = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    acc[k] = s;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNPartial; ++k) sh[wid][k] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x < kNPartial) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kStaticThreads / 32; ++w) s += sh[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * kNPartial + threadIdx.x] = s;
  }
}

// One block sums the partials in a fixed order.
__global__ void __launch_bounds__(256) static_final_kernel(const double* __restrict__ partials, int nblocks,
                                                           double* __restrict__ out) {
  __shared__ double sh[256];
  for (int k = 0; k < kNPartial; ++k) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) s += partials[(int64_t)b * kNPartial + k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
    __syncthreads();
  }
}

__global__ void static_limits_kernel(InvLimits* out) {
  InvLimits L;
  L.x_lo = x_of_t(kTMax);
  L.x_hi = x_of_t(kTMin);
  L.j2_lo = j2_of(fd_eval(L.x_lo));
  L.j2_hi = j2_of(fd_eval(L.x_hi));
  L.j4_lo = j4_of(fd_eval(L.x_lo));
  L.j4_hi = j4_of(fd_eval(L.x_hi));
  *out = L;
}

// Once per device, with that device current: device addresses of the static
// arrays, and the inversion limits.
lbm_status ensure_setup(int dev, cudaStream_t stream, double** partials, InvLimits** limits) {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
    if (e != cudaSuccess) return LBM_ECUDA;
    g_partials_ptr[dev] = (double*)p;
    e = cudaGetSymbolAddress(&p, g_static_limits);
    if (e != cudaSuccess) return LBM_ECUDA;
    g_limits_ptr[dev] = (InvLimits*)p;
    static_limits_kernel<<<1, 1, 0, stream>>>(g_limits_ptr[dev]);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return LBM_ECUDA;
    g_ready[dev] = true;
  }
  *partials = g_partials_ptr[dev];
  *limits = g_limits_ptr[dev];
  return LBM_OK;
}

}  // namespace

namespace lbm {
void set_global_error(const char* m);
}

// Formats the failure into a stack buffer and stores it for
// lbm_last_error(NULL) (no allocation), then returns the status.
static lbm_status static_fail(lbm_status st, const char* what, long long v = -1) {
  char m[256];
  if (v >= 0)
    std::snprintf(m, sizeof(m), "lbm_conservation_sums_static: nx * ny = %lld cells exceeds the limit of %lld "
                  "(LBM_STATIC_SUMS_MAX_CELLS)", v, (long long)kStaticMaxCells);
  else
    std::snprintf(m, sizeof(m), "lbm_conservation_sums_static: %s", what);
  lbm::set_global_error(m);
  return st;
}

extern "C" lbm_status lbm_conservation_sums_static(const double* f, int32_t nx, int32_t ny, const uint8_t* solid,
                                                   int32_t stat, double* out, void* cuda_stream) {
  if (!f || !out) return static_fail(LBM_EINVAL, "NULL populations or output");
  if (nx < 1 || ny < 1) return static_fail(LBM_EINVAL, "nx and ny must be >= 1");
  const int64_t cells = (int64_t)nx * ny;
  if (cells > kStaticMaxCells) return static_fail(LBM_EINVAL, "", (long long)cells);
  if (stat < LBM_STAT_FD || stat > LBM_STAT_FT) return static_fail(LBM_EINVAL, "bad stat");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return static_fail(LBM_ECUDA, "cudaGetDevice failed");
  if (dev < 0 || dev >= kMaxDevices) return static_fail(LBM_EUNSUPPORTED, "device index above 63");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  double* partials = nullptr;
  InvLimits* limits = nullptr;
  const lbm_status st = ensure_setup(dev, s, &partials, &limits);
  if (st != LBM_OK) return static_fail(st, "set-up on this device failed");
  const int64_t want = (cells + kStaticThreads - 1) / kStaticThreads;
  const int blocks = (int)(want < kStaticMaxBlocks ? want : kStaticMaxBlocks);
  switch (stat) {
    case LBM_STAT_FD:
      static_sums_kernel<LBM_STAT_FD><<<blocks, kStaticThreads, 0, s>>>(f, cells, solid, limits, partials);
      break;
    case LBM_STAT_FD_T0:
      static_sums_kernel<LBM_STAT_FD_T0><<<blocks, kStaticThreads, 0, s>>>(f, cells, solid, limits, partials);
      break;
    default:  // MB and FT: no inversion, nothing clamped
      static_sums_kernel<LBM_STAT_MB><<<blocks, kStaticThreads, 0, s>>>(f, cells, solid, limits, partials);
      break;
  }
  static_final_kernel<<<1, 256, 0, s>>>(partials, blocks, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(LBM_ECUDA, cudaGetErrorString(e));
  return LBM_OK;
}
