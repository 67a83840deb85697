// C ABI of the library (declared in include/lbm.h): contexts, buffers,
// dispatch of the kernels in lbm_kernels.cuh, CUDA-graph replay of steps.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "io_dev.cuh"
#include "launch.h"
#include "lbm.h"
#include "lbm_dev_x64.cuh"
#include "lbm_kernels.cuh"
#include "surrogate.cuh"

using namespace lbm;

namespace {

constexpr int kGraphChunk = 16;  // steps per captured graph (even: buffers return)
// counters of a learned-inversion context: fallbacks, evaluations, tensor-core
// round timeouts, timeouts of the final wait before tensor memory is freed
constexpr int kNSurrCounters = 4;

// ------------------------------------------------------------------ per-context setup

static __global__ void setup_kernel(InvLimits* out) {
  InvLimits L;
  L.x_lo = x_of_t(kTMax);
  L.x_hi = x_of_t(kTMin);
  L.j2_lo = j2_of(fd_eval(L.x_lo));
  L.j2_hi = j2_of(fd_eval(L.x_hi));
  L.j4_lo = j4_of(fd_eval(L.x_lo));
  L.j4_hi = j4_of(fd_eval(L.x_hi));
  *out = L;
}

// Deviation reference of each problem: J_2,ref from t_ref (or the closure's
// constant), W^ref = w_a(J_2,ref) n_ref and n_ref (3/2 - J_2,ref).
static __global__ void ref_kernel(ProbDev* probs, int nprob, int stat, int dim) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nprob) return;
  ProbDev& P = probs[p];
  if (dim == 1) {  // d1v3: W_0 = n (1 - J_2/3), W_+-1 = n J_2/6
    const double J2 = stat == STAT_T0 ? 5.0 / 3.0 : 1.0, n = P.n_ref;
    P.j2_ref = J2;
    P.ndelta_ref = 0.0;
    P.wref[0] = n * (1.0 - J2 / 3.0);
    P.wref[1] = P.wref[2] = n * J2 / 6.0;
    for (int a = 3; a < 9; ++a) P.wref[a] = 0.0;
    P.f.omega = (float)P.omega;
    P.f.n_ref = (float)n;
    P.f.ndelta_ref = 0.0f;
    P.f.wref[0] = (float)P.wref[0];
    P.f.wref[1] = P.f.wref[2] = (float)P.wref[1];
    return;
  }
  double J2, J4;
  if (stat == STAT_FD || stat == STAT_FT) {
    if (P.n_ref > 0.0) closure_from_t<STAT_FD>(P.t_ref, J2, J4); else J2 = 1.5;
  } else if (stat == STAT_T0) {
    J2 = FixedJ<STAT_T0>::j2;
  } else {
    J2 = FixedJ<STAT_MB>::j2;
  }
  const double n = P.n_ref;
  const double w0 = n * (1.0 - 5.0 * J2 / 9.0), ws = n * J2 / 9.0, wl = n * J2 / 36.0;
  P.j2_ref = J2;
  P.ndelta_ref = n * (1.5 - J2);
  P.wref[0] = w0;
  for (int a = 1; a <= 4; ++a) P.wref[a] = ws;
  for (int a = 5; a <= 8; ++a) P.wref[a] = wl;
  P.f.omega = (float)P.omega;
  P.f.n_ref = (float)n;
  P.f.ndelta_ref = (float)P.ndelta_ref;
  P.f.wref[0] = (float)w0;
  P.f.wref[1] = (float)ws;
  P.f.wref[2] = (float)wl;
  P.f.two_pi_theta = (float)(2.0 * kPi * P.theta);
  P.nsum_ref = w0 + 4.0 * ws + 4.0 * wl;
  P.esum_ref = 4.0 * ws + 8.0 * wl;
}


// One block sums the per-block partials in a fixed order.
static __global__ void __launch_bounds__(256) reduce_partials_kernel(const double* __restrict__ partials, int64_t nblocks,
                                                              double* __restrict__ out) {
  __shared__ double sh[256];
  for (int k = 0; k < kNPartial; ++k) {
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nblocks; b += 256) s += partials[b * kNPartial + k];
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



std::mutex g_err_mu;
char g_create_err[512] = "";  // last context-free failure (fixed buffer: no allocation)

size_t elem_size(int prec) { return prec == LBM_F64 ? 8 : prec == LBM_F32_DEV ? 4 : 2; }

}  // namespace

struct lbm_ctx {
  int stat = 0, prec = 0, inv = 0, nprob = 0;
  std::vector<lbm_problem> probs;
  std::vector<ProbDev> ph;  // host copy of the device table
  ProbDev* pd = nullptr;
  int64_t plane = 0, ntiles = 0;
  int dim = 2, q = 9;        // lattice: d2v9 or d1v3
  uint8_t* mask = nullptr;   // device: obstacle mask indexed like the cells (allocated on first use)
  uint16_t* pcode = nullptr; // device: pull codes indexed like the cells (with the mask)
  bool porous = false;       // some problem has obstacles or a body force
  int rows = kTileYDefault;  // rows per tile
  int ctas = 0;              // 0: one CTA per tile; else a persistent grid of this many CTAs
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  InvLimits lim{};
  InvLimitsF limf{};
  InvLimits* lim_d = nullptr;
  double* partials = nullptr;
  int64_t partials_cap = 0;
  double* diag_d = nullptr;
  double* tmp = nullptr;
  int64_t tmp_cap = 0;
  int64_t launches = 0;
  std::string err;
  MlpParams* surr = nullptr;               // host copy of the network (learned inversion)
  unsigned long long* surr_count = nullptr;  // device: fallbacks, evaluations, tensor-core round timeouts,
                                             // timeouts of the final wait before TMEM is freed
  int tc_polls = kTcWaitPolls;               // per-round poll limit of the tensor-core engine
  void* wtc = nullptr;                       // device: the network's FP16 tensor-core operands (kTcBytes)
  void* wmm = nullptr;                       // device: the network's warp-MMA fragments (kMmBytes)
  int surr_engine = LBM_SURROGATE_TENSOR_CORES;
  int64_t tc_grid[9] = {};  // persistent grid of the tensor-core kernel per rows per tile: SMs x resident CTAs
  int64_t mm_grid[9] = {};  // the same for the warp-MMA kernel
};

namespace {

lbm_status fail(lbm_ctx* ctx, lbm_status s, const std::string& m) {
  if (ctx) {
    ctx->err = m;
  } else {
    std::lock_guard<std::mutex> g(g_err_mu);
    std::snprintf(g_create_err, sizeof(g_create_err), "%s", m.c_str());
  }
  return s;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(ctx, LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CKL()                                                                           \
  do {                                                                                  \
    cudaError_t e_ = cudaGetLastError();                                                \
    if (e_ != cudaSuccess) return fail(ctx, LBM_ECUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
  } while (0)

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_step(lbm_ctx* c, const void* in, void* out, cudaStream_t s) {
  StepArgs a{in, out, c->pd, c->nprob, (int)c->ntiles, c->plane, c->lim, c->limf, c->tc_polls};
  const unsigned grid = c->ctas > 0 ? (unsigned)std::min<int64_t>(c->ctas, c->ntiles) : (unsigned)c->ntiles;
  if (c->dim == 1) {
    launch_step_d1(c->prec, c->stat, grid, s, a);
    return;
  }
  if (c->porous) {
    launch_step_porous(c->prec, c->stat, c->rows, grid, s, a);
    return;
  }
  if (c->inv == LBM_INV_SURROGATE) {
    const bool f32 = c->prec == LBM_F32_DEV;
    // the tensor-core kernels stage the network once per CTA: persistent grid
    if (c->surr_engine == LBM_SURROGATE_TENSOR_CORES) {
      const unsigned g = (unsigned)std::min<int64_t>(c->ctas > 0 ? c->ctas : c->tc_grid[c->rows], c->ntiles);
      if (f32) launch_step_surr_tc_f32(c->rows, g, s, a, c->surr_count, c->wtc);
      else launch_step_surr_tc_bf16(c->rows, g, s, a, c->surr_count, c->wtc);
    } else if (c->surr_engine == LBM_SURROGATE_WARP_MMA) {
      const unsigned g = (unsigned)std::min<int64_t>(c->ctas > 0 ? c->ctas : c->mm_grid[c->rows], c->ntiles);
      if (f32) launch_step_surr_mma_f32(c->rows, g, s, a, c->surr_count, c->wmm);
      else launch_step_surr_mma_bf16(c->rows, g, s, a, c->surr_count, c->wmm);
    } else {
      if (f32) launch_step_surr_f32(c->rows, grid, s, a, c->surr_count, *c->surr);
      else launch_step_surr_bf16(c->rows, grid, s, a, c->surr_count, *c->surr);
    }
    return;
  }
  if (c->inv == LBM_INV_EXACT_F64 && c->prec != LBM_F64) {  // deviation storage, FP64 inversion
    launch_step_x64(c->prec == LBM_F32_DEV, c->rows, grid, s, a);
    return;
  }
  switch (c->prec) {
    case LBM_F64: launch_step_f64(c->stat, c->rows, grid, s, a); break;
    case LBM_F32_DEV: launch_step_f32(c->stat, c->rows, grid, s, a); break;
    default: launch_step_bf16(c->stat, c->rows, grid, s, a); break;
  }
}

// Tile table for `rows` rows per tile: first tile of every problem, total.
int64_t layout_tiles(std::vector<ProbDev>& ph, int rows) {
  int64_t tiles = 0;
  for (auto& d : ph) {
    d.tile_begin = tiles;
    tiles += (int64_t)d.tiles_x * ((d.ny + rows - 1) / rows);
  }
  return tiles;
}

void drop_graphs(lbm_ctx* c) {
  for (int b = 0; b < 2; ++b) {
    if (c->graph[b]) cudaGraphExecDestroy(c->graph[b]);
    c->graph[b] = nullptr;
  }
}

template <class T>
void launch_init_t(lbm_ctx* c, const ProbDev& P, const InitDesc& d) {
  const int64_t cells = (int64_t)P.nx * P.ny;
  T* f = (T*)c->buf[c->cur];
  const unsigned g = blocks_for(cells, 256);
  // deviation storage: the FP32 equilibrium of the reduced-precision step
  if constexpr (Stor<T>::dev) {
    if (c->inv == LBM_INV_EXACT_F64) {  // FD statistics: the closure from t in FP64
      init_dev_kernel<T, STAT_FD, true><<<g, 256, 0, c->stream>>>(f, P, c->plane, d);
      return;
    }
    switch (c->stat) {
      case LBM_STAT_FD: init_dev_kernel<T, STAT_FD><<<g, 256, 0, c->stream>>>(f, P, c->plane, d); break;
      case LBM_STAT_FD_T0: init_dev_kernel<T, STAT_T0><<<g, 256, 0, c->stream>>>(f, P, c->plane, d); break;
      case LBM_STAT_FT: init_dev_kernel<T, STAT_FT><<<g, 256, 0, c->stream>>>(f, P, c->plane, d); break;
      default: init_dev_kernel<T, STAT_MB><<<g, 256, 0, c->stream>>>(f, P, c->plane, d); break;
    }
  } else {
    switch (c->stat) {
      case LBM_STAT_FD: init_kernel<T, STAT_FD><<<g, 256, 0, c->stream>>>(f, P, c->plane, d); break;
      case LBM_STAT_FD_T0: init_kernel<T, STAT_T0><<<g, 256, 0, c->stream>>>(f, P, c->plane, d); break;
      case LBM_STAT_FT: init_kernel<T, STAT_FT><<<g, 256, 0, c->stream>>>(f, P, c->plane, d); break;
      default: init_kernel<T, STAT_MB><<<g, 256, 0, c->stream>>>(f, P, c->plane, d); break;
    }
  }
}

template <class T, int STAT, class O>
void launch_moments_t(lbm_ctx* c, const ProbDev& P, O* o[6], unsigned g) {
  // deviation storage: error-free FP32 sums and the closure quantities from the FP32 inversion
  if constexpr (Stor<T>::dev)
    moments_dev_kernel<T, STAT, O><<<g, kMomThreads, 0, c->stream>>>(
        (const T*)c->buf[c->cur], P, c->plane, c->lim, c->limf, o[0], o[1], o[2], o[3], o[4], o[5], c->partials);
  else if constexpr (std::is_same<O, double>::value)  // FP64 storage reports FP64 arrays only
    moments_kernel<T, STAT><<<g, kMomThreads, 0, c->stream>>>(
        (const T*)c->buf[c->cur], P, c->plane, c->lim, c->limf, o[0], o[1], o[2], o[3], o[4], o[5], c->partials);
}

template <class T, class O>
void launch_moments_p(lbm_ctx* c, const ProbDev& P, O* o[6], unsigned g) {
  switch (c->stat) {
    case LBM_STAT_FD: launch_moments_t<T, STAT_FD, O>(c, P, o, g); break;
    case LBM_STAT_FD_T0: launch_moments_t<T, STAT_T0, O>(c, P, o, g); break;
    case LBM_STAT_FT: launch_moments_t<T, STAT_FT, O>(c, P, o, g); break;
    default: launch_moments_t<T, STAT_MB, O>(c, P, o, g); break;
  }
}

// T, mu, t of deviation-stored contexts with the FP64 inversion: overwrite
// what moments_dev_kernel wrote with the FP64 inversion of the same delta.
template <class O>
void launch_closure_x64(lbm_ctx* c, const ProbDev& P, O* const o[6]) {
  const unsigned g = blocks_for((int64_t)P.nx * P.ny, 256);
  if (c->prec == LBM_F32_DEV)
    closure_x64_kernel<float, O><<<g, 256, 0, c->stream>>>((const float*)c->buf[c->cur], P, c->plane, c->lim,
                                                            c->limf, o[3], o[4], o[5]);
  else
    closure_x64_kernel<__nv_bfloat16, O><<<g, 256, 0, c->stream>>>((const __nv_bfloat16*)c->buf[c->cur], P,
                                                                    c->plane, c->lim, c->limf, o[3], o[4], o[5]);
}

lbm_status ensure_tmp(lbm_ctx* ctx, int64_t doubles) {
  if (ctx->tmp_cap >= doubles) return LBM_OK;
  if (ctx->tmp) CK(cudaFree(ctx->tmp));
  ctx->tmp = nullptr;
  ctx->tmp_cap = 0;
  CK(cudaMalloc(&ctx->tmp, (size_t)doubles * sizeof(double)));
  ctx->tmp_cap = doubles;
  return LBM_OK;
}

bool valid_t(double t) { return t >= kTMin && t <= kTMax; }

// The device address of page-locked host memory that the GPU can reach
// directly (on a Grace-Blackwell node over the coherent chip-to-chip link),
// or NULL for pageable memory: kernels then read or write the caller's host
// array in place instead of going through a staging copy.
void* device_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of an unknown pointer
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer != nullptr) ? a.devicePointer : nullptr;
}

// lbm_moments and lbm_moments_f32: O is the output arrays' type.
template <class O>
lbm_status moments_impl(lbm_ctx* ctx, int32_t problem, O* const user[6], int32_t out_on_device, lbm_diag* diag,
                        const char* name) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, std::string(name) + ": NULL context");
  if (problem < 0 || problem >= ctx->nprob) return fail(ctx, LBM_EINVAL, std::string(name) + ": bad problem index");
  const ProbDev& P = ctx->ph[problem];
  const int64_t cells = (int64_t)P.nx * P.ny;
  const bool dev = ctx->dim == 2 && ctx->prec != LBM_F64;  // moments_dev_kernel: kMomDevCells per thread
  const unsigned g = blocks_for(cells, kMomThreads * (dev ? kMomDevCells : 1));
  if (ctx->partials_cap < (int64_t)g * kNPartial) {
    if (ctx->partials) CK(cudaFree(ctx->partials));
    ctx->partials = nullptr;
    ctx->partials_cap = 0;
    CK(cudaMalloc(&ctx->partials, sizeof(double) * kNPartial * g));
    ctx->partials_cap = (int64_t)g * kNPartial;
  }
  O* o[6] = {user[0], user[1], user[2], user[3], user[4], user[5]};
  bool staged[6] = {false, false, false, false, false, false};
  if (!out_on_device) {
    // page-locked host arrays are written in place by the kernel; the others
    // through device staging and a copy
    int nf = 0;
    for (int a = 0; a < 6; ++a) {
      if (!user[a]) continue;
      void* v = device_view(user[a]);
      if (v) {
        o[a] = (O*)v;
      } else {
        staged[a] = true;
        ++nf;
      }
    }
    if (nf > 0) {
      lbm_status s = ensure_tmp(ctx, nf * cells);  // doubles: room for nf arrays of O
      if (s != LBM_OK) return s;
    }
    O* const tmp = reinterpret_cast<O*>(ctx->tmp);
    int k = 0;
    for (int a = 0; a < 6; ++a)
      if (staged[a]) o[a] = tmp + (k++) * cells;
  }
  if (ctx->dim == 1) {
    if constexpr (std::is_same<O, double>::value)
      launch_moments_d1(ctx->prec, ctx->stat, ctx->buf[ctx->cur], P, ctx->plane, o, ctx->partials, g, ctx->stream);
  } else {
    switch (ctx->prec) {
      case LBM_F64: launch_moments_p<double, O>(ctx, P, o, g); break;
      case LBM_F32_DEV: launch_moments_p<float, O>(ctx, P, o, g); break;
      default: launch_moments_p<__nv_bfloat16, O>(ctx, P, o, g); break;
    }
  }
  CKL();
  ctx->launches += 1;
  if (ctx->dim == 2 && ctx->prec != LBM_F64 && ctx->inv == LBM_INV_EXACT_F64 && (o[3] || o[4] || o[5])) {
    launch_closure_x64<O>(ctx, P, o);
    CKL();
    ctx->launches += 1;
  }
  if (diag) {
    reduce_partials_kernel<<<1, 256, 0, ctx->stream>>>(ctx->partials, g, ctx->diag_d);
    CKL();
    ctx->launches += 1;
  }
  if (!out_on_device) {
    for (int a = 0; a < 6; ++a)
      if (staged[a]) CK(cudaMemcpyAsync(user[a], o[a], sizeof(O) * cells, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (diag) {
    double h[kNPartial];
    CK(cudaMemcpyAsync(h, ctx->diag_d, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    diag->sum_n = h[0];
    diag->sum_jx = h[1];
    diag->sum_jy = h[2];
    diag->sum_E = h[3];
    diag->clamped = (int64_t)h[4];
    diag->nonfinite = (int64_t)h[5];
  } else if (!out_on_device) {
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return LBM_OK;
}

}  // namespace

namespace lbm {
// Stores the message lbm_last_error(NULL) returns, for context-free calls;
// copies into a fixed buffer (allocates nothing).
void set_global_error(const char* m) {
  std::lock_guard<std::mutex> g(g_err_mu);
  std::snprintf(g_create_err, sizeof(g_create_err), "%s", m);
}
}  // namespace lbm

extern "C" {

const char* lbm_last_error(const lbm_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  std::lock_guard<std::mutex> g(g_err_mu);
  return g_create_err;
}

int64_t lbm_launch_count(const lbm_ctx* ctx) { return ctx ? ctx->launches : 0; }

lbm_status lbm_create(const lbm_params* p, void* cuda_stream, lbm_ctx** out) {
  lbm_ctx* ctx = nullptr;
  if (!p || !out) return fail(nullptr, LBM_EINVAL, "lbm_create: NULL argument");
  *out = nullptr;
  if (p->dim != 1 && p->dim != 2)
    return fail(nullptr, LBM_EUNSUPPORTED, "lbm_create: dim must be 1 (d1v3) or 2 (d2v9)");
  if (p->dim == 1 && (p->stat == LBM_STAT_FD || p->stat == LBM_STAT_FT))
    return fail(nullptr, LBM_EUNSUPPORTED,
                "lbm_create: d1v3 has no finite-temperature closure (n, j and E fix its three populations); "
                "use LBM_STAT_FD_T0 or LBM_STAT_MB");
  if (p->order != 3) return fail(nullptr, LBM_EUNSUPPORTED, "lbm_create: only order K = 3 is implemented");
  if (p->stat < 0 || p->stat > 3) return fail(nullptr, LBM_EINVAL, "lbm_create: bad stat");
  if (p->prec < 0 || p->prec > 2) return fail(nullptr, LBM_EINVAL, "lbm_create: bad prec");
  if (p->inv != LBM_INV_EXACT && p->inv != LBM_INV_SURROGATE && p->inv != LBM_INV_EXACT_F64)
    return fail(nullptr, LBM_EINVAL, "lbm_create: bad inv");
  if (p->inv == LBM_INV_EXACT_F64 && (p->stat != LBM_STAT_FD || p->dim != 2))
    return fail(nullptr, LBM_EUNSUPPORTED, "lbm_create: the FP64 inversion applies to LBM_STAT_FD on d2v9");
  if (p->inv == LBM_INV_SURROGATE && (p->prec == LBM_F64 || p->stat != LBM_STAT_FD || p->dim != 2))
    return fail(nullptr, LBM_EUNSUPPORTED,
                "lbm_create: the learned inversion needs LBM_STAT_FD with FP32 or BF16 deviation storage");
  if (p->nproblems < 1 || !p->problems) return fail(nullptr, LBM_EINVAL, "lbm_create: no problems");
  for (int i = 0; i < p->nproblems; ++i) {
    const lbm_problem& q = p->problems[i];
    if (q.nx < 1 || q.ny < 1) return fail(nullptr, LBM_EINVAL, "lbm_create: nx, ny must be >= 1");
    if (p->dim == 1 && q.ny != 1) return fail(nullptr, LBM_EINVAL, "lbm_create: d1v3 problems need ny = 1");
    if ((int64_t)q.nx * q.ny > ((int64_t)1 << 40)) return fail(nullptr, LBM_EINVAL, "lbm_create: problem too large");
    if (!(q.tau > 0.5) || !std::isfinite(q.tau)) return fail(nullptr, LBM_EINVAL, "lbm_create: tau must be > 1/2");
    if ((q.bc_x != 0 && q.bc_x != 1) || (q.bc_y != 0 && q.bc_y != 1))
      return fail(nullptr, LBM_EINVAL, "lbm_create: bad boundary kind");
    if (p->prec != LBM_F64 || p->stat == LBM_STAT_FT) {  // FT: theta = n_ref t_ref/(2 pi) at any precision
      if (!(q.n_ref > 0.0) || !std::isfinite(q.n_ref)) return fail(nullptr, LBM_EINVAL, "lbm_create: n_ref must be > 0");
      if ((p->stat == LBM_STAT_FD || p->stat == LBM_STAT_FT) && !valid_t(q.t_ref))
        return fail(nullptr, LBM_EINVAL, "lbm_create: t_ref must lie in [1e-3, 10]");
    }
  }
  ctx = new (std::nothrow) lbm_ctx();
  if (!ctx) return fail(nullptr, LBM_ENOMEM, "lbm_create: host allocation failed");
  ctx->stat = p->stat;
  ctx->prec = p->prec;
  ctx->dim = p->dim;
  ctx->q = p->dim == 1 ? 3 : 9;
  ctx->inv = p->inv;
  ctx->nprob = p->nproblems;
  ctx->probs.assign(p->problems, p->problems + p->nproblems);
  ctx->stream = (cudaStream_t)cuda_stream;
  int64_t base = 0;
  for (int i = 0; i < ctx->nprob; ++i) {
    const lbm_problem& q = ctx->probs[i];
    ProbDev d{};
    d.nx = q.nx;
    d.ny = q.ny;
    d.pitch = (q.nx + 31) / 32 * 32;
    d.bc_x = q.bc_x;
    d.bc_y = q.bc_y;
    d.tiles_x = (q.nx + kTileX - 1) / kTileX;
    d.base = base;
    d.tau = q.tau;
    d.omega = 1.0 / q.tau;
    d.theta = p->stat == LBM_STAT_FT ? q.n_ref * q.t_ref / (2.0 * kPi) : 0.0;
    d.n_ref = p->prec == LBM_F64 ? 0.0 : q.n_ref;
    d.t_ref = p->prec == LBM_F64 ? 0.0 : q.t_ref;
    base += (int64_t)d.pitch * q.ny;
    ctx->ph.push_back(d);
  }
  const int64_t tiles = layout_tiles(ctx->ph, ctx->rows);
  ctx->plane = (base + 31) / 32 * 32;
  ctx->ntiles = tiles;
  if (tiles > 0x7fffffffLL || ctx->plane > 0x7fffffffLL) {
    delete ctx;
    return fail(nullptr, LBM_EINVAL, "lbm_create: more than 2^31 cells in total is not supported");
  }
  auto cleanup = [&](lbm_status s, const std::string& m) {
    lbm_destroy(ctx);
    return fail(nullptr, s, m);
  };
  const size_t bytes = (size_t)ctx->plane * ctx->q * elem_size(ctx->prec);
  for (int b = 0; b < 2; ++b) {
    cudaError_t e = cudaMalloc(&ctx->buf[b], bytes);
    if (e != cudaSuccess) return cleanup(LBM_ENOMEM, std::string("lbm_create: population buffers: ") + cudaGetErrorString(e));
    e = cudaMemsetAsync(ctx->buf[b], 0, bytes, ctx->stream);
    if (e != cudaSuccess) return cleanup(LBM_ECUDA, std::string("lbm_create: memset: ") + cudaGetErrorString(e));
  }
  cudaError_t e = cudaMalloc(&ctx->pd, sizeof(ProbDev) * ctx->nprob);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->lim_d, sizeof(InvLimits));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->diag_d, sizeof(double) * kNPartial);
  if (e == cudaSuccess && p->inv == LBM_INV_SURROGATE) {
    e = cudaMalloc(&ctx->surr_count, kNSurrCounters * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->surr_count, 0, kNSurrCounters * sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->wtc, kTcBytes);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->wmm, kMmBytes);
    if (e == cudaSuccess) {
      int dev = 0, sms = 0;
      e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      for (int rows : {1, 2, 4, 8}) {
        const bool bf16 = p->prec == LBM_BF16_DEV;
        const int per_sm = e == cudaSuccess ? prepare_surr_tc(bf16, rows) : 0;
        const int per_sm_mm = e == cudaSuccess ? prepare_surr_mma(bf16, rows) : 0;
        if (e == cudaSuccess && (per_sm <= 0 || per_sm_mm <= 0)) e = cudaErrorInvalidConfiguration;
        ctx->tc_grid[rows] = (int64_t)per_sm * sms;
        ctx->mm_grid[rows] = (int64_t)per_sm_mm * sms;
      }
    }
  }
  if (e != cudaSuccess) return cleanup(LBM_ENOMEM, std::string("lbm_create: tables: ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(ctx->pd, ctx->ph.data(), sizeof(ProbDev) * ctx->nprob, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cleanup(LBM_ECUDA, std::string("lbm_create: upload: ") + cudaGetErrorString(e));
  setup_kernel<<<1, 1, 0, ctx->stream>>>(ctx->lim_d);
  ref_kernel<<<blocks_for(ctx->nprob, 64), 64, 0, ctx->stream>>>(ctx->pd, ctx->nprob, ctx->stat, ctx->dim);
  ctx->launches += 2;
  e = cudaMemcpyAsync(&ctx->lim, ctx->lim_d, sizeof(InvLimits), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->ph.data(), ctx->pd, sizeof(ProbDev) * ctx->nprob, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cleanup(LBM_ECUDA, std::string("lbm_create: setup: ") + cudaGetErrorString(e));
  ctx->limf = InvLimitsF{(float)ctx->lim.x_lo,  (float)ctx->lim.x_hi,  (float)ctx->lim.j2_lo,
                         (float)ctx->lim.j2_hi, (float)ctx->lim.j4_lo, (float)ctx->lim.j4_hi};
  e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cleanup(LBM_ECUDA, std::string("lbm_create: stream: ") + cudaGetErrorString(e));
  *out = ctx;
  return LBM_OK;
}

lbm_status lbm_init_riemann(lbm_ctx* ctx, int32_t problem, const lbm_riemann_desc* d) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_init_riemann: NULL context");
  if (!d) return fail(ctx, LBM_EINVAL, "lbm_init_riemann: NULL descriptor");
  if (problem < 0 || problem >= ctx->nprob) return fail(ctx, LBM_EINVAL, "lbm_init_riemann: bad problem index");
  const ProbDev& P = ctx->ph[problem];
  const int64_t cells = (int64_t)P.nx * P.ny;
  InitDesc k{};
  k.kind = d->kind;
  k.x0 = d->x0;
  k.y0 = d->y0;
  if (ctx->dim == 1 && d->kind == LBM_INIT_QUADRANT)
    return fail(ctx, LBM_EINVAL, "lbm_init_riemann: QUADRANT needs a two-dimensional lattice");
  if (d->kind == LBM_INIT_HALF || d->kind == LBM_INIT_QUADRANT) {
    const int ns = d->kind == LBM_INIT_HALF ? 2 : 4;
    for (int r = 0; r < ns; ++r) {
      const lbm_state& s = d->s[r];
      if (!(s.n > 0.0) || !std::isfinite(s.n) || !std::isfinite(s.ux) || !std::isfinite(s.uy))
        return fail(ctx, LBM_EINVAL, "lbm_init_riemann: region state needs n > 0 and finite u");
      if (ctx->stat == LBM_STAT_FD && !valid_t(s.t))
        return fail(ctx, LBM_EINVAL, "lbm_init_riemann: t must lie in [1e-3, 10]");
      k.s[r][0] = s.n;
      k.s[r][1] = s.ux;
      k.s[r][2] = s.uy;
      k.s[r][3] = s.t;
    }
  } else if (d->kind == LBM_INIT_FIELD) {
    if (!d->n || !d->ux || !d->uy || !d->t) return fail(ctx, LBM_EINVAL, "lbm_init_riemann: NULL field array");
    if (d->field_on_device) {
      k.n = d->n;
      k.ux = d->ux;
      k.uy = d->uy;
      k.t = d->t;
    } else {
      const double* src[4] = {d->n, d->ux, d->uy, d->t};
      void* view[4];
      bool direct = true;
      for (int a = 0; a < 4; ++a) direct = (view[a] = device_view(src[a])) != nullptr && direct;
      if (direct) {  // page-locked host fields: the kernel reads them in place
        k.n = (const double*)view[0];
        k.ux = (const double*)view[1];
        k.uy = (const double*)view[2];
        k.t = (const double*)view[3];
      } else {
        lbm_status s = ensure_tmp(ctx, 4 * cells);
        if (s != LBM_OK) return s;
        for (int a = 0; a < 4; ++a)
          CK(cudaMemcpyAsync(ctx->tmp + a * cells, src[a], sizeof(double) * cells, cudaMemcpyHostToDevice,
                             ctx->stream));
        k.n = ctx->tmp;
        k.ux = ctx->tmp + cells;
        k.uy = ctx->tmp + 2 * cells;
        k.t = ctx->tmp + 3 * cells;
      }
    }
  } else {
    return fail(ctx, LBM_EINVAL, "lbm_init_riemann: bad kind");
  }
  if (ctx->dim == 1) {
    launch_init_d1(ctx->prec, ctx->stat, ctx->buf[ctx->cur], P, ctx->plane, k, ctx->stream);
  } else {
    switch (ctx->prec) {
      case LBM_F64: launch_init_t<double>(ctx, P, k); break;
      case LBM_F32_DEV: launch_init_t<float>(ctx, P, k); break;
      default: launch_init_t<__nv_bfloat16>(ctx, P, k); break;
    }
  }
  CKL();
  ctx->launches += 1;
  if (d->kind == LBM_INIT_FIELD && !d->field_on_device) CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

lbm_status lbm_init_fields_f32(lbm_ctx* ctx, int32_t problem, const float* n, const float* ux, const float* uy,
                               const float* t, int32_t on_device) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_init_fields_f32: NULL context");
  if (problem < 0 || problem >= ctx->nprob) return fail(ctx, LBM_EINVAL, "lbm_init_fields_f32: bad problem index");
  if (ctx->dim != 2 || ctx->prec == LBM_F64)
    return fail(ctx, LBM_EUNSUPPORTED, "lbm_init_fields_f32: needs d2v9 with FP32 or BF16 deviation storage");
  if (!n || !ux || !uy || !t) return fail(ctx, LBM_EINVAL, "lbm_init_fields_f32: NULL field array");
  const ProbDev& P = ctx->ph[problem];
  const int64_t cells = (int64_t)P.nx * P.ny;
  InitDesc k{};
  k.kind = 3;  // FIELD, float arrays
  if (on_device) {
    k.nf = n;
    k.uxf = ux;
    k.uyf = uy;
    k.tf = t;
  } else {
    const float* src[4] = {n, ux, uy, t};
    void* view[4];
    bool direct = true;
    for (int a = 0; a < 4; ++a) direct = (view[a] = device_view(src[a])) != nullptr && direct;
    if (direct) {  // page-locked host fields: the kernel reads them in place
      k.nf = (const float*)view[0];
      k.uxf = (const float*)view[1];
      k.uyf = (const float*)view[2];
      k.tf = (const float*)view[3];
    } else {
      lbm_status s = ensure_tmp(ctx, 2 * cells);  // doubles: room for four float arrays
      if (s != LBM_OK) return s;
      float* const tmp = reinterpret_cast<float*>(ctx->tmp);
      for (int a = 0; a < 4; ++a)
        CK(cudaMemcpyAsync(tmp + a * cells, src[a], sizeof(float) * cells, cudaMemcpyHostToDevice, ctx->stream));
      k.nf = tmp;
      k.uxf = tmp + cells;
      k.uyf = tmp + 2 * cells;
      k.tf = tmp + 3 * cells;
    }
  }
  if (ctx->prec == LBM_F32_DEV) launch_init_t<float>(ctx, P, k);
  else launch_init_t<__nv_bfloat16>(ctx, P, k);
  CKL();
  ctx->launches += 1;
  if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* ctx, int32_t nsteps) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_step: NULL context");
  if (nsteps < 0) return fail(ctx, LBM_EINVAL, "lbm_step: nsteps < 0");
  if (ctx->inv == LBM_INV_SURROGATE && !ctx->surr)
    return fail(ctx, LBM_EINVAL, "lbm_step: load the network with lbm_surrogate_load first");
  while (nsteps >= kGraphChunk) {
    cudaGraphExec_t& ge = ctx->graph[ctx->cur];
    if (!ge) {
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
      int c = ctx->cur;
      for (int s = 0; s < kGraphChunk; ++s) {
        launch_step(ctx, ctx->buf[c], ctx->buf[c ^ 1], ctx->cap);
        c ^= 1;
      }
      cudaError_t le = cudaGetLastError();
      cudaError_t ee = cudaStreamEndCapture(ctx->cap, &g);
      if (le != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(ctx, LBM_ECUDA, std::string("lbm_step: capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ee));
      }
      cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        ge = nullptr;
        return fail(ctx, LBM_ECUDA, std::string("lbm_step: instantiate: ") + cudaGetErrorString(ie));
      }
    }
    CK(cudaGraphLaunch(ge, ctx->stream));
    ctx->launches += kGraphChunk;
    nsteps -= kGraphChunk;
  }
  for (int s = 0; s < nsteps; ++s) {
    launch_step(ctx, ctx->buf[ctx->cur], ctx->buf[ctx->cur ^ 1], ctx->stream);
    CKL();
    ctx->cur ^= 1;
    ctx->launches += 1;
  }
  return LBM_OK;
}

namespace {

lbm_status apply_tiling(lbm_ctx* ctx, int rows, int ctas) {
  std::vector<ProbDev> ph = ctx->ph;
  const int64_t tiles = layout_tiles(ph, rows);
  if (tiles > 0x7fffffffLL) return fail(ctx, LBM_EINVAL, "lbm_set_tiling: too many tiles");
  CK(cudaMemcpyAsync(ctx->pd, ph.data(), sizeof(ProbDev) * ctx->nprob, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));  // the host copy `ph` must outlive the transfer
  ctx->ph = ph;
  ctx->ntiles = tiles;
  ctx->rows = rows;
  ctx->ctas = ctas;
  drop_graphs(ctx);
  return LBM_OK;
}

}  // namespace

lbm_status lbm_set_tiling(lbm_ctx* ctx, int32_t rows_per_tile, int32_t ctas) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_set_tiling: NULL context");
  if (!valid_rows(rows_per_tile)) return fail(ctx, LBM_EINVAL, "lbm_set_tiling: rows_per_tile must be 1, 2, 4 or 8");
  if (ctas < 0) return fail(ctx, LBM_EINVAL, "lbm_set_tiling: ctas must be >= 0");
  return apply_tiling(ctx, rows_per_tile, ctas);
}

lbm_status lbm_get_tiling(const lbm_ctx* ctx, lbm_tiling* out) {
  if (!ctx || !out) return LBM_EINVAL;
  out->rows_per_tile = ctx->rows;
  out->ctas = ctx->ctas;
  out->ms_per_step = 0.0;
  return LBM_OK;
}

namespace {

// The network's FP16 tensor-core operands (layout in surrogate.cuh).  A value
// v enters as hi = fp16(v) and lo = fp16(v - hi).
std::vector<__half> pack_tc_operands(const float* p) {
  std::vector<__half> out(kTcBytes / 2, __float2half_rn(0.0f));
  auto put = [&](int base, int R, int r, int k, float v) { out[(base + tc_operand_byte(r, k, R)) / 2] = __float2half_rn(v); };
  auto hi = [](float v) { return __half2float(__float2half_rn(v)); };
  for (int j = 0; j < kH; ++j) {
    const float wn = 0.5f * p[kOW1 + 2 * j], wl = 0.5f * p[kOW1 + 2 * j + 1], b = 0.5f * p[kOB1 + j];
    const float row[8] = {hi(wn), hi(wn), wn - hi(wn), hi(wl), hi(wl), wl - hi(wl), hi(b), b - hi(b)};
    for (int k = 0; k < 8; ++k) put(kTcB1, kH, j, k, row[k]);
    for (int k = 0; k < kH; ++k) put(kTcB2, kH, j, k, 0.5f * p[kOW2 + kH * j + k]);
    const float b2 = 0.5f * p[kOB2 + j];
    put(kTcB2b, kH, j, 6, hi(b2));
    put(kTcB2b, kH, j, 7, b2 - hi(b2));
  }
  for (int o = 0; o < 2; ++o) {
    for (int k = 0; k < kH; ++k) {
      const float w = p[kOW3 + kH * o + k];
      put(kTcB3, 16, o, k, hi(w));
      put(kTcB3, 16, 2 + o, k, w - hi(w));
    }
    const float b3 = p[kOB3 + o];
    put(kTcB3b, 16, o, 6, hi(b3));
    put(kTcB3b, 16, o, 7, b3 - hi(b3));
  }
  return out;
}

// The network's warp-MMA fragments (layout in surrogate.cuh), as 32-bit words:
// two FP16 values per word, the lower k in the low half.
std::vector<uint32_t> pack_mma_operands(const float* p) {
  std::vector<uint32_t> out(kMmBytes / 4, 0u);
  auto h16 = [](float v) { const __half h = __float2half_rn(v); return (uint32_t)*reinterpret_cast<const uint16_t*>(&h); };
  auto pair = [&](float lo_k, float hi_k) { return h16(lo_k) | (h16(hi_k) << 16); };
  auto hi = [](float v) { return __half2float(__float2half_rn(v)); };
  auto f32 = [](float v) { uint32_t u; std::memcpy(&u, &v, 4); return u; };
  // layer-1 rows: the 8 features of hidden unit j (W1/2 and b1/2 split hi/lo)
  float w1[kH][8];
  for (int j = 0; j < kH; ++j) {
    const float wn = 0.5f * p[kOW1 + 2 * j], wl = 0.5f * p[kOW1 + 2 * j + 1], b = 0.5f * p[kOB1 + j];
    const float row[8] = {hi(wn), hi(wn), wn - hi(wn), hi(wl), hi(wl), wl - hi(wl), hi(b), b - hi(b)};
    for (int k = 0; k < 8; ++k) w1[j][k] = row[k];
  }
  for (int lane = 0; lane < 32; ++lane) {
    const int g = lane / 4, t = lane % 4;
    for (int q = 0; q < 4; ++q)
      for (int h = 0; h < 2; ++h) {
        const int n = 8 * (2 * q + h) + g;
        out[(kMmB1 + (q * 32 + lane) * 8) / 4 + h] = pair(w1[n][2 * t], w1[n][2 * t + 1]);
      }
    // layer 2: element (k, n) = W2[n][k]/2
    auto w2 = [&](int k, int n) { return 0.5f * p[kOW2 + kH * n + k]; };
    for (int c = 0; c < 4; ++c)
      for (int q = 0; q < 4; ++q)
        for (int h = 0; h < 2; ++h) {
          const int n = 8 * (2 * q + h) + g, k = 16 * c + 2 * t;
          const int w = (kMmB2 + ((c * 4 + q) * 32 + lane) * 16) / 4 + 2 * h;
          out[w] = pair(w2(k, n), w2(k + 1, n));
          out[w + 1] = pair(w2(k + 8, n), w2(k + 9, n));
        }
    // layer 3: element (k, n) = W3[n][k] for n = 0, 1, as hi and lo parts
    auto w3 = [&](int k, int n, bool lo) {
      if (n > 1) return 0.0f;
      const float v = p[kOW3 + kH * n + k];
      return lo ? v - hi(v) : hi(v);
    };
    for (int c = 0; c < 4; ++c)
      for (int h = 0; h < 2; ++h) {
        const int k = 16 * c + 2 * t, w = (kMmB3 + (c * 32 + lane) * 16) / 4 + 2 * h;
        out[w] = pair(w3(k, g, h == 1), w3(k + 1, g, h == 1));
        out[w + 1] = pair(w3(k + 8, g, h == 1), w3(k + 9, g, h == 1));
      }
  }
  for (int q = 0; q < 4; ++q)
    for (int t = 0; t < 4; ++t)
      for (int h = 0; h < 2; ++h) {
        const int nt = 2 * q + h;
        out[(kMmC2 + (q * 4 + t) * 8) / 4 + h] = pair(0.5f * p[kOB2 + 8 * nt + 2 * t], 0.5f * p[kOB2 + 8 * nt + 2 * t + 1]);
      }
  out[kMmC3 / 4] = f32(p[kOB3]);
  out[kMmC3 / 4 + 1] = f32(p[kOB3 + 1]);
  return out;
}

}  // namespace

lbm_status lbm_surrogate_load(lbm_ctx* ctx, const float* params) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_surrogate_load: NULL context");
  if (!params) return fail(ctx, LBM_EINVAL, "lbm_surrogate_load: NULL parameters");
  if (ctx->inv != LBM_INV_SURROGATE)
    return fail(ctx, LBM_EINVAL, "lbm_surrogate_load: the context was created with the exact inversion");
  for (int i = 0; i < kNParam; ++i)
    if (!std::isfinite(params[i])) return fail(ctx, LBM_EINVAL, "lbm_surrogate_load: non-finite parameter");
  if (!ctx->surr) ctx->surr = new (std::nothrow) MlpParams();
  if (!ctx->surr) return fail(ctx, LBM_ENOMEM, "lbm_surrogate_load: host allocation failed");
  std::memcpy(ctx->surr->p, params, sizeof(float) * kNParam);
  const std::vector<__half> wtc = pack_tc_operands(params);
  const std::vector<uint32_t> wmm = pack_mma_operands(params);
  CK(cudaMemcpyAsync(ctx->wtc, wtc.data(), kTcBytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(ctx->wmm, wmm.data(), kMmBytes, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  drop_graphs(ctx);
  return LBM_OK;
}

lbm_status lbm_surrogate_engine(lbm_ctx* ctx, int32_t engine) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_surrogate_engine: NULL context");
  if (engine != LBM_SURROGATE_FP32_PIPE && engine != LBM_SURROGATE_TENSOR_CORES && engine != LBM_SURROGATE_WARP_MMA)
    return fail(ctx, LBM_EINVAL, "lbm_surrogate_engine: bad engine");
  ctx->surr_engine = engine;
  drop_graphs(ctx);
  return LBM_OK;
}

lbm_status lbm_surrogate_stats(lbm_ctx* ctx, int64_t* fallbacks, int64_t* evaluations) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_surrogate_stats: NULL context");
  if (!ctx->surr_count) return fail(ctx, LBM_EINVAL, "lbm_surrogate_stats: not a learned-inversion context");
  unsigned long long h[kNSurrCounters] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(h, ctx->surr_count, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (fallbacks) *fallbacks = (int64_t)h[0];
  if (evaluations) *evaluations = (int64_t)h[1];
  if (h[3])
    return fail(ctx, LBM_ETIMEOUT,
                "lbm_surrogate_stats: a tensor-core wait before freeing tensor memory timed out; the results of "
                "the steps since the context was created are not trusted");
  if (h[2]) return fail(ctx, LBM_ETIMEOUT, "lbm_surrogate_stats: a tensor-core wait timed out (cells served exactly)");
  return LBM_OK;
}

lbm_status lbm_surrogate_wait_limit(lbm_ctx* ctx, int32_t polls) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_surrogate_wait_limit: NULL context");
  ctx->tc_polls = polls < 0 ? kTcWaitPolls : (int)polls;
  drop_graphs(ctx);
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx* ctx, int32_t steps_per_candidate, lbm_tiling* chosen) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_autotune: NULL context");
  if (ctx->inv == LBM_INV_SURROGATE && !ctx->surr)
    return fail(ctx, LBM_EINVAL, "lbm_autotune: load the network with lbm_surrogate_load first");
  if (steps_per_candidate < 1) return fail(ctx, LBM_EINVAL, "lbm_autotune: steps_per_candidate must be >= 1");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int rows_c[4] = {1, 2, 4, 8};
  const int ctas_c[4] = {0, 4 * sms, 8 * sms, 16 * sms};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  double best = 1e300;
  int best_r = ctx->rows, best_c = ctx->ctas;
  lbm_status st = LBM_OK;
  // Every candidate reads the current buffer and writes the other one only:
  // the state the caller sees does not change.
  for (int ri = 0; ri < 4 && st == LBM_OK; ++ri) {
    for (int ci = 0; ci < 4 && st == LBM_OK; ++ci) {
      st = apply_tiling(ctx, rows_c[ri], ctas_c[ci]);
      if (st != LBM_OK) break;
      launch_step(ctx, ctx->buf[ctx->cur], ctx->buf[ctx->cur ^ 1], ctx->stream);
      cudaEventRecord(e0, ctx->stream);
      for (int k = 0; k < steps_per_candidate; ++k)
        launch_step(ctx, ctx->buf[ctx->cur], ctx->buf[ctx->cur ^ 1], ctx->stream);
      cudaEventRecord(e1, ctx->stream);
      ctx->launches += steps_per_candidate + 1;
      cudaError_t e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) {
        st = fail(ctx, LBM_ECUDA, std::string("lbm_autotune: ") + cudaGetErrorString(e));
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double per = (double)ms / steps_per_candidate;
      if (per < best) {
        best = per;
        best_r = rows_c[ri];
        best_c = ctas_c[ci];
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != LBM_OK) return st;
  st = apply_tiling(ctx, best_r, best_c);
  if (st != LBM_OK) return st;
  if (chosen) {
    chosen->rows_per_tile = best_r;
    chosen->ctas = best_c;
    chosen->ms_per_step = best;
  }
  return LBM_OK;
}

lbm_status lbm_moments(lbm_ctx* ctx, int32_t problem, double* n, double* ux, double* uy, double* T, double* mu,
                       double* t, int32_t out_on_device, lbm_diag* diag) {
  double* const user[6] = {n, ux, uy, T, mu, t};
  return moments_impl<double>(ctx, problem, user, out_on_device, diag, "lbm_moments");
}

lbm_status lbm_moments_f32(lbm_ctx* ctx, int32_t problem, float* n, float* ux, float* uy, float* T, float* mu,
                           float* t, int32_t out_on_device, lbm_diag* diag) {
  if (ctx && (ctx->dim != 2 || ctx->prec == LBM_F64))
    return fail(ctx, LBM_EUNSUPPORTED, "lbm_moments_f32: needs d2v9 with FP32 or BF16 deviation storage");
  float* const user[6] = {n, ux, uy, T, mu, t};
  return moments_impl<float>(ctx, problem, user, out_on_device, diag, "lbm_moments_f32");
}

lbm_status lbm_get_populations(lbm_ctx* ctx, int32_t problem, double* f, int32_t on_device) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_get_populations: NULL context");
  if (problem < 0 || problem >= ctx->nprob || !f) return fail(ctx, LBM_EINVAL, "lbm_get_populations: bad argument");
  const ProbDev& P = ctx->ph[problem];
  const int64_t cells = (int64_t)P.nx * P.ny;
  double* dst = f;
  if (!on_device) {
    lbm_status s = ensure_tmp(ctx, ctx->q * cells);
    if (s != LBM_OK) return s;
    dst = ctx->tmp;
  }
  const unsigned g = blocks_for(cells, 256);
  if (ctx->dim == 1) launch_pop_d1(ctx->prec, true, ctx->buf[ctx->cur], P, ctx->plane, dst, ctx->stream);
  else switch (ctx->prec) {
    case LBM_F64: get_pop_kernel<double><<<g, 256, 0, ctx->stream>>>((const double*)ctx->buf[ctx->cur], P, ctx->plane, dst); break;
    case LBM_F32_DEV: get_pop_kernel<float><<<g, 256, 0, ctx->stream>>>((const float*)ctx->buf[ctx->cur], P, ctx->plane, dst); break;
    default: get_pop_kernel<__nv_bfloat16><<<g, 256, 0, ctx->stream>>>((const __nv_bfloat16*)ctx->buf[ctx->cur], P, ctx->plane, dst); break;
  }
  CKL();
  ctx->launches += 1;
  if (!on_device) {
    CK(cudaMemcpyAsync(f, dst, sizeof(double) * ctx->q * cells, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* ctx, int32_t problem, const double* f, int32_t on_device) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_set_populations: NULL context");
  if (problem < 0 || problem >= ctx->nprob || !f) return fail(ctx, LBM_EINVAL, "lbm_set_populations: bad argument");
  const ProbDev& P = ctx->ph[problem];
  const int64_t cells = (int64_t)P.nx * P.ny;
  const double* src = f;
  if (!on_device) {
    lbm_status s = ensure_tmp(ctx, ctx->q * cells);
    if (s != LBM_OK) return s;
    CK(cudaMemcpyAsync(ctx->tmp, f, sizeof(double) * ctx->q * cells, cudaMemcpyHostToDevice, ctx->stream));
    src = ctx->tmp;
  }
  const unsigned g = blocks_for(cells, 256);
  if (ctx->dim == 1) launch_pop_d1(ctx->prec, false, ctx->buf[ctx->cur], P, ctx->plane, (double*)src, ctx->stream);
  else switch (ctx->prec) {
    case LBM_F64: set_pop_kernel<double><<<g, 256, 0, ctx->stream>>>((double*)ctx->buf[ctx->cur], P, ctx->plane, src); break;
    case LBM_F32_DEV: set_pop_kernel<float><<<g, 256, 0, ctx->stream>>>((float*)ctx->buf[ctx->cur], P, ctx->plane, src); break;
    default: set_pop_kernel<__nv_bfloat16><<<g, 256, 0, ctx->stream>>>((__nv_bfloat16*)ctx->buf[ctx->cur], P, ctx->plane, src); break;
  }
  CKL();
  ctx->launches += 1;
  if (!on_device) CK(cudaStreamSynchronize(ctx->stream));
  return LBM_OK;
}

namespace {

// Re-upload the problem table after a host-side change and pick the step kernel.
lbm_status upload_problems(lbm_ctx* ctx) {
  ctx->porous = false;
  for (const ProbDev& P : ctx->ph) ctx->porous = ctx->porous || P.solid != nullptr || P.fx != 0.0 || P.fy != 0.0;
  CK(cudaMemcpyAsync(ctx->pd, ctx->ph.data(), sizeof(ProbDev) * ctx->nprob, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  drop_graphs(ctx);
  return LBM_OK;
}

lbm_status porous_allowed(lbm_ctx* ctx, const char* who) {
  if (ctx->dim != 2) return fail(ctx, LBM_EUNSUPPORTED, std::string(who) + ": obstacles and forces need d2v9");
  if (ctx->inv != LBM_INV_EXACT)
    return fail(ctx, LBM_EUNSUPPORTED, std::string(who) + ": obstacles and forces need the exact inversion");
  if (ctx->stat == LBM_STAT_FT)
    return fail(ctx, LBM_EUNSUPPORTED, std::string(who) + ": obstacles and forces are not built for LBM_STAT_FT");
  return LBM_OK;
}

}  // namespace

lbm_status lbm_set_obstacles(lbm_ctx* ctx, int32_t problem, const uint8_t* solid, int32_t on_device) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_set_obstacles: NULL context");
  if (problem < 0 || problem >= ctx->nprob) return fail(ctx, LBM_EINVAL, "lbm_set_obstacles: bad problem index");
  lbm_status st = porous_allowed(ctx, "lbm_set_obstacles");
  if (st != LBM_OK) return st;
  ProbDev& P = ctx->ph[problem];
  if (!solid) {
    P.solid = nullptr;
    P.pcode = nullptr;
    return upload_problems(ctx);
  }
  if (!ctx->mask) {
    CK(cudaMalloc(&ctx->mask, (size_t)ctx->plane));
    CK(cudaMemsetAsync(ctx->mask, 0, (size_t)ctx->plane, ctx->stream));
  }
  if (!ctx->pcode) CK(cudaMalloc(&ctx->pcode, sizeof(uint16_t) * (size_t)ctx->plane));
  CK(cudaMemcpy2DAsync(ctx->mask + P.base, (size_t)P.pitch, solid, (size_t)P.nx, (size_t)P.nx, (size_t)P.ny,
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  P.solid = ctx->mask;
  P.pcode = ctx->pcode;
  launch_pull_code(P, ctx->pcode, ctx->stream);  // from the mask just copied, in stream order
  ++ctx->launches;
  CKL();
  return upload_problems(ctx);
}

lbm_status lbm_set_force(lbm_ctx* ctx, int32_t problem, double fx, double fy) {
  if (!ctx) return fail(nullptr, LBM_EINVAL, "lbm_set_force: NULL context");
  if (problem < 0 || problem >= ctx->nprob) return fail(ctx, LBM_EINVAL, "lbm_set_force: bad problem index");
  if (!std::isfinite(fx) || !std::isfinite(fy)) return fail(ctx, LBM_EINVAL, "lbm_set_force: non-finite force");
  lbm_status st = porous_allowed(ctx, "lbm_set_force");
  if (st != LBM_OK) return st;
  ProbDev& P = ctx->ph[problem];
  P.fx = fx;
  P.fy = fy;
  P.f.fx = (float)fx;
  P.f.fy = (float)fy;
  return upload_problems(ctx);
}

lbm_status lbm_destroy(lbm_ctx* ctx) {
  if (!ctx) return LBM_OK;
  cudaStreamSynchronize(ctx->stream);
  drop_graphs(ctx);
  for (int b = 0; b < 2; ++b) {
    if (ctx->buf[b]) cudaFree(ctx->buf[b]);
  }
  if (ctx->pd) cudaFree(ctx->pd);
  if (ctx->lim_d) cudaFree(ctx->lim_d);
  if (ctx->diag_d) cudaFree(ctx->diag_d);
  if (ctx->partials) cudaFree(ctx->partials);
  if (ctx->tmp) cudaFree(ctx->tmp);
  if (ctx->cap) cudaStreamDestroy(ctx->cap);
  if (ctx->surr_count) cudaFree(ctx->surr_count);
  if (ctx->wtc) cudaFree(ctx->wtc);
  if (ctx->wmm) cudaFree(ctx->wmm);
  if (ctx->mask) cudaFree(ctx->mask);
  if (ctx->pcode) cudaFree(ctx->pcode);
  delete ctx->surr;
  delete ctx;
  return LBM_OK;
}

}  // extern "C"
