// Kernels of the d1v3 lattice (D = 1, Sect. "The Gaussian quadrature"):
// velocities e = 0, +1, -1 in planes 0, 1, 2, weights W_0 = n (1 - J_2/3),
// W_+-1 = n J_2/6.  Closures with constant J_N (there is no finite-temperature
// closure through the energy on three velocities): theta = 0, J_2 = 5/3,
// J_4 = 7/5 (J_N = 1 + 2/(N + D)); Maxwell-Boltzmann, J_2 = J_4 = 1.
//
// The K = 3 equilibrium in geometric velocities at D = 1, with
// Delta_2^2 = 2/((D + 2) - J_2 D) = 2/(3 - J_2): on the moving velocities
// (e^2 = 1, e u = +-u) the third-order bracket
//   3 (1 - J_2) J_4 D42 - 3 (1 - J_2) J_4 D42 e^2 - 3 J_4 D42 u^2
//   + 3 J_4 (D42 - 1) u^2 e^2 + 3 J_4 (e u)^2
// vanishes identically, so
//   f_0   = W_0 (1 - (3/2) Delta_2^2 u^2),
//   f_+-1 = W_+-1 (1 +- (3/J_2) u + (3/2) Delta_2^2 (3/J_2 - 1) u^2),
// and J_4 does not enter.  Layout as for d2v9 (one row per problem, ny = 1):
// plane a holds the cells of every problem at base_p + x.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_kernels.cuh"

namespace lbm {

// FP32 arithmetic on the stored deviations.
template <class T>
struct Dev1;
template <>
struct Dev1<float> {
  __device__ static __forceinline__ float ld(float v) { return v; }
  __device__ static __forceinline__ float st(float v) { return v; }
};
template <>
struct Dev1<__nv_bfloat16> {
  __device__ static __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __forceinline__ __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};

template <int STAT>
struct FixedJ1 {
  static constexpr double j2 = STAT == STAT_T0 ? 5.0 / 3.0 : 1.0;
};

// Equilibrium coefficients: f_0 = W_0 (1 + c0 u^2), f_+-1 = W_1 (1 +- a u + b u^2).
template <int STAT>
struct Feq1 {
  static constexpr double j2 = FixedJ1<STAT>::j2;
  static constexpr double d22 = 2.0 / (3.0 - j2);
  static constexpr double w0 = 1.0 - j2 / 3.0, w1 = j2 / 6.0;  // W / n
  static constexpr double c0 = -1.5 * d22;
  static constexpr double a = 3.0 / j2;
  static constexpr double b = 1.5 * d22 * (3.0 / j2 - 1.0);
};

// Pulled populations of cell x (periodic wrap or halfway bounce-back).
template <class T>
__device__ __forceinline__ void pull3(const T* __restrict__ fin, int64_t plane, const ProbDev& P, int x, T v[3]) {
  const int64_t c = P.base + x;
  const int xm = x > 0 ? x - 1 : (P.bc_x == BC_PERIODIC ? P.nx - 1 : -1);
  const int xp = x < P.nx - 1 ? x + 1 : (P.bc_x == BC_PERIODIC ? 0 : -1);
  v[0] = fin[c];
  v[1] = xm >= 0 ? fin[plane + P.base + xm] : fin[2 * plane + c];
  v[2] = xp >= 0 ? fin[2 * plane + P.base + xp] : fin[plane + c];
}

// Tiles of 128 cells per CTA and sweep: the loads of all of them are issued
// before the first collision, so each thread keeps 3 kTilesD1 loads in flight.
constexpr int kTilesD1 = 4;

// Collision of one cell from its pulled populations v (BGK on the closed-form
// equilibrium above); stores at c.  FP64: absolute populations.  FP32 / BF16:
// deviations g = f - W^ref with W^ref = w(J_2) n_ref; then dn = sum g,
// j = g_+1 - g_-1 and g_eq = w dn + W (S - 1) without forming f.
template <class T, int STAT>
__device__ __forceinline__ void collide_store_d1(const ProbDev& P, const T v[3], T* __restrict__ fout, int64_t plane,
                                                 int64_t c) {
  using K = Feq1<STAT>;
  if constexpr (Stor<T>::dev) {
    const float g0 = Dev1<T>::ld(v[0]), g1 = Dev1<T>::ld(v[1]), g2 = Dev1<T>::ld(v[2]);
    const float dn = (g0 + g1) + g2;
    const float n = P.f.n_ref + dn;
    const float u = __fdividef(g1 - g2, n);
    const float u2 = u * u;
    const float W0 = (float)K::w0 * n, W1 = (float)K::w1 * n;
    const float e0 = (float)K::w0 * dn + W0 * ((float)K::c0 * u2);
    const float ep = (float)K::w1 * dn + W1 * (u * ((float)K::a + (float)K::b * u));
    const float em = (float)K::w1 * dn + W1 * (u * (-(float)K::a + (float)K::b * u));
    const float w = P.f.omega;
    fout[c] = Dev1<T>::st(fmaf(w, e0 - g0, g0));
    fout[plane + c] = Dev1<T>::st(fmaf(w, ep - g1, g1));
    fout[2 * plane + c] = Dev1<T>::st(fmaf(w, em - g2, g2));
  } else {
    const double f0 = v[0], f1 = v[1], f2 = v[2];
    const double n = (f0 + f1) + f2;
    const double u = (f1 - f2) / n;
    const double u2 = u * u;
    const double W0 = K::w0 * n, W1 = K::w1 * n;
    const double e0 = W0 * (1.0 + K::c0 * u2);
    const double ep = W1 * (1.0 + u * (K::a + K::b * u));
    const double em = W1 * (1.0 + u * (-K::a + K::b * u));
    const double w = P.omega;
    fout[c] = f0 + w * (e0 - f0);
    fout[plane + c] = f1 + w * (ep - f1);
    fout[2 * plane + c] = f2 + w * (em - f2);
  }
}

// One sweep covers kTilesD1 tiles: CTA b takes tiles b, b + G, b + 2 G, ...
// (G = gridDim.x, so consecutive CTAs read consecutive tiles) and, for
// PERSIST, repeats with the base advanced by kTilesD1 G.
template <class T, int STAT, bool PERSIST>
__global__ void __launch_bounds__(kTileX) stream_collide_d1(const T* __restrict__ fin, T* __restrict__ fout,
                                                            const ProbDev* __restrict__ probs, int nprob, int ntiles,
                                                            int64_t plane) {
  const int G = (int)gridDim.x;
#pragma unroll 1
  for (int t0 = (int)blockIdx.x; t0 < ntiles; t0 += kTilesD1 * G) {
    T v[kTilesD1][3];
    int64_t c[kTilesD1];
    int pi[kTilesD1];
#pragma unroll
    for (int u = 0; u < kTilesD1; ++u) {
      const int tile = t0 + u * G;
      c[u] = -1;
      pi[u] = 0;
      if (tile < ntiles) {
        pi[u] = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
        const ProbDev& P = probs[pi[u]];
        const int x = (tile - (int)P.tile_begin) * kTileX + (int)threadIdx.x;
        if (x < P.nx) {
          pull3(fin, plane, P, x, v[u]);
          c[u] = P.base + x;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kTilesD1; ++u)
      if (c[u] >= 0) collide_store_d1<T, STAT>(probs[pi[u]], v[u], fout, plane, c[u]);
    if (!PERSIST) break;
  }
}

// f_eq of a state (n, u) in FP64.
template <int STAT>
__device__ __forceinline__ void feq1_f64(double n, double u, double fe[3]) {
  using K = Feq1<STAT>;
  fe[0] = K::w0 * n * (1.0 + K::c0 * u * u);
  fe[1] = K::w1 * n * (1.0 + u * (K::a + K::b * u));
  fe[2] = K::w1 * n * (1.0 + u * (-K::a + K::b * u));
}

template <class T, int STAT>
__global__ void init_d1_kernel(T* __restrict__ f, ProbDev P, int64_t plane, InitDesc d) {
  const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (x >= P.nx) return;
  double n, u;
  if (d.kind == 2) {
    n = d.n[x];
    u = d.ux[x];
  } else {
    const int r = x >= d.x0;
    n = d.s[r][0];
    u = d.s[r][1];
  }
  double fe[3];
  feq1_f64<STAT>(n, u, fe);
  const int64_t c = P.base + x;
#pragma unroll
  for (int a = 0; a < 3; ++a) f[a * plane + c] = Stor<T>::from_f64(fe[a], Stor<T>::dev ? P.wref[a] : 0.0);
}

template <class T>
__global__ void get_pop_d1_kernel(const T* __restrict__ f, ProbDev P, int64_t plane, double* __restrict__ out) {
  const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (x >= P.nx) return;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    out[(int64_t)a * P.nx + x] = Stor<T>::to_f64(f[a * plane + P.base + x], Stor<T>::dev ? P.wref[a] : 0.0);
}

template <class T>
__global__ void set_pop_d1_kernel(T* __restrict__ f, ProbDev P, int64_t plane, const double* __restrict__ in) {
  const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (x >= P.nx) return;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    f[a * plane + P.base + x] = Stor<T>::from_f64(in[(int64_t)a * P.nx + x], Stor<T>::dev ? P.wref[a] : 0.0);
}

// n, u, and at theta = 0 mu = n^2/8 (I_0 = (2 pi mu)^{1/2}/Gamma(3/2) = n),
// T = t = 0; NaN for the Maxwell-Boltzmann closure.  Per-block partial sums
// n, j, 0, E = sum f e^2, 0, non-finite cells, in the layout of moments_kernel.
template <class T, int STAT>
__global__ void __launch_bounds__(kMomThreads) moments_d1_kernel(const T* __restrict__ f, ProbDev P, int64_t plane,
                                                                 double* __restrict__ on, double* __restrict__ oux,
                                                                 double* __restrict__ ouy, double* __restrict__ oT,
                                                                 double* __restrict__ omu, double* __restrict__ ot,
                                                                 double* __restrict__ partials) {
  const int x = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  double acc[kNPartial] = {0, 0, 0, 0, 0, 0};
  if (x < P.nx) {
    double v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = Stor<T>::to_f64(f[a * plane + P.base + x], Stor<T>::dev ? P.wref[a] : 0.0);
    const double n = (v[0] + v[1]) + v[2];
    const double j = v[1] - v[2];
    const double E = v[1] + v[2];
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    if (on) on[x] = n;
    if (oux) oux[x] = j / n;
    if (ouy) ouy[x] = 0.0;
    if (oT) oT[x] = STAT == STAT_T0 ? 0.0 : nan;
    if (omu) omu[x] = STAT == STAT_T0 ? n * n / 8.0 : nan;
    if (ot) ot[x] = STAT == STAT_T0 ? 0.0 : nan;
    acc[0] = n;
    acc[1] = j;
    acc[3] = E;
    acc[5] = (isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2])) ? 0.0 : 1.0;
  }
  __shared__ double sh[kMomThreads / 32][kNPartial];
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
    for (int w = 0; w < kMomThreads / 32; ++w) s += sh[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * kNPartial + threadIdx.x] = s;
  }
}

}  // namespace lbm
