// Reduced-precision step: populations stored as deviations g_a = f_a - W_a^ref
// from a per-problem constant W^ref = w_a(J_2,ref) n_ref (the d2v9 weights of
// Sect. "The Gaussian quadrature"), in FP32 or BF16; every sum and the
// equilibrium in FP32.
//
// With dn = sum g, G1 = sum g (1 - |e|^2) = g_0 - (g_5 + g_6 + g_7 + g_8) and
// j = sum g e (sum W^ref e = 0), the moments follow without cancellation:
//   n = n_ref + dn,  u_0 = j/n,
//   n (3/2 - J_2) = n_ref (3/2 - J_2,ref) + (3/2)(G1 + n |u_0|^2),
// because sum W^ref (1 - |e|^2) = (2/3) n_ref (3/2 - J_2,ref) and
// J_2 = 3 (E/n - |u_0|^2)/2.  The weight change is then
//   W_0 - W_0^ref = dn/6 + (5/6)(G1 + n u^2),
//   W_s - W_s^ref = 4 (W_l - W_l^ref) = (dn - G1 - n u^2)/6,
// and g_eq,a = (W_a - W_a^ref) + W_a (S_a - 1) with S_a the bracket of the
// K = 3 equilibrium, so the stored quantity never passes through f itself.
#pragma once
#include <cuda_bf16.h>

#include "fd_device_f32.cuh"
#include "launch.h"
#include "lbm_kernels.cuh"
#include "surrogate.cuh"
#include "tc_sm100.cuh"

namespace lbm {

template <class T>
struct Dev;
template <>
struct Dev<float> {
  __device__ static __forceinline__ float ld(float v) { return v; }
  __device__ static __forceinline__ float st(float v) { return v; }
};
template <>
struct Dev<__nv_bfloat16> {
  __device__ static __forceinline__ float ld(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ static __forceinline__ __nv_bfloat16 st(float v) { return __float2bfloat16_rn(v); }
};

// Polish of the learned inversion's x_0 = mu/T: one Newton step on
// J_2(x) = J_2 to x_1; the residual check evaluates f_0..f_4 at x_1 and
// accepts when the remaining Newton correction dx is below 5e-4 x_1 (the
// acceptance of the exact iteration), returning J_4(x_1) + J_4'(x_1) dx.
// Otherwise *fallback is set and the exact inversion runs.
__device__ __forceinline__ float j4_polish_f(float x0, float delta, const InvLimitsF& L, int* fallback) {
  const float J2 = 1.5f - delta;
  float x = fminf(fmaxf(x0, L.x_lo), L.x_hi);
#pragma unroll 1
  for (int it = 0; it < 2; ++it) {
    const FD5f f = x >= 4.0f ? fd_eval_deg_f(x) : fd_eval_f(x);
    const float i1 = rcp_a(f.f1), i2 = rcp_a(f.f2), i3 = rcp_a(f.f3), i4 = rcp_a(f.f4);
    const float j = f.f2 * f.f2 * i1 * i3;
    const float dj = j * (2.0f * f.f1 * i2 - f.f0 * i1 - f.f2 * i3);
    const float dx = (J2 - j) * rcp_a(dj);
    if (it == 1) {
      if (fabsf(dx) < 5e-4f * x) {
        const float J4 = f.f3 * f.f3 * i2 * i4;
        const float dJ4 = J4 * (2.0f * f.f2 * i3 - f.f1 * i2 - f.f3 * i4);
        return J4 + dJ4 * dx;
      }
      break;
    }
    x = fminf(fmaxf(x + dx, L.x_lo), L.x_hi);
  }
  *fallback = 1;
  float xx;
  return j4_from_delta_f(delta, L, &xx);
}

// Cells the network handles: finite J_2 inside the clamp interval.
__device__ __forceinline__ bool net_cell(float delta, const InvLimitsF& L) {
  const float J2 = 1.5f - delta;
  return J2 == J2 && J2 < L.j2_hi && J2 > L.j2_lo;
}

// J_4 through the learned inversion, network on the FP32 pipe (the network
// gives (T, mu) from (n, e), e = 2 n J_2/3 entering as delta = 3/2 - J_2).
__device__ __forceinline__ float j4_surrogate_f(float n, float delta, const InvLimitsF& L, const MlpParams& W,
                                                int* fallback) {
  if (!net_cell(delta, L)) {  // non-finite or clamped: the exact path handles it
    float xx;
    return j4_from_delta_f(delta, L, &xx);
  }
  float y0, y1, T, mu;
  mlp_forward_f(W, n, delta, y0, y1);
  mlp_outputs_to_state(y0, y1, T, mu);
  return j4_polish_f(mu * rcp_a(T), delta, L, fallback);
}

// 32-bit in-plane pull offsets (every plane holds fewer than 2^31 cells);
// -1 marks an off-lattice source.
struct PullIdx32 {
  int row, rm, rp, xm, xp;
};

__device__ __forceinline__ PullIdx32 pull_index32(const ProbDev& P, int x, int y) {
  PullIdx32 q;
  const int base = (int)P.base;
  q.row = base + y * P.pitch;
  const int ym = y > 0 ? y - 1 : (P.bc_y == BC_PERIODIC ? P.ny - 1 : -1);
  const int yp = y < P.ny - 1 ? y + 1 : (P.bc_y == BC_PERIODIC ? 0 : -1);
  q.rm = ym >= 0 ? base + ym * P.pitch : -1;
  q.rp = yp >= 0 ? base + yp * P.pitch : -1;
  q.xm = x > 0 ? x - 1 : (P.bc_x == BC_PERIODIC ? P.nx - 1 : -1);
  q.xp = x < P.nx - 1 ? x + 1 : (P.bc_x == BC_PERIODIC ? 0 : -1);
  return q;
}

template <class T>
__device__ __forceinline__ void pull9_32(const T* __restrict__ fin, int64_t plane, const PullIdx32& q, int x, T v[9]) {
  auto ld = [&](int a, int r, int xs, int opp) -> T {
    return (r < 0 || xs < 0) ? fin[opp * plane + (q.row + x)] : fin[a * plane + (r + xs)];
  };
  v[0] = fin[q.row + x];
  v[1] = ld(1, q.row, q.xm, 3);
  v[2] = ld(2, q.rm, x, 4);
  v[3] = ld(3, q.row, q.xp, 1);
  v[4] = ld(4, q.rp, x, 2);
  v[5] = ld(5, q.rm, q.xm, 7);
  v[6] = ld(6, q.rm, q.xp, 8);
  v[7] = ld(7, q.rp, q.xp, 5);
  v[8] = ld(8, q.rp, q.xm, 6);
}

// Moments of one cell from its pulled deviations (FP32, deviation form).
struct CellMom {
  float dn, n, in, ux, uy, u2, X, delta;
};

__device__ __forceinline__ CellMom dev_moments(const ProbDev& P, const float g[9]) {
  CellMom m;
  const float nref = P.f.n_ref, ndref = P.f.ndelta_ref;
  m.dn = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
  const float jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
  const float G1 = g[0] - ((g[5] + g[6]) + (g[7] + g[8]));
  m.n = nref + m.dn;
  m.in = __fdividef(1.0f, m.n);
  m.ux = jx * m.in;
  m.uy = jy * m.in;
  m.u2 = m.ux * m.ux + m.uy * m.uy;
  m.X = G1 + m.n * m.u2;
  m.delta = (ndref + 1.5f * m.X) * m.in;  // 3/2 - J_2 (FD closure)
  return m;
}

// Equilibrium and BGK of one cell given J_2, J_4; stores at `off`.
template <class T, int STAT>
__device__ __forceinline__ void relax_store_dev(const ProbDev& P, const float g[9], const CellMom& m, float J2,
                                                float J4, T* __restrict__ fout, int64_t plane, int off) {
  const float dn = m.dn, X = m.X, ux = m.ux, uy = m.uy, u2 = m.u2;
  // weight changes against the reference (exact algebra, see header comment)
  float dW0, dWs, dWl;
  if (STAT == STAT_FD) {
    dW0 = dn * (1.0f / 6.0f) + (5.0f / 6.0f) * X;
    dWs = (dn - X) * (1.0f / 6.0f);
    dWl = 0.25f * dWs;
  } else {
    // fixed J_2: W scales with n only
    dW0 = dn * (1.0f - 5.0f * J2 / 9.0f);
    dWs = dn * J2 / 9.0f;
    dWl = dn * J2 / 36.0f;
  }
  const float W0 = P.f.wref[0] + dW0, Ws = P.f.wref[1] + dWs, Wl = P.f.wref[2] + dWl;
  const float D22 = __fdividef(1.0f, 2.0f - J2);
  const float D42 = __fdividef(1.0f, 3.0f - 2.0f * J4);
  const float iJ2 = __fdividef(1.0f, J2);
  const float a1 = 3.0f * iJ2, a2 = 4.5f * iJ2, b0 = 1.5f * iJ2;
  const float a3 = 2.25f * (D22 - 1.0f) * iJ2;
  const float a4 = 1.5f * D22;
  const float omJ = 1.0f - J2;
  const float k0 = 4.0f * omJ * J4 * D42, k1 = 3.0f * omJ * J4 * D42, k2 = 3.0f * J4 * D42;
  const float k3 = 2.25f * J4 * (D42 - 1.0f), k4 = 3.0f * J4;
  const float C1 = k0 - k1 + (k3 - k2) * u2, C2 = k0 - 2.0f * k1 + (2.0f * k3 - k2) * u2;
  const float Q0 = -a4 * u2, Q1 = (a3 - a4) * u2, Q2 = (2.0f * a3 - a4) * u2;
  auto Sm1 = [&](float eu, float C, float Qc) { return Qc + eu * (a1 + a2 * eu + b0 * (C + k4 * eu * eu)); };
  float ge[9];
  ge[0] = dW0 + W0 * Q0;
  ge[1] = dWs + Ws * Sm1(ux, C1, Q1);
  ge[2] = dWs + Ws * Sm1(uy, C1, Q1);
  ge[3] = dWs + Ws * Sm1(-ux, C1, Q1);
  ge[4] = dWs + Ws * Sm1(-uy, C1, Q1);
  ge[5] = dWl + Wl * Sm1(ux + uy, C2, Q2);
  ge[6] = dWl + Wl * Sm1(-ux + uy, C2, Q2);
  ge[7] = dWl + Wl * Sm1(-ux - uy, C2, Q2);
  ge[8] = dWl + Wl * Sm1(ux - uy, C2, Q2);
  const float w = P.f.omega;
#pragma unroll
  for (int a = 0; a < 9; ++a) fout[a * plane + off] = Dev<T>::st(fmaf(w, ge[a] - g[a], g[a]));
}

// Collision of one cell from its pulled deviations g[9]; stores at `off`.
template <class T, int STAT, bool SURR = false>
__device__ __forceinline__ void collide_store_dev(const ProbDev& P, const float g[9], T* __restrict__ fout,
                                                  int64_t plane, int off, const InvLimitsF& L,
                                                  const MlpParams* W = nullptr, int* fallback = nullptr) {
  const CellMom m = dev_moments(P, g);
  float J2, J4;
  if (STAT == STAT_FD) {
    J2 = 1.5f - m.delta;
    if (SURR) {
      J4 = j4_surrogate_f(m.n, m.delta, L, *W, fallback);
    } else {
      float xx;
      J4 = j4_from_delta_f(m.delta, L, &xx);
    }
  } else {
    J2 = (float)FixedJ<STAT>::j2;
    J4 = (float)FixedJ<STAT>::j4;
  }
  relax_store_dev<T, STAT>(P, g, m, J2, J4, fout, plane, off);
}

// Pulled deviations of cell (x, y): branch-free gather for interior tiles,
// general (wall / wrap aware) gather otherwise.  Returns the cell's offset.
template <class T>
__device__ __forceinline__ int gather_dev(const T* __restrict__ fin, int64_t plane, const ProbDev& P, int x, int y,
                                          bool xin, float g[9]) {
  if (xin && y >= 1 && y <= P.ny - 2) {
    const int off = (int)P.base + y * P.pitch + x;
    const int pt = P.pitch;
    g[0] = Dev<T>::ld(fin[off]);
    g[1] = Dev<T>::ld(fin[plane + (off - 1)]);
    g[2] = Dev<T>::ld(fin[2 * plane + (off - pt)]);
    g[3] = Dev<T>::ld(fin[3 * plane + (off + 1)]);
    g[4] = Dev<T>::ld(fin[4 * plane + (off + pt)]);
    g[5] = Dev<T>::ld(fin[5 * plane + (off - pt - 1)]);
    g[6] = Dev<T>::ld(fin[6 * plane + (off - pt + 1)]);
    g[7] = Dev<T>::ld(fin[7 * plane + (off + pt + 1)]);
    g[8] = Dev<T>::ld(fin[8 * plane + (off + pt - 1)]);
    return off;
  }
  const PullIdx32 q = pull_index32(P, x, y);
  T raw[9];
  pull9_32(fin, plane, q, x, raw);
#pragma unroll
  for (int a = 0; a < 9; ++a) g[a] = Dev<T>::ld(raw[a]);
  return q.row + x;
}

// One tile: kTileX consecutive cells of TY consecutive rows of one problem.
// PERSIST = false: one tile per CTA (grid = number of tiles).  PERSIST = true:
// a smaller grid whose CTAs walk tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// Tiles whose cells and neighbours are all inside the lattice (no wall, no
// wrap) take the branch-free interior gather; edge tiles take the general one.
// The next row's nine loads are issued before the current row's collision so
// that each thread keeps two rows of loads in flight.
template <class T, int STAT, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX, 10) stream_collide_dev(const T* __restrict__ fin, T* __restrict__ fout,
                                                                 const ProbDev* __restrict__ probs, int nprob,
                                                                 int ntiles, int64_t plane, InvLimitsF L) {
  int tile = (int)blockIdx.x;
#pragma unroll 1
  do {
    const int p = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
    const ProbDev& P = probs[p];
    const int lt = tile - (int)P.tile_begin;
    const int ty = lt / P.tiles_x;
    const int x0 = (lt - ty * P.tiles_x) * kTileX;
    const int x = x0 + (int)threadIdx.x;
    if (x < P.nx) {
      const int y0 = ty * TY;
      const int y1 = min(y0 + TY, P.ny);
      const bool xin = x0 >= 1 && x0 + kTileX <= P.nx - 1;
      float gn[9];
      int offn = gather_dev(fin, plane, P, x, y0, xin, gn);
#pragma unroll 1
      for (int y = y0; y < y1; ++y) {
        float g[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) g[a] = gn[a];
        const int off = offn;
        if (y + 1 < y1) offn = gather_dev(fin, plane, P, x, y + 1, xin, gn);
        collide_store_dev<T, STAT>(P, g, fout, plane, off, L);
      }
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
}

// The FD step with the learned inversion (see j4_surrogate_f).  counters[0]
// accumulates cells that fell back to the exact inversion, counters[1] cells
// that went through the network (one atomic per warp and row).
template <class T, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX) stream_collide_surr(const T* __restrict__ fin, T* __restrict__ fout,
                                                              const ProbDev* __restrict__ probs, int nprob, int ntiles,
                                                              int64_t plane, InvLimitsF L,
                                                              unsigned long long* __restrict__ counters,
                                                              const MlpParams W) {
  int tile = (int)blockIdx.x;
#pragma unroll 1
  do {
    const int p = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
    const ProbDev& P = probs[p];
    const int lt = tile - (int)P.tile_begin;
    const int ty = lt / P.tiles_x;
    const int x0 = (lt - ty * P.tiles_x) * kTileX;
    const int x = x0 + (int)threadIdx.x;
    const int y0 = ty * TY;
    const int y1 = min(y0 + TY, P.ny);
    const bool xin = x0 >= 1 && x0 + kTileX <= P.nx - 1;
#pragma unroll 1
    for (int y = y0; y < y1; ++y) {
      int fb = 0;
      const bool active = x < P.nx;
      if (active) {
        float g[9];
        const int off = gather_dev(fin, plane, P, x, y, xin, g);
        collide_store_dev<T, STAT_FD, true>(P, g, fout, plane, off, L, &W, &fb);
      }
      const unsigned nfb = __ballot_sync(0xffffffffu, fb != 0);
      const unsigned nact = __ballot_sync(0xffffffffu, active);
      if ((threadIdx.x & 31) == 0 && nact) {
        atomicAdd(&counters[0], (unsigned long long)__popc(nfb));
        atomicAdd(&counters[1], (unsigned long long)__popc(nact));
      }
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
}

// The FD step with the learned inversion, its 64 x 64 hidden layer on the
// tensor cores.  A tile row of 128 cells is one M = 128 MMA operand: every
// thread computes its cell's first layer (64 SiLU units) and writes it as
// FP16 into shared memory in the canonical K-major layout; one thread issues
// four tcgen05.mma (K = 16 each) against W2 (FP16, staged once per CTA from
// w2h, already in the canonical layout; SiLU by packed FP16 tanh) into an FP32 accumulator of 64 TMEM
// columns and commits to an mbarrier; each warp then reads its 32 lanes back
// (tcgen05.ld 32x32b.x64: one row, i.e. one cell, per thread), and the
// second SiLU, the output layer, the Newton polish and the relaxation run per
// thread.  A wait that exceeds its bound marks the CTA failed: it counts the
// event in counters[2], serves the remaining cells with the exact inversion
// and still frees its TMEM.
template <class T, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX) stream_collide_surr_tc(const T* __restrict__ fin, T* __restrict__ fout,
                                                                 const ProbDev* __restrict__ probs, int nprob,
                                                                 int ntiles, int64_t plane, InvLimitsF L,
                                                                 unsigned long long* __restrict__ counters,
                                                                 const __half* __restrict__ w2h, const MlpParams W) {
  __shared__ __align__(1024) __half sA[kTileX * kH];
  __shared__ __align__(1024) __half sB[kH * kH];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = (int)threadIdx.x, warp = tid >> 5;
  {
    const uint4* src = reinterpret_cast<const uint4*>(w2h);
    uint4* dst = reinterpret_cast<uint4*>(sB);
    for (int i = tid; i < kH * kH / 8; i += kTileX) dst[i] = src[i];
  }
  if (tid == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&tmem_slot, kH);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t idesc = tc::idesc_f16_f32(kTileX, kH);
  uint32_t phase = 0;
  bool failed = false;
  int tile = (int)blockIdx.x;
#pragma unroll 1
  do {
    const int p = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
    const ProbDev& P = probs[p];
    const int lt = tile - (int)P.tile_begin;
    const int ty = lt / P.tiles_x;
    const int x0 = (lt - ty * P.tiles_x) * kTileX;
    const int x = x0 + tid;
    const int y0 = ty * TY;
    const int y1 = min(y0 + TY, P.ny);
    const bool xin = x0 >= 1 && x0 + kTileX <= P.nx - 1;
    const bool active = x < P.nx;
#pragma unroll 1
    for (int y = y0; y < y1; ++y) {
      float g[9];
      int off = 0;
      CellMom m;
      if (active) {
        off = gather_dev(fin, plane, P, x, y, xin, g);
        m = dev_moments(P, g);
      } else {
        m.n = 1.0f;
        m.delta = 0.1f;
      }
      const bool use_net = active && !failed && net_cell(m.delta, L);
      // first layer, written as the M = 128 operand (row tid)
      {
        const float i0 = (m.n - kSurNMid) * (1.0f / kSurNHalf);
        const float i1 = (__logf(m.delta) - kSurLdMid) * (1.0f / kSurLdHalf);
#pragma unroll
        for (int kc = 0; kc < kH / 8; ++kc) {
          __align__(16) __half2 h[4];
#pragma unroll
          for (int kk = 0; kk < 8; kk += 2) {
            const int k = 8 * kc + kk;
            const float z0 = fmaf(W.p[kOW1 + 2 * k], i0, fmaf(W.p[kOW1 + 2 * k + 1], i1, W.p[kOB1 + k]));
            const float z1 = fmaf(W.p[kOW1 + 2 * k + 2], i0, fmaf(W.p[kOW1 + 2 * k + 3], i1, W.p[kOB1 + k + 1]));
            h[kk / 2] = use_net ? tc::silu2_h(z0, z1) : __floats2half2_rn(0.0f, 0.0f);
          }
          *reinterpret_cast<uint4*>(reinterpret_cast<char*>(sA) + tc::kmajor_off(tid, 8 * kc, kTileX)) =
              *reinterpret_cast<const uint4*>(h);
        }
      }
      bool ok = false;
      if (!failed) {
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
          const uint32_t a0 = tc::smem_u32(sA), b0 = tc::smem_u32(sB);
#pragma unroll
          for (int sidx = 0; sidx < kH / 16; ++sidx) {
            const uint64_t ad = tc::smem_desc(a0 + (uint32_t)(2 * sidx) * (kTileX / 8) * 128, (kTileX / 8) * 128, 128);
            const uint64_t bd = tc::smem_desc(b0 + (uint32_t)(2 * sidx) * (kH / 8) * 128, (kH / 8) * 128, 128);
            tc::mma_f16(tmem, ad, bd, idesc, sidx > 0 ? 1u : 0u);
          }
          tc::commit(&mbar);
        }
        const bool done = tc::mbar_wait(&mbar, phase, 1 << 22);
        phase ^= 1u;
        failed = __syncthreads_or(!done) != 0;
        if (failed && tid == 0) atomicAdd(&counters[2], 1ull);
        ok = !failed;
      }
      float J4 = 0.0f;
      int fb = 0;
      if (ok) {
        tc::fence_after();
        float z2[kH];
        tc::tmem_ld64(tmem + ((uint32_t)(warp * 32) << 16), z2);
        if (use_net) {
          float a0 = W.p[kOB3], a1 = W.p[kOB3 + 1];
#pragma unroll
          for (int j = 0; j < kH; j += 2) {
            const float2 h = __half22float2(tc::silu2_h(z2[j] + W.p[kOB2 + j], z2[j + 1] + W.p[kOB2 + j + 1]));
            a0 = fmaf(W.p[kOW3 + j], h.x, fmaf(W.p[kOW3 + j + 1], h.y, a0));
            a1 = fmaf(W.p[kOW3 + kH + j], h.x, fmaf(W.p[kOW3 + kH + j + 1], h.y, a1));
          }
          float temp, mu;
          mlp_outputs_to_state(a0, a1, temp, mu);
          J4 = j4_polish_f(mu * rcp_a(temp), m.delta, L, &fb);
        }
      }
      if (active) {
        if (!use_net || !ok) {
          float xx;
          J4 = j4_from_delta_f(m.delta, L, &xx);
          if (use_net) fb = 1;
        }
        relax_store_dev<T, STAT_FD>(P, g, m, 1.5f - m.delta, J4, fout, plane, off);
      }
      const unsigned nfb = __ballot_sync(0xffffffffu, fb != 0);
      const unsigned nact = __ballot_sync(0xffffffffu, active);
      if ((tid & 31) == 0 && nact) {
        atomicAdd(&counters[0], (unsigned long long)__popc(nfb));
        atomicAdd(&counters[1], (unsigned long long)__popc(nact));
      }
      tc::fence_before();  // this row's TMEM reads before the next row's MMA
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, kH);
}

}  // namespace lbm
