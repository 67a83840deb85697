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
  const float s56 = g[5] + g[6], s78 = g[7] + g[8], sd = s56 + s78;  // diagonal sums, shared
  m.dn = (g[0] + ((g[1] + g[2]) + (g[3] + g[4]))) + sd;
  const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
  const float jy = (g[2] - g[4]) + (s56 - s78);
  const float G1 = g[0] - sd;
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
//
// The moving populations come in opposite pairs (e_a' = -e_a), and
// S(+-eu) = (Q + a_2 eu^2) +- eu (a_1 + b_0 C + b_0 k_4 eu^2): one even and one
// odd part per pair.
template <class T, int STAT>
__device__ __forceinline__ void relax_store_dev(const ProbDev& P, const float g[9], const CellMom& m, float J2,
                                                float J4, T* __restrict__ fout, int64_t plane, int off) {
  const float dn = m.dn, X = m.X, ux = m.ux, uy = m.uy, u2 = m.u2;
  // weight changes against the reference (exact algebra, see header comment)
  float dW0, dWs, dWl;
  if (STAT == STAT_FD || STAT == STAT_FT) {  // X of the closure's J_2 (see header)
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
  const float D22 = delta22_f(J2);  // NaN outside 0 < J_2 < 2
  const float D42 = __fdividef(1.0f, 3.0f - 2.0f * J4);
  const float iJ2 = __fdividef(1.0f, J2);
  // The bracket's constants, with t = J_4 Delta_4^2 and P = (1 - J_2) t:
  //   C_short = P - (3/4 t + 9/4 J_4) u^2,  C_long = -2 P + (3/2 t - 9/2 J_4) u^2,
  //   A = a_1 + b_0 C (a_1 = 3/J_2, b_0 = 3/(2 J_2)),  b_0 k_4 = 9 J_4/(2 J_2),
  //   Q_rest = -3/2 Delta_2^2 u^2,  Q_short = (9/4 r - 3/2 Delta_2^2) u^2,
  //   Q_long = (9/2 r - 3/2 Delta_2^2) u^2,  r = (Delta_2^2 - 1)/J_2.
  const float t = J4 * D42, Pt = (1.0f - J2) * t;
  const float A1 = iJ2 * fmaf(-fmaf(1.125f, t, 3.375f * J4), u2, fmaf(1.5f, Pt, 3.0f));
  const float A2 = iJ2 * fmaf(fmaf(2.25f, t, -6.75f * J4), u2, fmaf(-3.0f, Pt, 3.0f));
  const float bk = 4.5f * J4 * iJ2, a2 = 4.5f * iJ2;
  const float h = 1.5f * D22, r = (D22 - 1.0f) * iJ2;
  const float Q0 = -h * u2, Q1 = fmaf(2.25f, r, -h) * u2, Q2 = fmaf(4.5f, r, -h) * u2;
  const float w = P.f.omega;
  // even and odd parts per opposite pair: g_eq(+-eu) = base +- wo
  float ge[9];
  ge[0] = fmaf(W0, Q0, dW0);
  auto pair = [&](float eu, float A, float Qc, float W, float dW, int ap, int am) {
    const float e2 = eu * eu;
    const float base = fmaf(W, fmaf(a2, e2, Qc), dW);
    const float wo = W * (eu * fmaf(bk, e2, A));
    ge[ap] = base + wo;
    ge[am] = base - wo;
  };
  pair(ux, A1, Q1, Ws, dWs, 1, 3);
  pair(uy, A1, Q1, Ws, dWs, 2, 4);
  pair(ux + uy, A2, Q2, Wl, dWl, 5, 7);
  pair(ux - uy, A2, Q2, Wl, dWl, 8, 6);
#pragma unroll
  for (int a = 0; a < 9; ++a) fout[a * plane + off] = Dev<T>::st(fmaf(w, ge[a] - g[a], g[a]));
}

// Collision of one cell from its pulled deviations g[9]; stores at `off`.
template <class T, int STAT>
__device__ __forceinline__ void collide_store_dev(const ProbDev& P, const float g[9], T* __restrict__ fout,
                                                  int64_t plane, int off, const InvLimitsF& L) {
  CellMom m = dev_moments(P, g);
  float J2, J4;
  if (STAT == STAT_FD) {
    J2 = 1.5f - m.delta;
    float xx;
    J4 = j4_from_delta_f(m.delta, L, &xx);
  } else if (STAT == STAT_FT) {
    // fixed theta: the cell's t = 2 pi theta/n; delta = 3/2 - J_2(t) without
    // subtraction, and X = (2/3)(n delta - n_ref delta_ref) for the weights
    float delta;
    closure_dev_from_t(P.f.two_pi_theta * m.in, delta, J4);
    m.delta = delta;
    m.X = (m.n * delta - P.f.ndelta_ref) * (2.0f / 3.0f);
    J2 = 1.5f - delta;
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
// FP32: the next row's nine loads are issued before the current row's
// collision, so that each thread keeps two rows of loads in flight.  BF16
// moves half the bytes per cell and is bound by instruction issue instead:
// it loads one row at a time, and the registers that frees go to resident
// warps.  Nine CTAs per SM for both (measured on the 4096^2 lattice: FP32
// 84.1 GLUPS at nine against 82.2 at eight; BF16 94.6 at nine without the
// prefetch against 86.6 at eight with it, 93.8 at ten and 90.8 at twelve).
constexpr int kDevCtasPerSm = 9;
template <class T, int STAT, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX, kDevCtasPerSm) stream_collide_dev(const T* __restrict__ fin, T* __restrict__ fout,
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
      if constexpr (sizeof(T) == 2) {
#pragma unroll 1
        for (int y = y0; y < y1; ++y) {
          float g[9];
          const int off = gather_dev(fin, plane, P, x, y, xin, g);
          collide_store_dev<T, STAT>(P, g, fout, plane, off, L);
        }
      } else {
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
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
}

// ------------------------------------------------------------------ moments of deviation storage

// Knuth's TwoSum: s + e = a + b exactly in round-to-nearest FP32 (no
// multiplication, so no contraction can change it).
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// A sum of FP32 terms as an unevaluated pair hi + lo: every addition's
// rounding error goes into lo, so hi + lo carries the sum to about 2^-47.
struct DFsum {
  float hi, lo;
};
__device__ __forceinline__ DFsum df_add(DFsum a, float b) {
  float s, e;
  two_sum_f(a.hi, b, s, e);
  return DFsum{s, a.lo + e};
}
__device__ __forceinline__ double df_value(DFsum a) { return (double)a.hi + (double)a.lo; }

// lbm_moments for FP32/BF16 deviation storage: the fields and diagnostics of
// moments_kernel, with x, t, theta, mu from the step's FP32 inversion and
// the FP64 work cut to what
// the results need (FP64 runs at 1/64 of the FP32 rate on this GPU): the
// deviation sums n - n_ref = sum g, j = sum g e and E - E_ref = sum g |e|^2
// as error-free FP32 sums (hi + lo, two_sum_f), converted once; 1/n as an
// FP32 reciprocal refined by two FP64 Newton steps in place of FP64
// divisions.  Both reach the FP64 sums of the stored values to a few units
// of 1e-16 relative.  n_ref = sum W_ref and E_ref = sum W_ref |e|^2 are the
// reference weights' sums (ProbDev::nsum_ref, esum_ref).  The clamp count and
// x, t, theta, mu come from the step's FP32 deviation moments and inversion.
// O: the output arrays' type (double, or float for lbm_moments_f32: the same
// values rounded once); the partial sums stay FP64.  Each thread takes
// kMomDevCells cells and each block writes one partial per sum (grid:
// cells / (kMomThreads kMomDevCells) blocks).
template <class T, int STAT, class O = double>
__global__ void __launch_bounds__(kMomThreads) moments_dev_kernel(const T* __restrict__ f, ProbDev P, int64_t plane,
                                                                  InvLimits L, InvLimitsF Lf, O* __restrict__ on,
                                                                  O* __restrict__ oux, O* __restrict__ ouy,
                                                                  O* __restrict__ oT, O* __restrict__ omu,
                                                                  O* __restrict__ ot,
                                                                  double* __restrict__ partials) {
  const int64_t cells = (int64_t)P.nx * P.ny;
  double acc[kNPartial] = {0, 0, 0, 0, 0, 0};
  // kMomDevCells cells per thread, strided by the block size (coalesced), so
  // that the FP64 block reduction below is shared by several cells
#pragma unroll 1
  for (int kk = 0; kk < kMomDevCells; ++kk) {
  const int64_t i = ((int64_t)blockIdx.x * kMomDevCells + kk) * blockDim.x + threadIdx.x;
  const int64_t c = i < cells ? P.base + (int64_t)(i / P.nx) * P.pitch + (int)(i % P.nx) : 0;
  if (i < cells && P.solid != nullptr && P.solid[c] != 0) {  // obstacle: no fluid
    if (on) on[i] = (O)0;
    if (oux) oux[i] = (O)0;
    if (ouy) ouy[i] = (O)0;
    if (oT) oT[i] = (O)0;
    if (omu) omu[i] = (O)0;
    if (ot) ot[i] = (O)0;
  } else if (i < cells) {
    float g[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) g[a] = Dev<T>::ld(f[a * plane + c]);
    DFsum sn{g[0], 0.0f}, sx{g[1], 0.0f}, sy{g[2], 0.0f}, se{g[1], 0.0f};
#pragma unroll
    for (int a = 1; a < 9; ++a) sn = df_add(sn, g[a]);
    sx = df_add(sx, -g[3]);
    sx = df_add(sx, g[5]);
    sx = df_add(sx, -g[6]);
    sx = df_add(sx, -g[7]);
    sx = df_add(sx, g[8]);
    sy = df_add(sy, -g[4]);
    sy = df_add(sy, g[5]);
    sy = df_add(sy, g[6]);
    sy = df_add(sy, -g[7]);
    sy = df_add(sy, -g[8]);
    se = df_add(se, g[2]);
    se = df_add(se, g[3]);
    se = df_add(se, g[4]);
#pragma unroll
    for (int a = 5; a < 9; ++a) se = df_add(se, 2.0f * g[a]);
    const double n = P.nsum_ref + df_value(sn);
    const double jx = df_value(sx), jy = df_value(sy);
    const double E = P.esum_ref + df_value(se);
    double r = (double)__frcp_rn((float)n);  // 1/n: FP32 seed, two Newton steps
    r = fma(r, fma(-n, r, 1.0), r);
    r = fma(r, fma(-n, r, 1.0), r);
    // the closure quantities in FP32 from the step's own deviation moments
    // (delta = 3/2 - J_2 without cancellation), as the step decides them
    const CellMom m = dev_moments(P, g);
    float theta_f = 0.0f, mu_f = 0.0f, t_f = 0.0f;
    double theta = 0.0, mu = 0.0, t = 0.0;
    int cl = 0;
    if (STAT == STAT_FD) {
      const float J2 = 1.5f - m.delta;
      cl = (J2 == J2 && (J2 >= Lf.j2_hi || J2 <= Lf.j2_lo)) ? 1 : 0;
      float xf;
      j4_from_delta_f(m.delta, Lf, &xf);
      t_f = 1.0f / (fmaxf(xf, 0.0f) + log1pf(expf(-fabsf(xf))));  // t = T/T_F = 1/f_1(x)
      theta_f = m.n * t_f * (float)(1.0 / (2.0 * kPi));            // theta = n t/(2 pi)
      mu_f = theta_f * xf;
      t = t_f; theta = theta_f; mu = mu_f;
    } else if (STAT == STAT_FT) {
      // fixed theta: t = 2 pi theta/n, x = a + ln(1 - e^{-a}) with a = 1/t
      theta = P.theta;
      t = 2.0 * kPi * theta * r;
      const double a = n / (2.0 * kPi * theta);
      mu = theta * (a + log(-expm1(-a)));
    } else if (STAT == STAT_T0) {
      theta = 0.0; t = 0.0; mu = n * (1.0 / (2.0 * kPi));
    } else {
      theta = mu = t = __longlong_as_double(0x7ff8000000000000LL);
    }
    if (on) on[i] = (O)n;
    if (oux) oux[i] = (O)((jx + 0.5 * P.fx) * r);  // velocity at the time level under a body force
    if (ouy) ouy[i] = (O)((jy + 0.5 * P.fy) * r);
    if (oT) oT[i] = (O)theta;
    if (omu) omu[i] = (O)mu;
    if (ot) ot[i] = (O)t;
    acc[0] += n; acc[1] += jx; acc[2] += jy; acc[3] += E;
    acc[4] += cl;
    bool fin = true;
#pragma unroll
    for (int a = 0; a < 9; ++a) fin = fin && isfinite(g[a]);
    acc[5] += (fin && isfinite(n)) ? 0.0 : 1.0;
  }
  }
  // fixed-order block reduction, as moments_kernel
  __shared__ double sh[kMomThreads / 32][kNPartial];
#pragma unroll
  for (int k = 0; k < kNPartial; ++k) {
    double v = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    acc[k] = v;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNPartial; ++k) sh[wid][k] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x < kNPartial) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kMomThreads / 32; ++w) v += sh[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * kNPartial + threadIdx.x] = v;
  }
}

}  // namespace lbm
