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

#include "launch.h"
#include "lbm_kernels.cuh"
#include "surrogate.cuh"

namespace lbm {

constexpr float kPi2f = 9.8696044010893586f;
constexpr float kXDegF = 17.0f;  // e^-17 = 4e-8: S_n tails below FP32 resolution

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

struct FD5f {
  float f0, f1, f2, f3, f4;
};

// 1/k for the series terms (k = 1..12), read warp-uniformly.
__constant__ float c_inv_k[13] = {0.f,     1.f,         0.5f,   1.f / 3.f, 0.25f,      0.2f,       1.f / 6.f,
                                  1.f / 7.f, 0.125f, 1.f / 9.f, 0.1f,  1.f / 11.f, 1.f / 12.f};

// FP32 f_0..f_4 (same expansions as the FP64 functions; FP32 term counts).
// For a = |x| >= 2 the series S_n(e^{-a}) needs ceil(17/a) terms: its tail is
// then below e^{-17} = 4e-8, under FP32 resolution of f_n >= 1.
__device__ __forceinline__ FD5f fd_eval_f(float x) {
  FD5f r;
  const float a = fabsf(x);
  const float em = __expf(-a);
  const float r1 = __fdividef(1.0f, 1.0f + em);
  r.f0 = x >= 0.0f ? r1 : em * r1;
  const float s = x * x;
  const float p2 = 0.5f * s + kPi2f / 6.0f;
  const float p3 = x * (s + kPi2f) * (1.0f / 6.0f);
  const float p4 = s * s * (1.0f / 24.0f) + kPi2f * s * (1.0f / 12.0f) + 7.0f * kPi2f * kPi2f / 360.0f;
  if (x >= kXDegF) {
    r.f1 = x + __logf(1.0f + em);
    r.f2 = p2; r.f3 = p3; r.f4 = p4;
    return r;
  }
  float s2 = 0.f, s3 = 0.f, s4 = 0.f;
  const float y = em;
  if (a >= 2.0f) {
    r.f1 = fmaxf(x, 0.0f) + __logf(1.0f + em);
    const int K = min(9, (int)(kXDegF / a) + 1);
    float yk = y, sg = 1.0f;
#pragma unroll 1
    for (int k = 1; k <= K; ++k) {
      const float ik = c_inv_k[k];
      const float t2 = yk * ik * ik, t3 = t2 * ik, t4 = t3 * ik;
      s2 = fmaf(sg, t2, s2); s3 = fmaf(sg, t3, s3); s4 = fmaf(sg, t4, s4);
      yk *= y;
      sg = -sg;
    }
  } else {
    r.f1 = fmaxf(x, 0.0f) + log1pf(em);
    // Cohen, Rodriguez Villegas, Zagier Algorithm 1, N = 12 ((3+sqrt 8)^12 ~ 1.5e9)
    const int N = 12;
    const float d = 0.5f * (1.5209e9f + 1.0f / 1.5209e9f);
    float b = -1.0f, c = -d, yk = y;
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      c = b - c;
      const float ik = c_inv_k[k + 1];
      const float a2 = yk * ik * ik, a3 = a2 * ik, a4 = a3 * ik;
      s2 = fmaf(c, a2, s2); s3 = fmaf(c, a3, s3); s4 = fmaf(c, a4, s4);
      b = (float)(k + N) * (float)(k - N) * b / (((float)k + 0.5f) * (float)(k + 1));
      yk *= y;
    }
    s2 /= d; s3 /= d; s4 /= d;
  }
  if (x > 0.0f) {
    r.f2 = p2 - s2; r.f3 = p3 + s3; r.f4 = p4 - s4;
  } else {
    r.f2 = s2; r.f3 = s3; r.f4 = s4;
  }
  return r;
}

// Single-instruction approximations (MUFU) for the inversion: about 1-2 ulp,
// far inside its FP32 error budget.
__device__ __forceinline__ float rcp_a(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float sqrt_a(float v) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float expm_a(float v) {  // e^{-v}
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-1.4426950408889634f * v));
  return r;
}

// P_2, P_3, P_4 of the inversion formula at x (the degenerate parts of f_n).
__device__ __forceinline__ void fd_poly_f(float x, float& p2, float& p3, float& p4) {
  const float s = x * x;
  p2 = 0.5f * s + kPi2f / 6.0f;
  p3 = x * (s + kPi2f) * (1.0f / 6.0f);
  p4 = s * s * (1.0f / 24.0f) + kPi2f * s * (1.0f / 12.0f) + 7.0f * kPi2f * kPi2f / 360.0f;
}

// Large root s = x^2 of 6 delta s^2 - (3 pi^2 - 6 delta pi^2) s + pi^4 = 0:
// the degenerate form 3/2 - J_2 = pi^2 (3 s - pi^2)/(6 s (s + pi^2)).
__device__ __forceinline__ float deg_root_f(float delta) {
  const float A = 6.0f * delta, B = 3.0f * kPi2f - 6.0f * delta * kPi2f, C = kPi2f * kPi2f;
  return (B + sqrt_a(fmaxf(B * B - 4.0f * A * C, 0.0f))) * rcp_a(2.0f * A);
}

// J_4 in the degenerate regime from s = x^2 (S_n tails dropped):
// J_4 = P_3^2/(P_2 P_4) = 60 s (s + pi^2)^2 / ((3 s + pi^2)(15 s^2 + 30 pi^2 s + 7 pi^4)).
__device__ __forceinline__ float j4_degenerate_f(float s) {
  const float sp = s + kPi2f;
  return 60.0f * s * sp * sp *
         rcp_a((3.0f * s + kPi2f) * (15.0f * s * s + 30.0f * kPi2f * s + 7.0f * kPi2f * kPi2f));
}

// One fixed-point pass that folds the leading tails into the degenerate
// root.  With y = e^{-x} the first series terms change f_1, f_2, f_3 by
// +y, -y, +y, hence J_2 by -J_2 y (2/P_2 + 1/x + 1/P_3); the pass solves the
// degenerate quadratic for delta minus that change at the current x.  The
// remaining error is O(y^2): below FP32 resolution of J_4 for x >= 9 after one
// pass and x >= 7 after two.
__device__ __forceinline__ float tail_pass_f(float delta, float x) {
  const float y = expm_a(x);
  float p2, p3, p4;
  fd_poly_f(x, p2, p3, p4);
  const float ip2 = rcp_a(p2), ip3 = rcp_a(p3), ix = rcp_a(x);
  const float J2d = p2 * p2 * ix * ip3;
  const float c = J2d * y * (2.0f * ip2 + ix + ip3);
  return sqrt_a(deg_root_f(delta - c));
}

// J_4 with the first two series terms of f_2, f_3, f_4 (error O(y^3)).
__device__ __forceinline__ float j4_tail_f(float x) {
  const float y = expm_a(x);
  float p2, p3, p4;
  fd_poly_f(x, p2, p3, p4);
  const float f2 = p2 - y * (1.0f - 0.25f * y);
  const float f3 = p3 + y * (1.0f - 0.125f * y);
  const float f4 = p4 - y * (1.0f - 0.0625f * y);
  return f3 * f3 * rcp_a(f2 * f4);
}

// f_0..f_4 for x >= 4 (y = e^{-x} <= 0.019): three series terms in Horner
// form (the fourth is below 2e-10 of f_2) and log1p(y) to y^4.
__device__ __forceinline__ FD5f fd_eval_deg_f(float x) {
  FD5f r;
  const float y = expm_a(x);
  float p2, p3, p4;
  fd_poly_f(x, p2, p3, p4);
  const float s2 = y * (1.0f + y * (-0.25f + y * (1.0f / 9.0f)));
  const float s3 = y * (1.0f + y * (-0.125f + y * (1.0f / 27.0f)));
  const float s4 = y * (1.0f + y * (-0.0625f + y * (1.0f / 81.0f)));
  r.f0 = rcp_a(1.0f + y);
  r.f1 = x + y * (1.0f + y * (-0.5f + y * (1.0f / 3.0f - 0.25f * y)));
  r.f2 = p2 - s2;
  r.f3 = p3 + s3;
  r.f4 = p4 - s4;
  return r;
}

// J_4 from delta = 3/2 - J_2 in FP32 (the exact inversion, to FP32
// resolution; *xout receives x).
//  * non-finite input: propagated at once;
//  * J_2 beyond the clamp interval: x at the nearest end;
//  * degenerate regime (delta < 0.15, x > 4.2): the quadratic root; closed
//    form J_4 for x >= 17; one tail pass for x >= 9, two for x >= 7; below
//    that Newton steps on J_2(x) from the second pass, each with one
//    evaluation of f_0..f_4, stopping when the step is below 5e-4 x and
//    returning x + dx and J_4 + J_4' dx (second-order remainder < 1e-7).
//    J_2' = J_2 (2 f_1/f_2 - f_0/f_1 - f_2/f_3), J_4' = J_4 (2 f_2/f_3 -
//    f_1/f_2 - f_3/f_4), from d f_n/dx = f_{n-1};
//  * otherwise (J_2 < 4/3): safeguarded Newton with the general FP32
//    evaluation, at most 24 evaluations.
__device__ __forceinline__ float j4_from_delta_f(float delta, const InvLimitsF& L, float* xout) {
  const float J2 = 1.5f - delta;
  if (!(J2 == J2)) {  // non-finite state: propagate without iterating
    *xout = J2;
    return J2;
  }
  if (!(J2 < L.j2_hi)) {
    *xout = L.x_hi;
    return j4_degenerate_f(L.x_hi * L.x_hi);
  }
  if (J2 <= L.j2_lo) {
    const FD5f f = fd_eval_f(L.x_lo);
    *xout = L.x_lo;
    return f.f3 * f.f3 * rcp_a(f.f2 * f.f4);
  }
  if (delta < 0.15f) {
    const float s = deg_root_f(delta);
    if (s >= kXDegF * kXDegF) {
      *xout = sqrt_a(s);
      return j4_degenerate_f(s);
    }
    float x = tail_pass_f(delta, sqrt_a(s));
    if (x >= 9.0f) {
      *xout = x;
      return j4_tail_f(x);
    }
    x = tail_pass_f(delta, x);
    if (x >= 7.0f) {
      *xout = x;
      return j4_tail_f(x);
    }
#pragma unroll 1
    for (int it = 0; it < 4; ++it) {
      const FD5f f = fd_eval_deg_f(x);
      const float i1 = rcp_a(f.f1), i2 = rcp_a(f.f2), i3 = rcp_a(f.f3), i4 = rcp_a(f.f4);
      const float j = f.f2 * f.f2 * i1 * i3;
      const float dj = j * (2.0f * f.f1 * i2 - f.f0 * i1 - f.f2 * i3);
      const float dx = (J2 - j) * rcp_a(dj);
      const float J4 = f.f3 * f.f3 * i2 * i4;
      if (fabsf(dx) < 5e-4f * x || it == 3) {
        const float dJ4 = J4 * (2.0f * f.f2 * i3 - f.f1 * i2 - f.f3 * i4);
        *xout = x + dx;
        return J4 + dJ4 * dx;
      }
      x += dx;
    }
  }
  float x = 1.0f, lo = L.x_lo, hi = 6.0f;  // J_2(6) = 1.40 > 4/3: the root lies below
  float J4 = 0.0f;
#pragma unroll 1
  for (int it = 0; it < 24; ++it) {
    const FD5f f = fd_eval_f(x);
    const float i1 = rcp_a(f.f1), i2 = rcp_a(f.f2), i3 = rcp_a(f.f3), i4 = rcp_a(f.f4);
    const float j = f.f2 * f.f2 * i1 * i3;
    const float g = j - J2;
    const float dj = j * (2.0f * f.f1 * i2 - f.f0 * i1 - f.f2 * i3);
    const float dx = -g * rcp_a(dj);
    J4 = f.f3 * f.f3 * i2 * i4;
    if (g < 0.0f) lo = x; else hi = x;
    if (fabsf(dx) < 5e-4f * fabsf(x) || it == 23) {
      const float dJ4 = J4 * (2.0f * f.f2 * i3 - f.f1 * i2 - f.f3 * i4);
      *xout = x + dx;
      return J4 + dJ4 * dx;
    }
    float xn = x + dx;
    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
    x = xn;
  }
  *xout = x;
  return J4;
}

// J_4 through the learned inversion: the network gives (T, mu) from (n, e),
// e = 2 n J_2/3, hence x_0 = mu/T; one Newton step on J_2(x) = J_2 polishes
// it to x_1; the residual check evaluates f_0..f_4 at x_1 and accepts when the
// remaining Newton correction dx is below 5e-4 x_1 (the acceptance of the
// exact iteration), returning J_4(x_1) + J_4'(x_1) dx.  Otherwise *fallback is
// set and the exact inversion runs.
__device__ __forceinline__ float j4_surrogate_f(float n, float delta, const InvLimitsF& L, const MlpParams& W,
                                                int* fallback) {
  const float J2 = 1.5f - delta;
  if (!(J2 == J2) || !(J2 < L.j2_hi) || J2 <= L.j2_lo) {  // non-finite or clamped: the exact path handles it
    float xx;
    return j4_from_delta_f(delta, L, &xx);
  }
  float y0, y1, T, mu;
  mlp_forward_f(W, n, delta, y0, y1);  // e = 2 n J_2/3 enters as delta = 3/2 - J_2
  mlp_outputs_to_state(y0, y1, T, mu);
  float x = fminf(fmaxf(mu * rcp_a(T), L.x_lo), L.x_hi);
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

// Collision of one cell from its pulled deviations g[9]; stores at `off`.
template <class T, int STAT, bool SURR = false>
__device__ __forceinline__ void collide_store_dev(const ProbDev& P, const float g[9], T* __restrict__ fout,
                                                  int64_t plane, int off, const InvLimitsF& L,
                                                  const MlpParams* W = nullptr, int* fallback = nullptr) {
  const float nref = P.f.n_ref, ndref = P.f.ndelta_ref;
  const float dn = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
  const float jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
  const float jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
  const float G1 = g[0] - ((g[5] + g[6]) + (g[7] + g[8]));
  const float n = nref + dn;
  const float in = __fdividef(1.0f, n);
  const float ux = jx * in, uy = jy * in;
  const float u2 = ux * ux + uy * uy;
  const float X = G1 + n * u2;
  float J2, J4;
  if (STAT == STAT_FD) {
    const float delta = (ndref + 1.5f * X) * in;  // 3/2 - J_2
    J2 = 1.5f - delta;
    if (SURR) {
      J4 = j4_surrogate_f(n, delta, L, *W, fallback);
    } else {
      float xx;
      J4 = j4_from_delta_f(delta, L, &xx);
    }
  } else {
    J2 = (float)FixedJ<STAT>::j2;
    J4 = (float)FixedJ<STAT>::j4;
  }
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

}  // namespace lbm
