// FP32 Fermi-Dirac functions and the FP32 inversion J_2 -> (x, J_4) for
// D = 2 (same expansions as fd_device.cuh, FP32 term counts, closed forms in
// the degenerate regime; J_4 straight from delta = 3/2 - J_2 by fitted
// polynomials).  Used by the reduced-precision step, and as the starting
// value of the FP64 step's inversion.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace lbm {

constexpr float kPi2f = 9.8696044010893586f;
constexpr float kXDegF = 17.0f;  // e^-17 = 4e-8: S_n tails below FP32 resolution

struct InvLimitsF {
  float x_lo, x_hi, j2_lo, j2_hi, j4_lo, j4_hi;  // the clamp interval's ends: x, J_2 and J_4
};

struct FD5f {
  float f0, f1, f2, f3, f4;
};

// 1/k for the series terms (k = 1..12), read warp-uniformly.
static __constant__ float c_inv_k[13] = {0.f,     1.f,         0.5f,   1.f / 3.f, 0.25f,      0.2f,       1.f / 6.f,
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

// 3/2 - J_2 at x = 7 and at x = 17 (the closed form's threshold).
constexpr float kDelta7 = 0.078501010f;
constexpr float kDelta17 = 0.016323599f;

// x for 7 < x < 17 from delta = 3/2 - J_2: a degree-8 polynomial in
// u = (ln delta - m)/h (u in [-1, 1] over [0.98 delta(17), 1.02 delta(7)]),
// largest relative error 5.4e-9 (least-squares fit to J_2 = f_2^2/(f_1 f_3)
// from mpmath's polylogarithm; fit_x_of_j2.py); 1.8e-7 in FP32 evaluation.
__device__ __forceinline__ float x_degenerate_fit(float delta) {
  constexpr float c[9] = {-2.114108754e-05f, -5.251981112e-05f, 5.705624853e-05f, -1.250000357e-03f, 1.020720050e-02f,
                          -1.428147596e-01f, 8.829952733e-01f, -4.990830054e+00f, 1.115240803e+01f};
  const float u = (__logf(delta) + 3.330093647f) * 1.241846532f;
  float x = c[0];
#pragma unroll
  for (int k = 1; k < 9; ++k) x = fmaf(x, u, c[k]);
  return x;
}

// J_4 for x >= 17 straight from delta = 3/2 - J_2 (no root, no division): a
// degree-4 polynomial in delta over [0, 1.02 delta(17)], within 1.6e-10 of
// the degenerate closed form J_4 = P_3^2/(P_2 P_4) at the quadratic root
// (whose dropped e^{-x} tails are below 3.4e-9 of J_4 there); about one
// FP32 ulp in FP32 evaluation (least-squares fit, fit_x_of_j2.py).
__device__ __forceinline__ float j4_degenerate_poly(float delta) {
  constexpr float c[5] = {-6.607502108e+00f, -3.215488438e+00f, 1.066513921e+00f, -8.888885225e-01f,
                          1.333333333e+00f};
  float j = c[0];
#pragma unroll
  for (int k = 1; k < 5; ++k) j = fmaf(j, delta, c[k]);
  return j;
}

// J_4 for 7 < x < 17 straight from delta: a degree-7 polynomial in
// v = (delta - m)/h (v in [-1, 1] over [0.98 delta(17), 1.02 delta(7)]),
// within 1.4e-9 of J_4 = f_3^2/(f_2 f_4) (least-squares fit to mpmath's
// polylogarithm, fit_x_of_j2.py); about one FP32 ulp in FP32 evaluation.
__device__ __forceinline__ float j4_mid_poly(float delta) {
  constexpr float c[8] = {3.285286587e-07f, -6.328906060e-07f, -9.770357170e-07f, 1.359526894e-05f,
                          -7.823930935e-05f, 6.168045261e-04f, -2.594511986e-02f, 1.292719233e+00f};
  const float v = fmaf(delta, 3.121395636e+01f, -4.803407843e-02f * 3.121395636e+01f);
  float j = c[0];
#pragma unroll
  for (int k = 1; k < 8; ++k) j = fmaf(j, v, c[k]);
  return j;
}

// J_4 for x_lo < x <= 7 straight from delta: a degree-12 polynomial in
// v = (delta - m)/h (v in [-1, 1] over [delta(7.1), delta(x_lo - 0.05)],
// x_lo = x(t = 10)), within 5.6e-10 of J_4 = f_3^2/(f_2 f_4) (Chebyshev
// least-squares fit to mpmath's polylogarithm, fit_x_of_j2.py); about one
// FP32 ulp in FP32 evaluation.
__device__ __forceinline__ float j4_low_poly(float delta) {
  constexpr float c[13] = {3.751275144e-06f,  -8.171843462e-06f, 5.219605688e-06f,  -9.016432491e-06f,
                           3.008137632e-05f,  -5.869911291e-05f, 1.010758946e-04f,  -1.385486611e-04f,
                           3.636938822e-05f,  2.824311568e-04f,  1.345504631e-02f,  -1.320218322e-01f,
                           1.124292938e+00f};
  const float v = fmaf(delta, 4.861925282e+00f, -2.824715949e-01f * 4.861925282e+00f);
  float j = c[0];
#pragma unroll
  for (int k = 1; k < 13; ++k) j = fmaf(j, v, c[k]);
  return j;
}

// Starting value of the Newton branch (J_2(x_lo) < J_2 <= J_2(7)): x as a
// degree-8 polynomial in v = ln((J_2 - 1)/(3/2 - J_2)), largest error 4.0e-5
// over x in [x(t = 10) - 0.05, 7.3] (least-squares fit to J_2 = f_2^2/(f_1 f_3)
// from mpmath's polylogarithm; fit_x_of_j2.py).
__device__ __forceinline__ float x_start_general(float J2) {
  constexpr float c[9] = {5.482719542e-06f, 6.089144600e-05f, 1.952511272e-04f, 2.676517802e-04f, 6.391339607e-03f,
                          6.971210059e-02f, 3.455914096e-01f, 1.903484720e+00f, 2.431969767e+00f};
  const float v = __logf(__fdividef(J2 - 1.0f, 1.5f - J2));
  float x = c[0];
#pragma unroll
  for (int k = 1; k < 9; ++k) x = fmaf(x, v, c[k]);
  return x;
}

// x for x_lo < x <= 7 from J_2 (J_2(x_lo) < J_2 <= J_2(7)): safeguarded
// Newton on J_2(x) from the fitted start x_start_general (within 4e-5), each
// step one evaluation of f_0..f_3 (three-term series for x >= 4), stopping
// when the step is below 5e-4 |x| and returning x + dx (second-order
// remainder below 1e-7 |x|): one evaluation in practice, at most 24.
// J_2' = J_2 (2 f_1/f_2 - f_0/f_1 - f_2/f_3), from d f_n/dx = f_{n-1}.
__device__ __forceinline__ float x_general_f(float J2, const InvLimitsF& L) {
  float lo = L.x_lo, hi = 8.0f;  // J_2(8) > J_2(7): the root lies below
  float x = fminf(fmaxf(x_start_general(J2), lo), hi);
#pragma unroll 1
  for (int it = 0; it < 24; ++it) {
    const FD5f f = x >= 4.0f ? fd_eval_deg_f(x) : fd_eval_f(x);
    const float i1 = rcp_a(f.f1), i2 = rcp_a(f.f2), i3 = rcp_a(f.f3);
    const float j = f.f2 * f.f2 * i1 * i3;
    const float g = j - J2;
    const float dj = j * (2.0f * f.f1 * i2 - f.f0 * i1 - f.f2 * i3);
    const float dx = -g * rcp_a(dj);
    if (g < 0.0f) lo = x; else hi = x;
    if (fabsf(dx) < 5e-4f * fabsf(x) || it == 23) return x + dx;
    float xn = x + dx;
    if (!(xn > lo && xn < hi)) xn = 0.5f * (lo + hi);
    x = xn;
  }
  return x;
}

// J_4 from delta = 3/2 - J_2 in FP32 (the exact inversion, to FP32
// resolution; *xout receives x).
//  * non-finite input: propagated at once;
//  * J_2 beyond the clamp interval: x at the nearest end;
//  * otherwise J_4 from its polynomial in delta on each of three intervals,
//    and x (for callers that use it; the step does not) as follows:
//    - x >= 17 (delta <= 3/2 - J_2(17)): j4_degenerate_poly, x from the
//      degenerate quadratic root;
//    - 7 < x < 17 (delta < 3/2 - J_2(7)): j4_mid_poly, x from the fit
//      x_degenerate_fit (FP32-exact);
//    - x_lo < x <= 7: j4_low_poly, x by x_general_f (Newton).
__device__ __forceinline__ float j4_from_delta_f(float delta, const InvLimitsF& L, float* xout) {
  const float J2 = 1.5f - delta;
  if (!(J2 == J2)) {  // non-finite state: propagate without iterating
    *xout = J2;
    return J2;
  }
  if (!(J2 < L.j2_hi)) {
    *xout = L.x_hi;
    return L.j4_hi;
  }
  if (J2 <= L.j2_lo) {
    *xout = L.x_lo;
    return L.j4_lo;
  }
  if (delta <= kDelta17) {  // x (for callers that use it) from the degenerate root
    *xout = sqrt_a(deg_root_f(delta));
    return j4_degenerate_poly(delta);
  }
  if (delta < kDelta7) {
    *xout = x_degenerate_fit(delta);
    return j4_mid_poly(delta);
  }
  *xout = x_general_f(J2, L);
  return j4_low_poly(delta);
}

// delta = 3/2 - J_2 and J_4 of the FD equilibrium at t = T/T_F, FP32.
// x = mu/theta solves t = 1/f_1(x): x = 1/t + ln(1 - e^{-1/t}).  delta is
// formed without subtracting from 3/2 where it is small:
//  * x >= 17: the degenerate forms (tails e^{-x} < 4e-8 dropped),
//    3/2 - J_2 = pi^2 (3 s - pi^2)/(6 s (s + pi^2)), s = x^2, and
//    J_4 = P_3^2/(P_2 P_4);
//  * 4 <= x < 17: with y = e^{-x}, f_1 = x + l_1, f_2 = P_2 - s_2,
//    f_3 = P_3 + s_3 (three series terms, l_1 = ln(1 + y)),
//    1.5 f_1 f_3 - f_2^2 = pi^2 (3 s - pi^2)/36 + 1.5 (x s_3 + l_1 P_3 + l_1 s_3)
//                          + 2 P_2 s_2 - s_2^2,
//    since 1.5 x P_3 - P_2^2 = pi^2 (3 s - pi^2)/36; every correction is
//    positive and small, and delta = (1.5 f_1 f_3 - f_2^2)/(f_1 f_3);
//  * x < 4: delta >= 0.15 and 3/2 - J_2 from the FP32 series loses under 4 bits.
__device__ __forceinline__ void closure_dev_from_t(float t, float& delta, float& J4) {
  const float v = 1.0f / t;
  const float x = v + logf(-expm1f(-v));
  const float s = x * x;
  if (x >= kXDegF) {
    delta = kPi2f * (3.0f * s - kPi2f) / (6.0f * s * (s + kPi2f));
    J4 = j4_degenerate_f(s);
  } else if (x >= 4.0f) {
    const float y = expf(-x);
    float p2, p3, p4;
    fd_poly_f(x, p2, p3, p4);
    const float s2 = y * (1.0f + y * (-0.25f + y * (1.0f / 9.0f)));
    const float s3 = y * (1.0f + y * (-0.125f + y * (1.0f / 27.0f)));
    const float s4 = y * (1.0f + y * (-0.0625f + y * (1.0f / 81.0f)));
    const float l1 = log1pf(y);
    const float f1 = x + l1, f2 = p2 - s2, f3 = p3 + s3, f4 = p4 - s4;
    const float num = kPi2f * (3.0f * s - kPi2f) * (1.0f / 36.0f) + 1.5f * (x * s3 + l1 * p3 + l1 * s3) +
                      s2 * (2.0f * p2 - s2);
    delta = num / (f1 * f3);
    J4 = f3 * f3 / (f2 * f4);
  } else {
    const FD5f f = fd_eval_f(x);
    delta = 1.5f - f.f2 * f.f2 / (f.f1 * f.f3);
    J4 = f.f3 * f.f3 / (f.f2 * f.f4);
  }
}

}  // namespace lbm
