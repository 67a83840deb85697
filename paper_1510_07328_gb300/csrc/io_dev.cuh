// Initial state of deviation-stored contexts (FP32 or BF16 g = f - W_ref),
// computed with the reduced-precision step's own arithmetic: the equilibrium
// in FP32 deviation form and the Fermi-Dirac closure from t in FP32, with
// errors of the order of one FP32 step.  (Their moments take the closure
// quantities from the FP32 inversion: moments_kernel with F32CL.)
#pragma once
#include "lbm_dev32.cuh"

namespace lbm {

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

// g = f_eq(n, u, t) - W_ref per cell, FP32 deviation form: the step's
// relaxation with omega = 1 from g = 0 (g_eq = Delta W + W (S - 1), never f).
template <class T, int STAT>
__global__ void init_dev_kernel(T* __restrict__ f, ProbDev P, int64_t plane, InitDesc d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cells = (int64_t)P.nx * P.ny;
  if (i >= cells) return;
  const int y = (int)(i / P.nx), x = (int)(i % P.nx);
  double n, ux, uy, t;
  if (d.kind == 2) {
    n = d.n[i]; ux = d.ux[i]; uy = d.uy[i]; t = d.t[i];
  } else {
    const int r = d.kind == 0 ? (x >= d.x0) : (x >= d.x0) + 2 * (y >= d.y0);
    n = d.s[r][0]; ux = d.s[r][1]; uy = d.s[r][2]; t = d.s[r][3];
  }
  float delta, J4;
  if (STAT == STAT_FD) {
    closure_dev_from_t((float)t, delta, J4);
  } else {
    delta = (float)(1.5 - FixedJ<STAT>::j2);
    J4 = (float)FixedJ<STAT>::j4;
  }
  CellMom m;
  m.n = (float)n;
  m.dn = (float)(n - P.n_ref);
  m.in = 1.0f / m.n;
  m.ux = (float)ux;
  m.uy = (float)uy;
  m.u2 = m.ux * m.ux + m.uy * m.uy;
  m.delta = delta;
  // n (3/2 - J_2) = n_ref (3/2 - J_2,ref) + (3/2) X  (the deviation moments)
  m.X = (m.n * delta - P.f.ndelta_ref) * (2.0f / 3.0f);
  ProbDev Q = P;
  Q.f.omega = 1.0f;
  const float g0[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int c = (int)(P.base + (int64_t)y * P.pitch + x);
  relax_store_dev<T, STAT>(Q, g0, m, 1.5f - delta, J4, f, plane, c);
}

}  // namespace lbm
