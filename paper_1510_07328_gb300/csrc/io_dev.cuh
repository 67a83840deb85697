// Initial state of deviation-stored contexts (FP32 or BF16 g = f - W_ref),
// computed with the reduced-precision step's own arithmetic: the equilibrium
// in FP32 deviation form and the Fermi-Dirac closure from t in FP32, with
// errors of the order of one FP32 step.  (Their moments take the closure
// quantities from the FP32 inversion: moments_dev_kernel.)
#pragma once
#include "lbm_dev32.cuh"

namespace lbm {


// g = f_eq(n, u, t) - W_ref per cell, FP32 deviation form: the step's
// relaxation with omega = 1 from g = 0 (g_eq = Delta W + W (S - 1), never f).
// X64 (contexts with the FP64 inversion, FD statistics): the closure
// delta = 3/2 - J_2(t) and J_4(t) in FP64, each rounded once to FP32.
template <class T, int STAT, bool X64 = false>
__global__ void init_dev_kernel(T* __restrict__ f, ProbDev P, int64_t plane, InitDesc d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cells = (int64_t)P.nx * P.ny;
  if (i >= cells) return;
  const int y = (int)(i / P.nx), x = (int)(i % P.nx);
  double n, ux, uy, t;
  if (d.kind == 2) {
    n = d.n[i]; ux = d.ux[i]; uy = d.uy[i]; t = d.t[i];
  } else if (d.kind == 3) {
    n = d.nf[i]; ux = d.uxf[i]; uy = d.uyf[i]; t = d.tf[i];
  } else {
    const int r = d.kind == 0 ? (x >= d.x0) : (x >= d.x0) + 2 * (y >= d.y0);
    n = d.s[r][0]; ux = d.s[r][1]; uy = d.s[r][2]; t = d.s[r][3];
  }
  float delta, J4;
  if (X64) {
    double J2d, J4d;
    closure_from_t<STAT_FD>(t, J2d, J4d);
    delta = (float)(1.5 - J2d);
    J4 = (float)J4d;
  } else if (STAT == STAT_FD || STAT == STAT_FT) {
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
