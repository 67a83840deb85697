// FP32 / BF16 deviation storage with the Fermi-Dirac inversion in FP64
// (LBM_INV_EXACT_F64): the reduced-precision step of lbm_dev32.cuh, whose
// populations, moment sums and equilibrium stay FP32, except for the
// inversion J_2 -> (x, J_4) of Sect. "Generalized polynomials in D
// dimensions", which runs in FP64 as in the FP64 step.
//
// delta = 3/2 - J_2 comes from the FP32 deviation moments (no cancellation);
// widened to FP64, J_2 = 3/2 - delta is exact for delta >= 2^-29 (every t of
// the clamp interval gives delta > 4e-6).  j4_fp64 then inverts it in FP64
// (degenerate closed form for x >= 40, else Newton from the FP32 start to
// 1e-13), and J_4 is rounded once to FP32 for the equilibrium.  The only
// difference from the FP32 step is therefore the inversion's own error:
// about 1e-7 relative in FP32 against 1e-13 here.
#pragma once
#include "launch.h"
#include "lbm_dev32.cuh"

namespace lbm {

// J_4 (and x) of a cell from its FP32 delta, by the FP64 inversion.
__device__ __forceinline__ float j4_x64(float delta, const InvLimits& L, const InvLimitsF& Lf, double* x) {
  int clamped;
  return (float)j4_fp64(1.5 - (double)delta, L, Lf, x, &clamped);
}

// The FP32/BF16 deviation step with the FP64 inversion: tiles, gather, moments
// and relaxation as stream_collide_dev (the next row's loads in flight during
// the current row's collision).
template <class T, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX) stream_collide_dev_x64(const T* __restrict__ fin, T* __restrict__ fout,
                                                                 const ProbDev* __restrict__ probs, int nprob,
                                                                 int ntiles, int64_t plane, InvLimits L,
                                                                 InvLimitsF Lf) {
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
        const CellMom m = dev_moments(P, g);
        double xx;
        const float J4 = j4_x64(m.delta, L, Lf, &xx);
        relax_store_dev<T, STAT_FD>(P, g, m, 1.5f - m.delta, J4, fout, plane, off);
      }
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
}

// T, mu and t = T/T_F of every cell of one problem from the FP64 inversion of
// the step's own FP32 delta, for lbm_moments of these contexts (run after
// moments_dev_kernel, whose other outputs and sums stand): x from j4_x64,
// t = 1/f_1(x), theta = n t/(2 pi) with n the FP64 sum of the stored
// populations, mu = theta x.  Null outputs are skipped.
template <class T, class O>
__global__ void closure_x64_kernel(const T* __restrict__ f, ProbDev P, int64_t plane, InvLimits L, InvLimitsF Lf,
                                   O* __restrict__ oT, O* __restrict__ omu, O* __restrict__ ot) {
  const int64_t cells = (int64_t)P.nx * P.ny;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cells) return;
  const int64_t c = P.base + (i / P.nx) * P.pitch + (i % P.nx);
  float g[9];
  double n = P.nsum_ref;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    g[a] = Dev<T>::ld(f[a * plane + c]);
    n += (double)g[a];
  }
  const CellMom m = dev_moments(P, g);
  double x;
  j4_x64(m.delta, L, Lf, &x);
  const double t = 1.0 / (fmax(x, 0.0) + log1p(exp(-fabs(x))));  // 1/f_1(x)
  const double theta = n * t * (1.0 / (2.0 * kPi));
  if (oT) oT[i] = (O)theta;
  if (omu) omu[i] = (O)(theta * x);
  if (ot) ot[i] = (O)t;
}

// Launcher of the step for FP32 (f32) or BF16 deviations, step_x64.cu.
void launch_step_x64(bool f32, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);

}  // namespace lbm
