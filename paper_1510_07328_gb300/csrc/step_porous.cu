// d2v9 step with obstacles and a body force: instantiations and launcher
// (prec 0 FP64, 1 FP32 deviations, 2 BF16 deviations).
#include "launch.h"
#include "lbm_porous.cuh"

namespace lbm {

template <class T, int STAT, int TY>
static void go_porous(unsigned grid, cudaStream_t s, const StepArgs& a) {
  if ((int)grid < a.ntiles)
    stream_collide_porous<T, STAT, TY, true><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob,
                                                                     a.ntiles, a.plane, a.lim, a.limf);
  else
    stream_collide_porous<T, STAT, TY, false><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob,
                                                                      a.ntiles, a.plane, a.lim, a.limf);
}

template <class T, int STAT>
static void rows_t(int rows, unsigned grid, cudaStream_t s, const StepArgs& a) {
  switch (rows) {
    case 1: go_porous<T, STAT, 1>(grid, s, a); break;
    case 2: go_porous<T, STAT, 2>(grid, s, a); break;
    case 8: go_porous<T, STAT, 8>(grid, s, a); break;
    default: go_porous<T, STAT, 4>(grid, s, a); break;
  }
}

template <class T>
static void stat_t(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a) {
  switch (stat) {
    case STAT_FD: rows_t<T, STAT_FD>(rows, grid, s, a); break;
    case STAT_T0: rows_t<T, STAT_T0>(rows, grid, s, a); break;
    default: rows_t<T, STAT_MB>(rows, grid, s, a); break;
  }
}

void launch_pull_code(const ProbDev& P, uint16_t* code, cudaStream_t s) {
  const int64_t cells = (int64_t)P.nx * P.ny;
  pull_code_kernel<<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(P, code);
}

void launch_step_porous(int prec, int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a) {
  switch (prec) {
    case 0: stat_t<double>(stat, rows, grid, s, a); break;
    case 1: stat_t<float>(stat, rows, grid, s, a); break;
    default: stat_t<__nv_bfloat16>(stat, rows, grid, s, a); break;
  }
}

}  // namespace lbm
