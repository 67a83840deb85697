// FP64 step kernels: instantiations and launcher.
#include "launch.h"

namespace lbm {

bool valid_rows(int rows) { return rows == 1 || rows == 2 || rows == 4 || rows == 8; }

template <int STAT, int TY>
static void go(unsigned grid, cudaStream_t s, const StepArgs& a) {
  if ((int)grid < a.ntiles)
    stream_collide_f64<STAT, TY, true><<<grid, kTileX, 0, s>>>((const double*)a.in, (double*)a.out, a.probs, a.nprob,
                                                               a.ntiles, a.plane, a.lim, a.limf);
  else
    stream_collide_f64<STAT, TY, false><<<grid, kTileX, 0, s>>>((const double*)a.in, (double*)a.out, a.probs, a.nprob,
                                                       a.ntiles, a.plane, a.lim, a.limf);
}

template <int STAT>
static void by_rows(int rows, unsigned grid, cudaStream_t s, const StepArgs& a) {
  switch (rows) {
    case 1: go<STAT, 1>(grid, s, a); break;
    case 2: go<STAT, 2>(grid, s, a); break;
    case 8: go<STAT, 8>(grid, s, a); break;
    default: go<STAT, 4>(grid, s, a); break;
  }
}

void launch_step_f64(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a) {
  switch (stat) {
    case STAT_FD: by_rows<STAT_FD>(rows, grid, s, a); break;
    case STAT_T0: by_rows<STAT_T0>(rows, grid, s, a); break;
    case STAT_FT: by_rows<STAT_FT>(rows, grid, s, a); break;
    default: by_rows<STAT_MB>(rows, grid, s, a); break;
  }
}

}  // namespace lbm
