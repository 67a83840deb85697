// Step kernels with __nv_bfloat16 deviation storage: instantiations and launcher.
#include "lbm_dev32.cuh"

namespace lbm {

template <int STAT, int TY>
static void go(unsigned grid, cudaStream_t s, const StepArgs& a) {
  if ((int)grid < a.ntiles)
    stream_collide_dev<__nv_bfloat16, STAT, TY, true><<<grid, kTileX, 0, s>>>((const __nv_bfloat16*)a.in, (__nv_bfloat16*)a.out, a.probs, a.nprob,
                                                                   a.ntiles, a.plane, a.limf);
  else
    stream_collide_dev<__nv_bfloat16, STAT, TY, false><<<grid, kTileX, 0, s>>>((const __nv_bfloat16*)a.in, (__nv_bfloat16*)a.out, a.probs, a.nprob,
                                                          a.ntiles, a.plane, a.limf);
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

void launch_step_bf16(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a) {
  switch (stat) {
    case STAT_FD: by_rows<STAT_FD>(rows, grid, s, a); break;
    case STAT_T0: by_rows<STAT_T0>(rows, grid, s, a); break;
    case STAT_FT: by_rows<STAT_FT>(rows, grid, s, a); break;
    default: by_rows<STAT_MB>(rows, grid, s, a); break;
  }
}

}  // namespace lbm
