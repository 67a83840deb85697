// Step kernels with float deviation storage: instantiations and launcher.
#include "lbm_dev32.cuh"

namespace lbm {

template <int STAT, int TY>
static void go(unsigned grid, cudaStream_t s, const StepArgs& a) {
  if ((int)grid < a.ntiles)
    stream_collide_dev<float, STAT, TY, true><<<grid, kTileX, 0, s>>>((const float*)a.in, (float*)a.out, a.probs, a.nprob,
                                                                   a.ntiles, a.plane, a.limf);
  else
    stream_collide_dev<float, STAT, TY, false><<<grid, kTileX, 0, s>>>((const float*)a.in, (float*)a.out, a.probs, a.nprob,
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

void launch_step_f32(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a) {
  switch (stat) {
    case STAT_FD: by_rows<STAT_FD>(rows, grid, s, a); break;
    case STAT_T0: by_rows<STAT_T0>(rows, grid, s, a); break;
    default: by_rows<STAT_MB>(rows, grid, s, a); break;
  }
}

template <int TY>
static void go_surr(unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c, const MlpParams& W) {
  if ((int)grid < a.ntiles)
    stream_collide_surr<float, TY, true><<<grid, kTileX, 0, s>>>((const float*)a.in, (float*)a.out, a.probs, a.nprob,
                                                              a.ntiles, a.plane, a.limf, c, W);
  else
    stream_collide_surr<float, TY, false><<<grid, kTileX, 0, s>>>((const float*)a.in, (float*)a.out, a.probs, a.nprob,
                                                               a.ntiles, a.plane, a.limf, c, W);
}

void launch_step_surr_f32(int rows, unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c,
                          const MlpParams& W) {
  switch (rows) {
    case 1: go_surr<1>(grid, s, a, c, W); break;
    case 2: go_surr<2>(grid, s, a, c, W); break;
    case 8: go_surr<8>(grid, s, a, c, W); break;
    default: go_surr<4>(grid, s, a, c, W); break;
  }
}

template <int TY>
static void go_surr_tc(unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c, const void* w2h,
                       const MlpParams& W) {
  const __half* w = (const __half*)w2h;
  if ((int)grid < a.ntiles)
    stream_collide_surr_tc<float, TY, true><<<grid, kTileX, 0, s>>>((const float*)a.in, (float*)a.out, a.probs,
                                                                 a.nprob, a.ntiles, a.plane, a.limf, c, w, W);
  else
    stream_collide_surr_tc<float, TY, false><<<grid, kTileX, 0, s>>>((const float*)a.in, (float*)a.out, a.probs,
                                                                  a.nprob, a.ntiles, a.plane, a.limf, c, w, W);
}

void launch_step_surr_tc_f32(int rows, unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c,
                             const void* w2h, const MlpParams& W) {
  switch (rows) {
    case 1: go_surr_tc<1>(grid, s, a, c, w2h, W); break;
    case 2: go_surr_tc<2>(grid, s, a, c, w2h, W); break;
    case 8: go_surr_tc<8>(grid, s, a, c, w2h, W); break;
    default: go_surr_tc<4>(grid, s, a, c, w2h, W); break;
  }
}

}  // namespace lbm
