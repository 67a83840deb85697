// Step kernels of FP32 / BF16 deviation storage with the FP64 inversion
// (lbm_dev_x64.cuh): instantiations and launcher.
#include "lbm_dev_x64.cuh"

namespace lbm {

template <class T, int TY>
static void go(unsigned grid, cudaStream_t s, const StepArgs& a) {
  if ((int)grid < a.ntiles)
    stream_collide_dev_x64<T, TY, true><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob,
                                                               a.ntiles, a.plane, a.lim, a.limf);
  else
    stream_collide_dev_x64<T, TY, false><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob,
                                                                a.ntiles, a.plane, a.lim, a.limf);
}

template <class T>
static void by_rows(int rows, unsigned grid, cudaStream_t s, const StepArgs& a) {
  switch (rows) {
    case 1: go<T, 1>(grid, s, a); break;
    case 2: go<T, 2>(grid, s, a); break;
    case 8: go<T, 8>(grid, s, a); break;
    default: go<T, 4>(grid, s, a); break;
  }
}

void launch_step_x64(bool f32, int rows, unsigned grid, cudaStream_t s, const StepArgs& a) {
  if (f32)
    by_rows<float>(rows, grid, s, a);
  else
    by_rows<__nv_bfloat16>(rows, grid, s, a);
}

}  // namespace lbm
