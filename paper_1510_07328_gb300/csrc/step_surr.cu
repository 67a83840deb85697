// Step kernels with the learned inversion (FP32 and BF16 deviation storage):
// instantiations and launchers.
#include <algorithm>

#include "lbm_surr.cuh"
#include "lbm_surr_mma.cuh"

namespace lbm {

template <class T, int TY>
static void go_surr(unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c, const MlpParams& W) {
  if ((int)grid < a.ntiles)
    stream_collide_surr<T, TY, true><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob, a.ntiles,
                                                             a.plane, a.limf, c, W);
  else
    stream_collide_surr<T, TY, false><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob, a.ntiles,
                                                              a.plane, a.limf, c, W);
}

template <class T>
static void surr_rows(int rows, unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c,
                      const MlpParams& W) {
  switch (rows) {
    case 1: go_surr<T, 1>(grid, s, a, c, W); break;
    case 2: go_surr<T, 2>(grid, s, a, c, W); break;
    case 8: go_surr<T, 8>(grid, s, a, c, W); break;
    default: go_surr<T, 4>(grid, s, a, c, W); break;
  }
}

void launch_step_surr_f32(int rows, unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c,
                          const MlpParams& W) {
  surr_rows<float>(rows, grid, s, a, c, W);
}

void launch_step_surr_bf16(int rows, unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c,
                           const MlpParams& W) {
  surr_rows<__nv_bfloat16>(rows, grid, s, a, c, W);
}

template <class T, int TY>
static void go_surr_tc(unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c, const void* wtc) {
  constexpr int smem = tc_smem(tc_rows(TY));
  const uint4* w = (const uint4*)wtc;
  if ((int)grid < a.ntiles)
    stream_collide_surr_tc<T, TY, true><<<grid, kTileX, smem, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob,
                                                                   a.ntiles, a.plane, a.limf, c, w, a.tc_polls);
  else
    stream_collide_surr_tc<T, TY, false><<<grid, kTileX, smem, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob,
                                                                    a.ntiles, a.plane, a.limf, c, w, a.tc_polls);
}

// Sets one instantiation's shared-memory attributes and returns the CTAs
// resident per SM, from its registers, its shared memory and its TMEM
// columns (the runtime's occupancy query does not account for tensor
// memory); 0 on error.
template <class T, int TY, bool PERSIST>
static int prepare_one() {
  auto k = stream_collide_surr_tc<T, TY, PERSIST>;
  constexpr int R = tc_rows(TY);
  constexpr int smem_k = tc_smem(R);
  constexpr int cols = R * kH;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_k) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess) return 0;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 0;
  int dev = 0, regs_sm = 0, smem_sm = 0, reserved = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess) return 0;
  const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;  // allocated per warp in units of 256
  const int by_regs = regs_sm / (warp_regs * (kTileX / 32));
  const int by_smem = smem_sm / ((int)fa.sharedSizeBytes + smem_k + reserved);
  const int by_tmem = 512 / cols;
  return std::max(0, std::min(std::min(by_regs, by_smem), std::min(by_tmem, 2048 / kTileX)));
}

template <class T, int TY>
static int prepare_rows() {
  return std::min(prepare_one<T, TY, true>(), prepare_one<T, TY, false>());
}

int prepare_surr_tc(bool bf16, int rows) {
  switch (rows) {
    case 1: return bf16 ? prepare_rows<__nv_bfloat16, 1>() : prepare_rows<float, 1>();
    case 2: return bf16 ? prepare_rows<__nv_bfloat16, 2>() : prepare_rows<float, 2>();
    case 8: return bf16 ? prepare_rows<__nv_bfloat16, 8>() : prepare_rows<float, 8>();
    default: return bf16 ? prepare_rows<__nv_bfloat16, 4>() : prepare_rows<float, 4>();
  }
}

template <class T>
static void surr_tc_rows(int rows, unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c,
                         const void* wtc) {
  switch (rows) {
    case 1: go_surr_tc<T, 1>(grid, s, a, c, wtc); break;
    case 2: go_surr_tc<T, 2>(grid, s, a, c, wtc); break;
    case 8: go_surr_tc<T, 8>(grid, s, a, c, wtc); break;
    default: go_surr_tc<T, 4>(grid, s, a, c, wtc); break;
  }
}

void launch_step_surr_tc_f32(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                             unsigned long long* counters, const void* wtc) {
  surr_tc_rows<float>(rows, grid, s, a, counters, wtc);
}

void launch_step_surr_tc_bf16(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                              unsigned long long* counters, const void* wtc) {
  surr_tc_rows<__nv_bfloat16>(rows, grid, s, a, counters, wtc);
}

template <class T, int TY>
static void go_surr_mma(unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c, const void* wmm) {
  const uint4* w = (const uint4*)wmm;
  if ((int)grid < a.ntiles)
    stream_collide_surr_mma<T, TY, true><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob,
                                                                 a.ntiles, a.plane, a.limf, c, w);
  else
    stream_collide_surr_mma<T, TY, false><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob,
                                                                  a.ntiles, a.plane, a.limf, c, w);
}

template <class T, int TY>
static int resident_mma() {
  int n1 = 0, n2 = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, stream_collide_surr_mma<T, TY, true>, kTileX, 0) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n2, stream_collide_surr_mma<T, TY, false>, kTileX, 0) !=
          cudaSuccess)
    return 0;
  return std::min(n1, n2);
}

int prepare_surr_mma(bool bf16, int rows) {
  switch (rows) {
    case 1: return bf16 ? resident_mma<__nv_bfloat16, 1>() : resident_mma<float, 1>();
    case 2: return bf16 ? resident_mma<__nv_bfloat16, 2>() : resident_mma<float, 2>();
    case 8: return bf16 ? resident_mma<__nv_bfloat16, 8>() : resident_mma<float, 8>();
    default: return bf16 ? resident_mma<__nv_bfloat16, 4>() : resident_mma<float, 4>();
  }
}

template <class T>
static void surr_mma_rows(int rows, unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* c,
                          const void* wmm) {
  switch (rows) {
    case 1: go_surr_mma<T, 1>(grid, s, a, c, wmm); break;
    case 2: go_surr_mma<T, 2>(grid, s, a, c, wmm); break;
    case 8: go_surr_mma<T, 8>(grid, s, a, c, wmm); break;
    default: go_surr_mma<T, 4>(grid, s, a, c, wmm); break;
  }
}

void launch_step_surr_mma_f32(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                              unsigned long long* counters, const void* wmm) {
  surr_mma_rows<float>(rows, grid, s, a, counters, wmm);
}

void launch_step_surr_mma_bf16(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                               unsigned long long* counters, const void* wmm) {
  surr_mma_rows<__nv_bfloat16>(rows, grid, s, a, counters, wmm);
}

}  // namespace lbm
