// Host-side launchers of the step kernels, one translation unit per storage
// type (compiled in parallel).  rows: rows per tile (1, 2, 4 or 8); grid: CTAs
// launched (ntiles for one tile per CTA, fewer for a persistent sweep).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_device_f32.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

struct StepArgs {
  const void* in;
  void* out;
  const ProbDev* probs;
  int nprob;
  int ntiles;
  int64_t plane;
  InvLimits lim;
  InvLimitsF limf;
};

struct MlpParams;

bool valid_rows(int rows);
// learned-inversion step (FD statistics only); counters: fallbacks, evaluations
void launch_step_surr_f32(int rows, unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* counters,
                          const MlpParams& W);
void launch_step_surr_bf16(int rows, unsigned grid, cudaStream_t s, const StepArgs& a, unsigned long long* counters,
                           const MlpParams& W);
// the same with the hidden layer on the tensor cores (tcgen05); w2h: W2 as
// FP16 in the canonical K-major layout (4096 halves, 16-byte aligned)
void launch_step_surr_tc_f32(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                             unsigned long long* counters, const void* w2h, const MlpParams& W);
void launch_step_surr_tc_bf16(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                              unsigned long long* counters, const void* w2h, const MlpParams& W);
void launch_step_f64(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);
void launch_step_f32(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);
void launch_step_bf16(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);

}  // namespace lbm
