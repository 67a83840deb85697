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
// the same with the network's three layers on the tensor cores (tcgen05);
// wtc: the network's FP16 operands (kTcBytes bytes, 16-byte aligned).  The
// kernels need prepare_surr_tc first (outside stream capture): it sets the
// shared-memory attributes of the kernels for `rows` rows per tile and
// returns their CTAs resident per SM (0: error).
int prepare_surr_tc(bool bf16, int rows);
void launch_step_surr_tc_f32(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                             unsigned long long* counters, const void* wtc);
void launch_step_surr_tc_bf16(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                              unsigned long long* counters, const void* wtc);
void launch_step_f64(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);
void launch_step_f32(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);
void launch_step_bf16(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);

}  // namespace lbm
