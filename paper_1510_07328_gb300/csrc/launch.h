// Host-side launchers of the step kernels, one translation unit per storage
// type (compiled in parallel).  rows: rows per tile (1, 2, 4 or 8); grid: CTAs
// launched (ntiles for one tile per CTA, fewer for a persistent sweep).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_device_f32.cuh"
#include "lbm_kernels.cuh"

namespace lbm {

// Polls of an mbarrier wait of the tensor-core engine before it counts as
// failed (per layer round; the wait at the end of the kernel always uses this
// full limit).
constexpr int kTcWaitPolls = 1 << 22;

struct StepArgs {
  const void* in;
  void* out;
  const ProbDev* probs;
  int nprob;
  int ntiles;
  int64_t plane;
  InvLimits lim;
  InvLimitsF limf;
  int tc_polls;  // per-round poll limit of the tensor-core engine (lbm_surrogate_wait_limit)
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
// the same with the network by warp-level MMAs (mma.sync); wmm: the network's
// fragments (kMmBytes bytes, 16-byte aligned).  prepare_surr_mma returns the
// kernels' CTAs resident per SM for `rows` rows per tile (0: error).
int prepare_surr_mma(bool bf16, int rows);
void launch_step_surr_mma_f32(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                              unsigned long long* counters, const void* wmm);
void launch_step_surr_mma_bf16(int rows, unsigned grid, cudaStream_t s, const StepArgs& a,
                               unsigned long long* counters, const void* wmm);
// d1v3 (prec 0 FP64, 1 FP32 deviations, 2 BF16 deviations; stat STAT_T0 or
// STAT_MB): step, initial equilibrium, moments with per-block partial sums,
// and populations to (get) or from FP64 buffers [3][nx]
void launch_step_d1(int prec, int stat, unsigned grid, cudaStream_t s, const StepArgs& a);
void launch_init_d1(int prec, int stat, void* f, const ProbDev& P, int64_t plane, const InitDesc& d, cudaStream_t s);
void launch_moments_d1(int prec, int stat, const void* f, const ProbDev& P, int64_t plane, double* const o[6],
                       double* partials, unsigned g, cudaStream_t s);
void launch_pop_d1(int prec, bool get, void* f, const ProbDev& P, int64_t plane, double* buf, cudaStream_t s);
// d2v9 with obstacles (ProbDev::solid) and a body force (ProbDev::fx, fy)
void launch_step_porous(int prec, int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);
// Pull codes of one problem's cells from its obstacle mask (lbm_porous.cuh).
void launch_pull_code(const ProbDev& P, uint16_t* code, cudaStream_t s);
void launch_step_f64(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);
void launch_step_f32(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);
void launch_step_bf16(int stat, int rows, unsigned grid, cudaStream_t s, const StepArgs& a);

}  // namespace lbm
