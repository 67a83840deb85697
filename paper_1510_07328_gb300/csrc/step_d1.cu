// d1v3 kernels: instantiations and launchers (prec: 0 FP64, 1 FP32
// deviations, 2 BF16 deviations; stat: STAT_T0 or STAT_MB).
#include "launch.h"
#include "lbm_d1.cuh"

namespace lbm {

// grid: CTAs requested (ntiles: one sweep of kTilesD1 tiles per CTA).
template <class T, int STAT>
static void go_d1(unsigned grid, cudaStream_t s, const StepArgs& a) {
  const unsigned one_sweep = (unsigned)((a.ntiles + kTilesD1 - 1) / kTilesD1);
  if (grid >= one_sweep) grid = one_sweep;
  if ((long long)grid * kTilesD1 < a.ntiles)
    stream_collide_d1<T, STAT, true><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob, a.ntiles,
                                                             a.plane);
  else
    stream_collide_d1<T, STAT, false><<<grid, kTileX, 0, s>>>((const T*)a.in, (T*)a.out, a.probs, a.nprob, a.ntiles,
                                                              a.plane);
}

template <class T>
static void step_t(int stat, unsigned grid, cudaStream_t s, const StepArgs& a) {
  if (stat == STAT_T0) go_d1<T, STAT_T0>(grid, s, a);
  else go_d1<T, STAT_MB>(grid, s, a);
}

void launch_step_d1(int prec, int stat, unsigned grid, cudaStream_t s, const StepArgs& a) {
  switch (prec) {
    case 0: step_t<double>(stat, grid, s, a); break;
    case 1: step_t<float>(stat, grid, s, a); break;
    default: step_t<__nv_bfloat16>(stat, grid, s, a); break;
  }
}

template <class T>
static void init_t(int stat, void* f, const ProbDev& P, int64_t plane, const InitDesc& d, cudaStream_t s) {
  const unsigned g = (unsigned)((P.nx + 255) / 256);
  if (stat == STAT_T0) init_d1_kernel<T, STAT_T0><<<g, 256, 0, s>>>((T*)f, P, plane, d);
  else init_d1_kernel<T, STAT_MB><<<g, 256, 0, s>>>((T*)f, P, plane, d);
}

void launch_init_d1(int prec, int stat, void* f, const ProbDev& P, int64_t plane, const InitDesc& d, cudaStream_t s) {
  switch (prec) {
    case 0: init_t<double>(stat, f, P, plane, d, s); break;
    case 1: init_t<float>(stat, f, P, plane, d, s); break;
    default: init_t<__nv_bfloat16>(stat, f, P, plane, d, s); break;
  }
}

template <class T>
static void moments_t(int stat, const void* f, const ProbDev& P, int64_t plane, double* const o[6], double* partials,
                      unsigned g, cudaStream_t s) {
  if (stat == STAT_T0)
    moments_d1_kernel<T, STAT_T0><<<g, kMomThreads, 0, s>>>((const T*)f, P, plane, o[0], o[1], o[2], o[3], o[4], o[5],
                                                            partials);
  else
    moments_d1_kernel<T, STAT_MB><<<g, kMomThreads, 0, s>>>((const T*)f, P, plane, o[0], o[1], o[2], o[3], o[4], o[5],
                                                            partials);
}

void launch_moments_d1(int prec, int stat, const void* f, const ProbDev& P, int64_t plane, double* const o[6],
                       double* partials, unsigned g, cudaStream_t s) {
  switch (prec) {
    case 0: moments_t<double>(stat, f, P, plane, o, partials, g, s); break;
    case 1: moments_t<float>(stat, f, P, plane, o, partials, g, s); break;
    default: moments_t<__nv_bfloat16>(stat, f, P, plane, o, partials, g, s); break;
  }
}

template <class T>
static void pop_t(bool get, void* f, const ProbDev& P, int64_t plane, double* buf, cudaStream_t s) {
  const unsigned g = (unsigned)((P.nx + 255) / 256);
  if (get) get_pop_d1_kernel<T><<<g, 256, 0, s>>>((const T*)f, P, plane, buf);
  else set_pop_d1_kernel<T><<<g, 256, 0, s>>>((T*)f, P, plane, buf);
}

void launch_pop_d1(int prec, bool get, void* f, const ProbDev& P, int64_t plane, double* buf, cudaStream_t s) {
  switch (prec) {
    case 0: pop_t<double>(get, f, P, plane, buf, s); break;
    case 1: pop_t<float>(get, f, P, plane, buf, s); break;
    default: pop_t<__nv_bfloat16>(get, f, P, plane, buf, s); break;
  }
}

}  // namespace lbm
