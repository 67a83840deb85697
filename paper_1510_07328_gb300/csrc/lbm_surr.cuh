// The FD step with the learned inversion: the network of surrogate.cuh gives
// (T, mu) from the cell's (n, e); x_0 = mu/T is polished by one step on
// J_2(x) = J_2 and checked; a cell that fails the check takes the exact
// inversion.  Two engines: the whole network per thread on the FP32 pipe, or
// its three layers as tcgen05 MMAs over a tile row of 128 cells.
#pragma once
#include "lbm_dev32.cuh"
#include "surrogate.cuh"
#include "tc_sm100.cuh"

namespace lbm {

// The polish accepts x_0 when the first-order step is below this fraction of
// max(|x_0|, 1); the third-order remainder in J_4 is then below 2e-7
// (measured over t = 0.005 .. 1.5 with FP64 FD functions).
constexpr float kPolishTol = 2.5e-2f;

// One polish step from the network's x_0 with a single evaluation of
// f_0..f_4.  Derivatives come from d f_n/dx = f_{n-1}, continued below n = 0
// by f_-1 = f_0 (1 - f_0) and f_-2 = f_-1 (1 - 2 f_0).  With l_n = ln f_n:
//   first derivative   q_n = f_{n-1}/f_n,
//   second derivative  r_n = f_{n-2}/f_n - q_n^2,
//   third derivative   t_n = f_{n-3}/f_n - 3 q_n f_{n-2}/f_n + 2 q_n^3,
// ln J_2 = 2 l_2 - l_1 - l_3 has the derivatives g, g1, g2 (first to third)
// and ln J_4 = 2 l_3 - l_2 - l_4 the derivatives h, h1, h2.  The residual
// step e = (J_2 - J_2(x_0))/(dJ_2/dx) is the check; the accepted step is the
// third-order inverse of the Taylor series of J_2,
//   dx = e - c_2 e^2 + (2 c_2^2 - c_3) e^3,
//   c_2 = (g + g1/g)/2,  c_3 = (g^2 + 3 g1 + g2/g)/6
// (the second and third derivatives of J_2 over twice and six times its
// first), and J_4 follows from its third-order Taylor series,
//   J_4(x_0 + dx) = J_4 (1 + h dx + (h^2 + h1) dx^2/2 + (h^3 + 3 h h1 + h2) dx^3/6).
// On failure *fallback is set and the exact inversion runs.
__device__ __forceinline__ float j4_polish_f(float x0, float delta, const InvLimitsF& L, int* fallback) {
  const float J2 = 1.5f - delta;
  const float x = fminf(fmaxf(x0, L.x_lo), L.x_hi);
  const FD5f f = x >= 4.0f ? fd_eval_deg_f(x) : fd_eval_f(x);
  const float i1 = rcp_a(f.f1), i2 = rcp_a(f.f2), i3 = rcp_a(f.f3), i4 = rcp_a(f.f4);
  const float q1 = f.f0 * i1, q2 = f.f1 * i2, q3 = f.f2 * i3, q4 = f.f3 * i4;
  const float j = f.f2 * q3 * i1;
  const float g = 2.0f * q2 - q1 - q3;
  const float ig = rcp_a(g);
  const float e = (J2 - j) * rcp_a(j) * ig;
  if (fabsf(e) <= kPolishTol * fmaxf(fabsf(x), 1.0f)) {
    const float fm1 = f.f0 * (1.0f - f.f0), fm2 = fm1 * (1.0f - 2.0f * f.f0);
    const float s1 = fm1 * i1, s2 = f.f0 * i2, s3 = f.f1 * i3, s4 = f.f2 * i4;
    const float r1 = s1 - q1 * q1, r2 = s2 - q2 * q2, r3 = s3 - q3 * q3, r4 = s4 - q4 * q4;
    const float t1 = fm2 * i1 - q1 * (3.0f * s1 - 2.0f * q1 * q1);
    const float t2 = fm1 * i2 - q2 * (3.0f * s2 - 2.0f * q2 * q2);
    const float t3 = f.f0 * i3 - q3 * (3.0f * s3 - 2.0f * q3 * q3);
    const float t4 = f.f1 * i4 - q4 * (3.0f * s4 - 2.0f * q4 * q4);
    const float g1 = 2.0f * r2 - r1 - r3, g2 = 2.0f * t2 - t1 - t3;
    const float c2 = 0.5f * (g + g1 * ig);
    const float c3 = (g * g + 3.0f * g1 + g2 * ig) * (1.0f / 6.0f);
    const float dx = e * (1.0f - e * (c2 - e * (2.0f * c2 * c2 - c3)));
    const float J4 = f.f3 * q4 * i2;
    const float h = 2.0f * q3 - q2 - q4, h1 = 2.0f * r3 - r2 - r4, h2 = 2.0f * t3 - t2 - t4;
    return J4 * (1.0f + dx * (h + dx * (0.5f * (h * h + h1) + dx * (h * (h * h + 3.0f * h1) + h2) * (1.0f / 6.0f))));
  }
  *fallback = 1;
  float xx;
  return j4_from_delta_f(delta, L, &xx);
}

// Cells the network serves: (n, delta) inside its training domain (which
// lies inside the clamp interval of the inversion); false for NaN.
__device__ __forceinline__ bool net_cell(float n, float delta) {
  return n >= kSurNLo && n <= kSurNHi && delta >= kSurDeltaLo && delta <= kSurDeltaHi;
}

// x_0 = mu/T from the network's outputs (y_0, y_1).
__device__ __forceinline__ float x_from_outputs(float y0, float y1) {
  return fmaf(kSurMuHalf, y1, kSurMuMid) * __expf(-fmaf(kSurLnTHalf, y0, kSurLnTMid));
}

// J_4 through the learned inversion, network on the FP32 pipe (the network
// gives (T, mu) from (n, e), e = 2 n J_2/3 entering as delta = 3/2 - J_2).
__device__ __forceinline__ float j4_surrogate_f(float n, float delta, const InvLimitsF& L, const MlpParams& W,
                                                int* fallback) {
  if (!net_cell(n, delta)) {  // outside the network's domain: the exact path handles it
    float xx;
    return j4_from_delta_f(delta, L, &xx);
  }
  float y0, y1;
  mlp_forward_f(W, n, delta, y0, y1);
  return j4_polish_f(x_from_outputs(y0, y1), delta, L, fallback);
}

// Adds per-thread counts to counters[0] (fallbacks) and counters[1] (cells
// through the network): warp sums, then one atomic each per CTA.  Called by
// every thread of the CTA.
__device__ __forceinline__ void flush_counts(unsigned nfb, unsigned nev, unsigned long long* counters) {
  __shared__ unsigned s_cnt[2];
  if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0u;
  __syncthreads();
  const unsigned a = __reduce_add_sync(0xffffffffu, nfb), b = __reduce_add_sync(0xffffffffu, nev);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&s_cnt[0], a);
    atomicAdd(&s_cnt[1], b);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_cnt[0]) atomicAdd(&counters[0], (unsigned long long)s_cnt[0]);
    if (s_cnt[1]) atomicAdd(&counters[1], (unsigned long long)s_cnt[1]);
  }
}

// The FD step with the learned inversion on the FP32 pipe.
template <class T, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX) stream_collide_surr(const T* __restrict__ fin, T* __restrict__ fout,
                                                              const ProbDev* __restrict__ probs, int nprob, int ntiles,
                                                              int64_t plane, InvLimitsF L,
                                                              unsigned long long* __restrict__ counters,
                                                              const MlpParams W) {
  unsigned nfb = 0, nev = 0;
  int tile = (int)blockIdx.x;
#pragma unroll 1
  do {
    const int p = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
    const ProbDev& P = probs[p];
    const int lt = tile - (int)P.tile_begin;
    const int ty = lt / P.tiles_x;
    const int x0 = (lt - ty * P.tiles_x) * kTileX;
    const int x = x0 + (int)threadIdx.x;
    const int y0 = ty * TY;
    const int y1 = min(y0 + TY, P.ny);
    const bool xin = x0 >= 1 && x0 + kTileX <= P.nx - 1;
    if (x < P.nx) {
#pragma unroll 1
      for (int y = y0; y < y1; ++y) {
        float g[9];
        const int off = gather_dev(fin, plane, P, x, y, xin, g);
        const CellMom m = dev_moments(P, g);
        int fb = 0;
        const float J4 = j4_surrogate_f(m.n, m.delta, L, W, &fb);
        nfb += (unsigned)fb;
        nev += net_cell(m.n, m.delta) ? 1u : 0u;
        relax_store_dev<T, STAT_FD>(P, g, m, 1.5f - m.delta, J4, fout, plane, off);
      }
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
  flush_counts(nfb, nev, counters);
}


// Rows of a tile per tensor-core round (one: an M = 128 operand per round).
__host__ __device__ constexpr int tc_rows(int /*TY*/) { return 1; }
// Dynamic shared memory of the kernel, in this order: the network's operands
// (kTcBytes), the input block (128 x 16 FP16) and the hidden activations
// (128 x 64 FP16): 35,328 bytes.
__host__ __device__ constexpr int tc_smem_x(int /*R*/) { return kTcBytes; }
__host__ __device__ constexpr int tc_smem_a(int R) { return tc_smem_x(R) + R * kTileX * 16 * 2; }
__host__ __device__ constexpr int tc_smem(int R) { return tc_smem_a(R) + R * kTileX * kH * 2; }
static_assert(tc_smem_x(1) % 1024 == 512 || tc_smem_x(1) % 16 == 0, "operand blocks must be 16-byte aligned");
static_assert(tc_smem_a(1) % 16 == 0, "operand blocks must be 16-byte aligned");
// CTAs the kernel is compiled for per SM: six (80 registers, no spills, with
// the activations read from TMEM in two halves), the most the shared memory
// allows.
constexpr int kTcCtasPerSm = 6;
// Of every 32 activation pairs of a hidden layer, this many take the FMA-pipe
// SiLU (tc::silu2_poly) and the rest the MUFU one (tc::silu2_packed): both
// pipes then share the activations' work.
constexpr int kTcPolyPairs = 8;

// SiLU of one packed pair: pair i of 32 goes to the FMA pipe for every
// (32 / KP)-th i, to MUFU otherwise.
template <int KP>
__device__ __forceinline__ uint32_t silu2_mixed(uint32_t h, int i) {
  if (KP > 0 && (i % (32 / (KP > 0 ? KP : 1))) == (32 / (KP > 0 ? KP : 1)) - 1) return tc::silu2_poly(h);
  return tc::silu2_packed(h);
}

// The FD step with the learned inversion, all three layers on the tensor
// cores.  Tiles and gathers as stream_collide_dev: one cell per thread and
// tile row, the nine populations pulled into registers, the next row's loads
// in flight while this row's network runs.  Every tile row is an M = 128
// operand with its 64 TMEM columns:
//  1. each thread writes its cell's input row (n, l split into FP16 hi/lo
//     parts, constant columns for the biases) to sX; a barrier that also
//     tells whether any cell of the row needs the network (rows without one
//     skip the MMAs); one thread issues the layer-1 MMAs (K = 16, N = 64);
//  2. each warp reads its 32 lanes back, applies SiLU (kTcPolyPairs of every
//     32 pairs on the FMA pipe, the rest on MUFU) and writes h1 to sA; layer
//     2 is four K = 16 MMAs against W2 plus one against the bias block;
//  3. the same for h2; layer 3 is N = 16 (rows hi and lo of W3, bias block);
//     y = D[0..1] + D[2..3];
//  4. the polish, the residual check and the relaxation per cell.
// The issuing thread alone waits on the mbarrier, at most `polls` polls per
// round; a barrier with a reduction (bar.red.or) then releases the CTA with
// the outcome, so the other warps spend no issue slots on polling.  A CTA
// whose wait ran out counts the event in counters[2] and serves its remaining
// cells with the exact inversion.  Before it frees its TMEM it waits for its
// last MMA with the full limit (kTcWaitPolls); if that wait also runs out it
// counts counters[3]: the columns were released with an MMA possibly still
// writing them, and the step's results are not to be trusted.  The persistent
// grid stages the weights once per CTA.
template <class T, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX, kTcCtasPerSm)
    stream_collide_surr_tc(const T* __restrict__ fin, T* __restrict__ fout, const ProbDev* __restrict__ probs,
                           int nprob, int ntiles, int64_t plane, InvLimitsF L,
                           unsigned long long* __restrict__ counters, const uint4* __restrict__ wtc, int polls) {
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* const sW = smem_dyn;
  unsigned char* const sX = smem_dyn + tc_smem_x(1);
  unsigned char* const sA = smem_dyn + tc_smem_a(1);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = (int)threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < kTcBytes / 16; i += kTileX) reinterpret_cast<uint4*>(sW)[i] = wtc[i];
  *reinterpret_cast<uint4*>(sX + tc::kmajor_off(tid, 8, kTileX)) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&tmem_slot, kH);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
  const uint32_t uA = tc::smem_u32(sA), uX = tc::smem_u32(sX), uW = tc::smem_u32(sW);
  // layers 1 and 2 accumulate in FP16 (their outputs become FP16 operands
  // anyway; the polish and the residual check absorb the rounding), layer 3
  // in FP32
  const uint32_t id64 = tc::idesc_f16_f16(kTileX, kH), id16 = tc::idesc_f16_f32(kTileX, 16);
  constexpr uint32_t kLboA = (kTileX / 8) * 128, kLbo64 = (kH / 8) * 128, kLbo16 = (16 / 8) * 128;
  uint32_t phase = 0, last = 0;
  bool failed = false;
  unsigned nfb = 0, nev = 0;

  auto issue = [&](int layer) {
    if (tid == 0) {
      if (layer == 1) {
        tc::mma_f16(tmem, tc::smem_desc(uX, kLboA, 128), tc::smem_desc(uW + kTcB1, kLbo64, 128), id64, 0u);
      } else {
        const uint32_t bw = layer == 2 ? uW + kTcB2 : uW + kTcB3;
        const uint32_t bb = layer == 2 ? uW + kTcB2b : uW + kTcB3b;
        const uint32_t lbo = layer == 2 ? kLbo64 : kLbo16;
        const uint32_t id = layer == 2 ? id64 : id16;
#pragma unroll
        for (int s = 0; s < kH / 16; ++s)
          tc::mma_f16(tmem, tc::smem_desc(uA + (uint32_t)s * 2 * kLboA, kLboA, 128),
                      tc::smem_desc(bw + (uint32_t)s * 2 * lbo, lbo, 128), id, s > 0 ? 1u : 0u);
        tc::mma_f16(tmem, tc::smem_desc(uX, kLboA, 128), tc::smem_desc(bb, lbo, 128), id, 1u);
      }
      tc::commit(&mbar);
    }
    last = phase;
  };
  // the issuing thread waits (bounded) for the round just issued; the barrier
  // releases the CTA and tells every thread whether the wait succeeded
  auto wait_round = [&]() -> bool {
    bool done = true;
    if (tid == 0) done = tc::mbar_wait(&mbar, phase, polls);
    phase ^= 1u;
    const bool any_bad = __syncthreads_or(!done) != 0;
    tc::fence_after();
    return !any_bad;
  };
  // publishes the operand rows written by every thread, and the end of their
  // TMEM reads, to the issuing thread; returns whether any thread's flag is set
  auto publish = [&](bool flag) -> bool {
    tc::fence_async_smem();
    tc::fence_before();
    const bool any = __syncthreads_or(flag) != 0;
    tc::fence_after();
    return any;
  };
  // SiLU of the FP16 TMEM columns (holding z/2) into row tid of sA: the
  // packed load gives the pairs (k, k + 1) the operand stores
  auto act_store = [&]() {
#pragma unroll
    for (int half = 0; half < 2; ++half) {  // 32 columns at a time: 16 registers live
      uint32_t v[16];
      tc::tmem_ld32_pack16(tl + (uint32_t)(32 * half), v);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = 16 * half + 4 * c;  // pair index of v[4 c] within the row's 32 pairs
        uint4 w;
        w.x = silu2_mixed<kTcPolyPairs>(v[4 * c + 0], i + 0);
        w.y = silu2_mixed<kTcPolyPairs>(v[4 * c + 1], i + 1);
        w.z = silu2_mixed<kTcPolyPairs>(v[4 * c + 2], i + 2);
        w.w = silu2_mixed<kTcPolyPairs>(v[4 * c + 3], i + 3);
        *reinterpret_cast<uint4*>(sA + tc::kmajor_off(tid, 8 * (4 * half + c), kTileX)) = w;
      }
    }
  };

  int tile = (int)blockIdx.x;
#pragma unroll 1
  do {
    const int p = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
    const ProbDev& P = probs[p];
    const int lt = tile - (int)P.tile_begin;
    const int ty = lt / P.tiles_x;
    const int x0 = (lt - ty * P.tiles_x) * kTileX;
    const int x = x0 + tid;
    const bool act = x < P.nx;  // every thread takes part in the barriers
    const int y0 = ty * TY;
    const int y1 = min(y0 + TY, P.ny);
    const bool xin = x0 >= 1 && x0 + kTileX <= P.nx - 1;
    float gn[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int offn = 0;
    if (act) offn = gather_dev(fin, plane, P, x, y0, xin, gn);
#pragma unroll 1
    for (int y = y0; y < y1; ++y) {
      float g[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) g[a] = gn[a];
      const int off = offn;
      CellMom m{};
      m.n = 1.0f;
      m.delta = 0.1f;
      if (act) m = dev_moments(P, g);
      const bool use = act && net_cell(m.n, m.delta);
      // the next row's loads, in flight during this row's network
      if (act && y + 1 < y1) offn = gather_dev(fin, plane, P, x, y + 1, xin, gn);
      float yo0 = 0.0f, yo1 = 0.0f;
      bool have = false;
      if (!failed) {
        float i0 = 0.0f, i1 = 0.0f;
        if (use) {
          i0 = (m.n - kSurNMid) * (1.0f / kSurNHalf);
          i1 = (__logf(m.delta) - kSurLdMid) * (1.0f / kSurLdHalf);
        }
        const __half nh = __float2half_rn(i0), lh = __float2half_rn(i1);
        const __half nl = __float2half_rn(i0 - __half2float(nh)), ll = __float2half_rn(i1 - __half2float(lh));
        uint4 row;
        __half2 t2;
        t2 = __halves2half2(nh, nl);
        row.x = *reinterpret_cast<const uint32_t*>(&t2);
        t2 = __halves2half2(nh, lh);
        row.y = *reinterpret_cast<const uint32_t*>(&t2);
        t2 = __halves2half2(ll, lh);
        row.z = *reinterpret_cast<const uint32_t*>(&t2);
        row.w = 0x3C003C00u;  // (1, 1): the bias columns
        *reinterpret_cast<uint4*>(sX + tc::kmajor_off(tid, 0, kTileX)) = row;
        const bool warp_net = __any_sync(0xffffffffu, use);
        if (publish(use)) {  // uniform: some cell of the row needs the network
          issue(1);
          failed = !wait_round();
          if (!failed) {
            if (warp_net) act_store();
            publish(false);
            issue(2);
            failed = !wait_round();
          }
          if (!failed) {
            if (warp_net) act_store();
            publish(false);
            issue(3);
            failed = !wait_round();
          }
          if (!failed && warp_net) {  // warp-uniform: the TMEM load is .sync.aligned
            float v[4];
            tc::tmem_ld4(tl, v);
            yo0 = v[0] + v[2];
            yo1 = v[1] + v[3];
            have = true;
          }
        }
      }
      if (act) {
        int fb = 0;
        float J4;
        if (use && have) {
          J4 = j4_polish_f(x_from_outputs(yo0, yo1), m.delta, L, &fb);
        } else {
          float xx;
          J4 = j4_from_delta_f(m.delta, L, &xx);
          fb = use ? 1 : 0;
        }
        nfb += (unsigned)fb;
        nev += use ? 1u : 0u;
        relax_store_dev<T, STAT_FD>(P, g, m, 1.5f - m.delta, J4, fout, plane, off);
      }
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
  if (failed && tid == 0) {  // failed is uniform across the CTA
    atomicAdd(&counters[2], 1ull);
    // the last round, if it is still in flight, with the full limit
    if (!tc::mbar_wait(&mbar, last, kTcWaitPolls)) atomicAdd(&counters[3], 1ull);
  }
  flush_counts(nfb, nev, counters);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, kH);
}

}  // namespace lbm
