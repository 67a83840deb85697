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


// Tile rows per tensor-core round.  Two rows per round (two independent MMA
// chains in flight) need 128 TMEM columns, 74 KB of shared memory and about
// 170 registers per thread, leaving 3 CTAs per SM; one row per round leaves 5
// and measured 12 % faster on the 4096^2 lattice.
__host__ __device__ constexpr int tc_rows(int /*TY*/) { return 1; }
// Dynamic shared memory of the kernel, in this order: the network's operands;
// per round row the input block (128 x 16 FP16) and the hidden activations
// (128 x 64 FP16); two stages of pulled populations (per row 9 x 128 words).
__host__ __device__ constexpr int tc_smem_x(int /*R*/) { return kTcBytes; }
__host__ __device__ constexpr int tc_smem_a(int R) { return tc_smem_x(R) + R * kTileX * 16 * 2; }
__host__ __device__ constexpr int tc_smem_g(int R) { return tc_smem_a(R) + R * kTileX * kH * 2; }
__host__ __device__ constexpr int tc_smem(int R) { return tc_smem_g(R) + 2 * R * 9 * kTileX * 4; }
static_assert(tc_smem_a(1) % 16 == 0 && tc_smem_g(2) % 16 == 0, "operand blocks must be 16-byte aligned");

__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Starts the asynchronous pull of cell (x, y)'s nine populations into the
// stage words st + a * 512 bytes (a = 0..8; same sources as gather_dev).
// 16-bit populations travel in the aligned 4-byte word that holds them; the
// returned bits say which half (bit a set: the upper one).
template <class T>
__device__ __forceinline__ uint32_t prefetch_cell(const T* __restrict__ fin, int64_t plane, const ProbDev& P, int x,
                                                  int y, bool xin, uint32_t st) {
  const T* src[9];
  if (xin && y >= 1 && y <= P.ny - 2) {
    const int off = (int)P.base + y * P.pitch + x;
    const int pt = P.pitch;
    src[0] = fin + off;
    src[1] = fin + (plane + (off - 1));
    src[2] = fin + (2 * plane + (off - pt));
    src[3] = fin + (3 * plane + (off + 1));
    src[4] = fin + (4 * plane + (off + pt));
    src[5] = fin + (5 * plane + (off - pt - 1));
    src[6] = fin + (6 * plane + (off - pt + 1));
    src[7] = fin + (7 * plane + (off + pt + 1));
    src[8] = fin + (8 * plane + (off + pt - 1));
  } else {
    const PullIdx32 q = pull_index32(P, x, y);
    auto s = [&](int a, int r, int xs, int opp) -> const T* {
      return (r < 0 || xs < 0) ? fin + (opp * plane + (q.row + x)) : fin + (a * plane + (r + xs));
    };
    src[0] = fin + (q.row + x);
    src[1] = s(1, q.row, q.xm, 3);
    src[2] = s(2, q.rm, x, 4);
    src[3] = s(3, q.row, q.xp, 1);
    src[4] = s(4, q.rp, x, 2);
    src[5] = s(5, q.rm, q.xm, 7);
    src[6] = s(6, q.rm, q.xp, 8);
    src[7] = s(7, q.rp, q.xp, 5);
    src[8] = s(8, q.rp, q.xm, 6);
  }
  uint32_t bits = 0;
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    uintptr_t p = reinterpret_cast<uintptr_t>(src[a]);
    if (sizeof(T) == 2) {
      bits |= (uint32_t)((p >> 1) & 1u) << a;
      p &= ~(uintptr_t)3;
    }
    cp_async4(st + (uint32_t)(a * kTileX * 4), reinterpret_cast<const void*>(p));
  }
  return bits;
}

// Population a of this thread's cell from its stage words.
template <class T>
__device__ __forceinline__ float stage_pop(const unsigned char* st, int a, uint32_t bits) {
  const uint32_t w = *reinterpret_cast<const uint32_t*>(st + a * kTileX * 4);
  if (sizeof(T) == 4) return __uint_as_float(w);
  const uint32_t h = ((bits >> a) & 1u) ? (w >> 16) : (w & 0xffffu);
  return __uint_as_float(h << 16);  // bfloat16 -> float
}

// The FD step with the learned inversion, all three layers on the tensor
// cores.  Each round serves R = tc_rows(TY) tile rows of 128 cells (one cell
// per thread and row); every row is an M = 128 operand with its own 64 TMEM
// columns:
//  0. the populations of the round were pulled into a shared stage by
//     cp.async during the previous round; the next round's pull starts as
//     soon as this round's moments are formed (across tile boundaries of the
//     persistent sweep);
//  1. each thread writes its cells' input rows (n, l split into FP16 hi/lo
//     parts, constant columns for the biases) to sX; one thread issues the
//     layer-1 MMAs (K = 16, N = 64);
//  2. each warp reads its 32 lanes back, applies SiLU by packed FP16 tanh
//     and writes h1 to sA; layer 2 is four K = 16 MMAs against W2 plus one
//     against the bias block (N = 64), per row;
//  3. the same for h2; layer 3 is N = 16 (rows hi and lo of W3, bias block);
//     y = D[0..1] + D[2..3];
//  4. the polish, the residual check and the relaxation per cell, with the
//     populations read again from the stage.
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
__global__ void __launch_bounds__(kTileX, tc_rows(TY) == 1 ? 5 : 3)
    stream_collide_surr_tc(const T* __restrict__ fin, T* __restrict__ fout, const ProbDev* __restrict__ probs,
                           int nprob, int ntiles, int64_t plane, InvLimitsF L,
                           unsigned long long* __restrict__ counters, const uint4* __restrict__ wtc, int polls) {
  constexpr int R = tc_rows(TY);
  constexpr int RPT = (TY + R - 1) / R;  // rounds per tile
  constexpr int kCols = R * kH;          // TMEM columns
  extern __shared__ __align__(1024) unsigned char smem_dyn[];
  unsigned char* const sW = smem_dyn;
  unsigned char* const sX = smem_dyn + tc_smem_x(R);
  unsigned char* const sA = smem_dyn + tc_smem_a(R);
  unsigned char* const sG = smem_dyn + tc_smem_g(R);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int tid = (int)threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < kTcBytes / 16; i += kTileX) reinterpret_cast<uint4*>(sW)[i] = wtc[i];
#pragma unroll
  for (int r = 0; r < R; ++r)
    *reinterpret_cast<uint4*>(sX + r * kTileX * 32 + tc::kmajor_off(tid, 8, kTileX)) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&tmem_slot, kCols);
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
  const uint32_t uA = tc::smem_u32(sA), uX = tc::smem_u32(sX), uW = tc::smem_u32(sW), uG = tc::smem_u32(sG);
  // layers 1 and 2 accumulate in FP16 (their outputs become FP16 operands
  // anyway; the polish and the residual check absorb the rounding), layer 3
  // in FP32
  const uint32_t id64 = tc::idesc_f16_f16(kTileX, kH), id16 = tc::idesc_f16_f32(kTileX, 16);
  constexpr uint32_t kLboA = (kTileX / 8) * 128, kLbo64 = (kH / 8) * 128, kLbo16 = (16 / 8) * 128;
  constexpr uint32_t kBlkX = kTileX * 16 * 2, kBlkA = kTileX * kH * 2, kRowG = 9 * kTileX * 4;
  uint32_t phase = 0, last = 0;
  bool failed = false;
  unsigned nfb = 0, nev = 0;

  auto issue = [&](int layer) {
    if (tid == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const uint32_t d = tmem + (uint32_t)(r * kH), xb = uX + r * kBlkX, ab = uA + r * kBlkA;
        if (layer == 1) {
          tc::mma_f16(d, tc::smem_desc(xb, kLboA, 128), tc::smem_desc(uW + kTcB1, kLbo64, 128), id64, 0u);
        } else {
          const uint32_t bw = layer == 2 ? uW + kTcB2 : uW + kTcB3;
          const uint32_t bb = layer == 2 ? uW + kTcB2b : uW + kTcB3b;
          const uint32_t lbo = layer == 2 ? kLbo64 : kLbo16;
          const uint32_t id = layer == 2 ? id64 : id16;
#pragma unroll
          for (int s = 0; s < kH / 16; ++s)
            tc::mma_f16(d, tc::smem_desc(ab + (uint32_t)s * 2 * kLboA, kLboA, 128),
                        tc::smem_desc(bw + (uint32_t)s * 2 * lbo, lbo, 128), id, s > 0 ? 1u : 0u);
          tc::mma_f16(d, tc::smem_desc(xb, kLboA, 128), tc::smem_desc(bb, lbo, 128), id, 1u);
        }
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
  // TMEM reads, to the issuing thread
  auto publish = [&]() {
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  };
  // SiLU of the FP16 TMEM columns of row r (holding z/2) into row tid of sA
  // block r: the packed load gives the pairs (k, k + 1) the operand stores
  auto act_store = [&](int r) {
    uint32_t v[32];
    tc::tmem_ld64_pack16(tl + (uint32_t)(r * kH), v);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      uint4 w;
      w.x = tc::silu2_packed(v[4 * c + 0]);
      w.y = tc::silu2_packed(v[4 * c + 1]);
      w.z = tc::silu2_packed(v[4 * c + 2]);
      w.w = tc::silu2_packed(v[4 * c + 3]);
      *reinterpret_cast<uint4*>(sA + r * kBlkA + tc::kmajor_off(tid, 8 * c, kTileX)) = w;
    }
  };
  // round k of this CTA: its problem, tile origin and rows
  struct Round {
    int p, x0, yb, y1;
    bool xin, valid;
  };
  auto decode = [&](int k) -> Round {
    Round rd{0, 0, 0, 0, false, false};
    const int tile = (int)blockIdx.x + (k / RPT) * (int)gridDim.x;
    rd.valid = PERSIST ? tile < ntiles : k < RPT;
    if (rd.valid) {
      rd.p = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
      const ProbDev& P = probs[rd.p];
      const int lt = tile - (int)P.tile_begin;
      const int ty = lt / P.tiles_x;
      rd.x0 = (lt - ty * P.tiles_x) * kTileX;
      rd.yb = ty * TY + (k % RPT) * R;
      rd.y1 = min(ty * TY + TY, P.ny);
      rd.xin = rd.x0 >= 1 && rd.x0 + kTileX <= P.nx - 1;
    }
    return rd;
  };
  auto prefetch = [&](const Round& rd, int stage) -> uint32_t {
    uint32_t bits = 0;
    if (rd.valid) {
      const ProbDev& P = probs[rd.p];
      const int x = rd.x0 + tid;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (x < P.nx && rd.yb + r < rd.y1)
          bits |= prefetch_cell<T>(fin, plane, P, x, rd.yb + r, rd.xin,
                                   uG + (uint32_t)((stage * R + r) * kRowG + tid * 4))
                  << (9 * r);
    }
    cp_async_commit();
    return bits;
  };

  Round cur = decode(0);
  uint32_t bits = prefetch(cur, 0);
#pragma unroll 1
  for (int k = 0; cur.valid; ++k) {
    const int stage = k & 1;
    cp_async_wait_all();
    const Round nxt = decode(k + 1);
    const ProbDev& P = probs[cur.p];
    const int x = cur.x0 + tid;
    CellMom m[R];
    bool act[R], use[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      act[r] = x < P.nx && cur.yb + r < cur.y1;
      m[r] = CellMom{};
      m[r].n = 1.0f;
      m[r].delta = 0.1f;
      if (act[r]) {
        const unsigned char* st = sG + (stage * R + r) * kRowG + tid * 4;
        float g[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) g[a] = stage_pop<T>(st, a, bits >> (9 * r));
        m[r] = dev_moments(P, g);
      }
      use[r] = act[r] && net_cell(m[r].n, m[r].delta);
    }
    const uint32_t bits_nxt = prefetch(nxt, stage ^ 1);
    float yo[R][2];
    bool have = false;
    if (!failed) {
      bool warp_net = false;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        float i0 = 0.0f, i1 = 0.0f;
        if (use[r]) {
          i0 = fminf(fmaxf((m[r].n - kSurNMid) * (1.0f / kSurNHalf), -8.0f), 8.0f);
          i1 = fminf(fmaxf((__logf(m[r].delta) - kSurLdMid) * (1.0f / kSurLdHalf), -8.0f), 8.0f);
        }
        const __half nh = __float2half_rn(i0), lh = __float2half_rn(i1);
        const __half nl = __float2half_rn(i0 - __half2float(nh)), ll = __float2half_rn(i1 - __half2float(lh));
        const __half one = __float2half_rn(1.0f);
        uint4 row;
        __half2 t;
        t = __halves2half2(nh, nl);
        row.x = *reinterpret_cast<const uint32_t*>(&t);
        t = __halves2half2(nh, lh);
        row.y = *reinterpret_cast<const uint32_t*>(&t);
        t = __halves2half2(ll, lh);
        row.z = *reinterpret_cast<const uint32_t*>(&t);
        t = __halves2half2(one, one);
        row.w = *reinterpret_cast<const uint32_t*>(&t);
        *reinterpret_cast<uint4*>(sX + r * kBlkX + tc::kmajor_off(tid, 0, kTileX)) = row;
        warp_net = warp_net || use[r];
      }
      warp_net = __any_sync(0xffffffffu, warp_net);
      publish();
#pragma unroll 1
      for (int layer = 1; layer <= 2 && !failed; ++layer) {
        issue(layer);
        failed = !wait_round();
        if (!failed) {
          if (warp_net) {
#pragma unroll
            for (int r = 0; r < R; ++r) act_store(r);
          }
          publish();
        }
      }
      if (!failed) {
        issue(3);
        failed = !wait_round();
        if (!failed && warp_net) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            float v[4];
            tc::tmem_ld4(tl + (uint32_t)(r * kH), v);
            yo[r][0] = v[0] + v[2];
            yo[r][1] = v[1] + v[3];
          }
          have = true;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (!act[r]) continue;
      int fb = 0;
      float J4;
      if (use[r] && have) {
        J4 = j4_polish_f(x_from_outputs(yo[r][0], yo[r][1]), m[r].delta, L, &fb);
      } else {
        float xx;
        J4 = j4_from_delta_f(m[r].delta, L, &xx);
        fb = use[r] ? 1 : 0;
      }
      nfb += (unsigned)fb;
      nev += use[r] ? 1u : 0u;
      const unsigned char* st = sG + (stage * R + r) * kRowG + tid * 4;
      float g[9];
#pragma unroll
      for (int a = 0; a < 9; ++a) g[a] = stage_pop<T>(st, a, bits >> (9 * r));
      const int off = (int)P.base + (cur.yb + r) * P.pitch + x;
      relax_store_dev<T, STAT_FD>(P, g, m[r], 1.5f - m[r].delta, J4, fout, plane, off);
    }
    cur = nxt;
    bits = bits_nxt;
  }
  cp_async_wait_all();
  if (failed && tid == 0) {  // failed is uniform across the CTA
    atomicAdd(&counters[2], 1ull);
    // the last round, if it is still in flight, with the full limit
    if (!tc::mbar_wait(&mbar, last, kTcWaitPolls)) atomicAdd(&counters[3], 1ull);
  }
  flush_counts(nfb, nev, counters);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

}  // namespace lbm
