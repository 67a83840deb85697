// The FD step with the learned inversion, the network evaluated by each warp
// on its own 32 cells with warp-level MMAs (mma.sync, FP16 operands,
// accumulators in registers: FP16 for the hidden layers, FP32 for the
// output).  Same network, input split, polish, residual check and fallback as
// the tcgen05 engine (lbm_surr.cuh); what differs is where the activations
// live.  The accumulator fragment of an m16n8 MMA holds the same (row,
// column) pairs as the A fragment of the next K = 16 MMA, so a layer's SiLU
// output feeds the next layer straight from registers: no shared memory round
// trip, no tensor memory, no barrier between the warps of a CTA.
#pragma once
#include "lbm_surr.cuh"

namespace lbm {
namespace wm {

constexpr unsigned kFull = 0xffffffffu;

// D = A B + D for a 16 x 8 x 8 product, FP16 accumulator (A two packed-FP16
// registers, B one, D two: rows g and g + 8, columns 2t, 2t + 1).
__device__ __forceinline__ void mma_k8_h(uint32_t (&d)[2], uint32_t a0, uint32_t a1, uint32_t b0) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f16.f16.f16.f16 {%0,%1}, {%2,%3}, {%4}, {%0,%1};"
               : "+r"(d[0]), "+r"(d[1])
               : "r"(a0), "r"(a1), "r"(b0));
}

// D += A B for a 16 x 8 x 16 product, FP16 accumulator.
__device__ __forceinline__ void mma_k16_h(uint32_t (&d)[2], const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f16.f16.f16.f16 {%0,%1}, {%2,%3,%4,%5}, {%6,%7}, {%0,%1};"
               : "+r"(d[0]), "+r"(d[1])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// D += A B for a 16 x 8 x 16 product, FP32 accumulator (rows g, g + 8 in
// d[0..1], d[2..3]).
__device__ __forceinline__ void mma_k16(float (&d)[4], const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared-memory fragment loads, kept in program order with the MMAs (volatile)
// so that the compiler does not hoist all of a layer's operands at once.
__device__ __forceinline__ uint2 lds2(const unsigned char* p) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(tc::smem_u32(p)));
  return v;
}
__device__ __forceinline__ uint4 lds4(const unsigned char* p) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(tc::smem_u32(p)));
  return v;
}
__device__ __forceinline__ float2 ldsf2(const unsigned char* p) {
  const uint2 v = lds2(p);
  return make_float2(__uint_as_float(v.x), __uint_as_float(v.y));
}

// Packed FP16 pairs (hi, lo) of the two network inputs of this lane's cell:
// v = hi + lo to about 2^-22.
__device__ __forceinline__ void split_inputs(float i0, float i1, uint32_t& nn, uint32_t& ll) {
  const __half nh = __float2half_rn(i0), lh = __float2half_rn(i1);
  const __half nl = __float2half_rn(i0 - __half2float(nh)), lo = __float2half_rn(i1 - __half2float(lh));
  const __half2 a = __halves2half2(nh, nl), b = __halves2half2(lh, lo);
  nn = *reinterpret_cast<const uint32_t*>(&a);
  ll = *reinterpret_cast<const uint32_t*>(&b);
}

// One m-tile (cells 16 mt .. 16 mt + 15 of the warp): layer-1 A fragment rows
// g and g + 8, then the three layers.  Layers 1 and 2 accumulate in FP16: the
// accumulator pair of rows g / g + 8 and columns 2t, 2t + 1 is already the
// packed operand the next layer's A fragment needs (their inputs and
// activations are FP16 anyway; the polish and the residual check absorb the
// accumulation rounding).  Layer 3 accumulates in FP32.  Returns this lane's
// accumulator of layer 3 (lanes with t = 0 hold (y_0, y_1) of rows g and
// g + 8).
__device__ __forceinline__ void net_mtile(const unsigned char* sW, int lane, uint32_t a0, uint32_t a1,
                                          float (&y)[4]) {
  const int t = lane & 3;
  uint32_t h[16];  // SiLU(layer 1): h[2 nt] row g, h[2 nt + 1] row g + 8, columns 8 nt + 2t, + 1
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const uint2 b = lds2(sW + kMmB1 + (p * 32 + lane) * 8);
    uint32_t d0[2] = {0u, 0u}, d1[2] = {0u, 0u};
    mma_k8_h(d0, a0, a1, b.x);
    mma_k8_h(d1, a0, a1, b.y);
    h[4 * p + 0] = tc::silu2_packed(d0[0]);
    h[4 * p + 1] = tc::silu2_packed(d0[1]);
    h[4 * p + 2] = tc::silu2_packed(d1[0]);
    h[4 * p + 3] = tc::silu2_packed(d1[1]);
  }
  // h[4c .. 4c + 3] is the A fragment of K chunk c of layer 2.  Its eight
  // n-tiles accumulate side by side (eight independent MMA chains); their
  // SiLU, in place, gives the four A fragments of layer 3.
  uint32_t d[16];  // layer-2 accumulators: d[2 nt] row g, d[2 nt + 1] row g + 8
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const uint2 c = lds2(sW + kMmC2 + (p * 4 + t) * 8);  // b2/2 of n-tiles 2p, 2p + 1 (FP16 pairs)
    d[4 * p + 0] = c.x;
    d[4 * p + 1] = c.x;
    d[4 * p + 2] = c.y;
    d[4 * p + 3] = c.y;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const uint4 b = lds4(sW + kMmB2 + ((k * 4 + p) * 32 + lane) * 16);
      mma_k16_h(*reinterpret_cast<uint32_t(*)[2]>(d + 4 * p), h + 4 * k, b.x, b.y);
      mma_k16_h(*reinterpret_cast<uint32_t(*)[2]>(d + 4 * p + 2), h + 4 * k, b.z, b.w);
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) d[i] = tc::silu2_packed(d[i]);
  // layer 3: the hi and lo weights as two chains, summed at the end
  const float2 b3 = ldsf2(sW + kMmC3);
  float yl[4] = {0.f, 0.f, 0.f, 0.f};
  y[0] = t == 0 ? b3.x : 0.0f;
  y[1] = t == 0 ? b3.y : 0.0f;
  y[2] = y[0];
  y[3] = y[1];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint4 b = lds4(sW + kMmB3 + (k * 32 + lane) * 16);
    mma_k16(y, d + 4 * k, b.x, b.y);   // W3 hi
    mma_k16(yl, d + 4 * k, b.z, b.w);  // W3 lo
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) y[i] += yl[i];
}

// Network outputs (y_0, y_1) of this lane's cell; every lane of the warp
// calls it (inputs of cells outside the network's domain are 0).
__device__ __forceinline__ void warp_net(const unsigned char* sW, int lane, float i0, float i1, float& y0,
                                         float& y1) {
  uint32_t nn, ll;
  split_inputs(i0, i1, nn, ll);
  const int g = lane >> 2, t = lane & 3;
  // feature pair t of the row (n hi, n lo | n hi, l hi | l lo, l hi | 1, 1)
  const uint32_t sel = t == 0 ? 0x3210u : (t == 1 ? 0x5410u : 0x5476u);
  const int src = (lane & 7) << 2;  // the lane holding this lane's output row
#pragma unroll
  for (int mt = 0; mt < 2; ++mt) {
    const int r0 = 16 * mt + g;
    const uint32_t n0 = __shfl_sync(kFull, nn, r0), l0 = __shfl_sync(kFull, ll, r0);
    const uint32_t n1 = __shfl_sync(kFull, nn, r0 + 8), l1 = __shfl_sync(kFull, ll, r0 + 8);
    const uint32_t a0 = t == 3 ? 0x3C003C00u : __byte_perm(n0, l0, sel);
    const uint32_t a1 = t == 3 ? 0x3C003C00u : __byte_perm(n1, l1, sel);
    float y[4];
    net_mtile(sW, lane, a0, a1, y);
    const float v0 = __shfl_sync(kFull, y[0], src), v1 = __shfl_sync(kFull, y[1], src);
    const float v2 = __shfl_sync(kFull, y[2], src), v3 = __shfl_sync(kFull, y[3], src);
    if ((lane >> 4) == mt) {
      y0 = (lane & 8) ? v2 : v0;
      y1 = (lane & 8) ? v3 : v1;
    }
  }
}

}  // namespace wm

// The FD step with the learned inversion, network by warp-level MMAs.  Tiles
// and gathers as stream_collide_dev (the next row's loads are issued after the
// current row's network, before its polish and relaxation); every lane of a warp that holds a cell of the
// lattice takes part in the network, lanes past the lattice's end with zero
// inputs.  A warp none of whose cells is a network cell skips it.  The
// persistent grid stages the operands (kMmBytes) once per CTA.
template <class T, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX, 5)
    stream_collide_surr_mma(const T* __restrict__ fin, T* __restrict__ fout, const ProbDev* __restrict__ probs,
                            int nprob, int ntiles, int64_t plane, InvLimitsF L,
                            unsigned long long* __restrict__ counters, const uint4* __restrict__ wmm) {
  __shared__ __align__(16) unsigned char sW[kMmBytes];
  const int tid = (int)threadIdx.x, lane = tid & 31;
  for (int i = tid; i < kMmBytes / 16; i += kTileX) reinterpret_cast<uint4*>(sW)[i] = wmm[i];
  __syncthreads();
  unsigned nfb = 0, nev = 0;
  int tile = (int)blockIdx.x;
#pragma unroll 1
  do {
    const int p = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
    const ProbDev& P = probs[p];
    const int lt = tile - (int)P.tile_begin;
    const int ty = lt / P.tiles_x;
    const int x0 = (lt - ty * P.tiles_x) * kTileX;
    const int x = x0 + tid;
    if (x0 + (tid & ~31) < P.nx) {  // warp-uniform
      const bool act = x < P.nx;
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
        const CellMom m = dev_moments(P, g);
        const bool use = act && net_cell(m.n, m.delta);
        float yo0 = 0.0f, yo1 = 0.0f;
        if (__any_sync(wm::kFull, use)) {
          float i0 = 0.0f, i1 = 0.0f;
          if (use) {
            i0 = fminf(fmaxf((m.n - kSurNMid) * (1.0f / kSurNHalf), -8.0f), 8.0f);
            i1 = fminf(fmaxf((__logf(m.delta) - kSurLdMid) * (1.0f / kSurLdHalf), -8.0f), 8.0f);
          }
          wm::warp_net(sW, lane, i0, i1, yo0, yo1);
        }
        // the next row's loads, in flight during this row's polish and relaxation
        if (act && y + 1 < y1) offn = gather_dev(fin, plane, P, x, y + 1, xin, gn);
        if (act) {
          int fb = 0;
          float J4;
          if (use) {
            J4 = j4_polish_f(x_from_outputs(yo0, yo1), m.delta, L, &fb);
          } else {
            float xx;
            J4 = j4_from_delta_f(m.delta, L, &xx);
          }
          nfb += (unsigned)fb;
          nev += use ? 1u : 0u;
          relax_store_dev<T, STAT_FD>(P, g, m, 1.5f - m.delta, J4, fout, plane, off);
        }
      }
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
  flush_counts(nfb, nev, counters);
}

}  // namespace lbm
