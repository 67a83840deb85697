// Minimal tcgen05 (5th-generation tensor core) helpers for sm_100-family
// GPUs: TMEM allocation, shared-memory matrix descriptors for the canonical
// K-major layout without swizzle, the f16-kind MMA with an FP32 or FP16
// accumulator in TMEM, commit to an mbarrier, bounded waits, TMEM loads, and
// the packed FP16 SiLU both tensor-core engines use.
//
// Canonical K-major layout (no swizzle): an R x K operand of 16-bit elements
// is cut into core matrices of 8 rows x 8 elements (8 rows of 16 bytes, 128
// contiguous bytes).  Core (r/8, k/8) sits at ((k/8) * (R/8) + r/8) * 128
// bytes, so neighbouring cores are 128 bytes apart along R (the descriptor's
// stride byte offset) and R/8 * 128 bytes apart along K (its leading byte
// offset).  One MMA consumes K = 16: two core columns.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) of an R x K operand in the canonical layout.
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int R) {
  return (uint32_t)(((k >> 3) * (R >> 3) + (r >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// 64-bit shared-memory matrix descriptor: start address, leading byte offset
// (K direction), stride byte offset (R direction), all >> 4; version 1 (bit
// 46); base offset 0; no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16 with FP16 A and B (both K-major) and an
// FP32 accumulator: D format at bit 4, N/8 at bit 17, M/16 at bit 24.
__host__ __device__ constexpr uint32_t idesc_f16_f32(uint32_t M, uint32_t N) {
  return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// The same with an FP16 accumulator (D format 0).
__host__ __device__ constexpr uint32_t idesc_f16_f16(uint32_t M, uint32_t N) {
  return ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {  // one full warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // one full warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// D (+)= A * B^T for one K = 16 slice; accumulate != 0 adds to D.
__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// The mbarrier completes once every prior tcgen05 operation of this thread has.
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// Wait for the given phase parity, at most `limit` polls; true if completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
  uint32_t done = 0;
  for (int it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// 64 consecutive 16-bit columns of this thread's TMEM lane (an FP16
// accumulator), packed in pairs: r[i] holds columns 2i (low half) and 2i + 1
// (the .x32 repetition count counts the 32-bit registers written).
__device__ __forceinline__ void tmem_ld64_pack16(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.pack::16b.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%"
      "28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 consecutive 16-bit columns of this thread's TMEM lane, packed in pairs
// as tmem_ld64_pack16 (half the registers live at a time).
__device__ __forceinline__ void tmem_ld32_pack16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.pack::16b.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 4 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = __uint_as_float(r[c]);
}

// SiLU of a packed FP16 pair of halved arguments h = z/2: h + h tanh(h).
__device__ __forceinline__ uint32_t silu2_packed(uint32_t h) {
  uint32_t t;
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(h));
  const __half2 hv = *reinterpret_cast<const __half2*>(&h), tv = *reinterpret_cast<const __half2*>(&t);
  const __half2 s = __hfma2(hv, tv, hv);
  return *reinterpret_cast<const uint32_t*>(&s);
}

// SiLU of a packed FP16 pair of halved arguments h = z/2 on the FMA pipe:
//   silu(z) = relu(z) + q(|h|),  q(s) = s tanh(s) - s,
// with q by its degree-6 minimax polynomial in t = min(|h|, 4.5) (2/4.5) - 1
// (Lawson's algorithm; fit_silu_poly.py prints the coefficients), evaluated
// by Horner's rule in packed FP16.  Error within 3.6e-3 of max(1, |silu(z)|)
// (the MUFU path: 1.1e-3), including the clamp's tail |q(4.5)| = 1.1e-3.
// Constants: FP16 bit patterns, the same value in both halves.
constexpr uint32_t kSiluClamp = 0x44804480u, kSiluScale = 0x371C371Cu, kSiluMinus1 = 0xBC00BC00u,
                   kSiluTwo = 0x40004000u;
// coefficients of t^6 .. t^0
constexpr uint32_t kSiluC6 = 0x31AD31ADu, kSiluC5 = 0xB747B747u, kSiluC4 = 0x32383238u, kSiluC3 = 0x349D349Du,
                   kSiluC2 = 0xB534B534u, kSiluC1 = 0x313A313Au, kSiluC0 = 0xAA04AA04u;

__device__ __forceinline__ __half2 h2bits(uint32_t b) { return *reinterpret_cast<const __half2*>(&b); }

__device__ __forceinline__ uint32_t silu2_poly(uint32_t hu) {
  const __half2 h = h2bits(hu);
  const __half2 s = __hmin2(__habs2(h), h2bits(kSiluClamp));
  const __half2 t = __hfma2(s, h2bits(kSiluScale), h2bits(kSiluMinus1));
  __half2 p = __hfma2(h2bits(kSiluC6), t, h2bits(kSiluC5));
  p = __hfma2(p, t, h2bits(kSiluC4));
  p = __hfma2(p, t, h2bits(kSiluC3));
  p = __hfma2(p, t, h2bits(kSiluC2));
  p = __hfma2(p, t, h2bits(kSiluC1));
  p = __hfma2(p, t, h2bits(kSiluC0));
  const __half2 o = __hfma2(__hmax2(h, h2bits(0u)), h2bits(kSiluTwo), p);
  return *reinterpret_cast<const uint32_t*>(&o);
}

}  // namespace tc
}  // namespace lbm
