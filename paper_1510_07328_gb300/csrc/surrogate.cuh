// Learned Fermi-Dirac inversion: a 2 -> 64 -> 64 -> 2 network with SiLU
// activations that maps a cell's density and internal energy (n, e) to its
// temperature and chemical potential (T, mu).  It stands in for the
// per-cell inversion of the FD moment ratio J_2(x), x = mu/T (the FD form of
// I_2N, Sect. "Generalized polynomials in D dimensions"); the paper itself
// has no network.
//
// Model (the interface the header documents; training and inference share it):
//   inputs    (n, e), e = D n J_2/3 (D = 2): the internal energy in lattice
//             units; fixed embedding n_hat = (n - 1.25)/0.75 and
//             l_hat = (ln delta + 5.3)/3.7, delta = 3/2 - 3 e/(2 n) = 3/2 - J_2
//   layers    h1 = silu(W1 x + b1), h2 = silu(W2 h1 + b2), y = W3 h2 + b3
//   outputs   ln T = 0.5 y_0 - 5.09, mu = 0.12 y_1 + 0.1985
//   params    W1 [64][2], b1 [64], W2 [64][64], b2 [64], W3 [2][64], b3 [2]
#pragma once
#include <cuda_runtime.h>

namespace lbm {

constexpr int kH = 64;
constexpr int kNParam = kH * 2 + kH + kH * kH + kH + 2 * kH + 2;  // 4482

constexpr float kSurNMid = 1.25f, kSurNHalf = 0.75f;
constexpr float kSurLdMid = -5.3f, kSurLdHalf = 3.7f;
constexpr float kSurLnTMid = -5.09f, kSurLnTHalf = 0.5f;
constexpr float kSurMuMid = 0.1985f, kSurMuHalf = 0.12f;

// The network's domain: the ranges of its training set, n in [0.5, 2] and
// t = T/T_F in [0.005, 0.3], the latter as delta = 3/2 - J_2 in
// [delta(t = 0.3), delta(t = 0.005)] (D = 2, values of the exact forward map
// t -> x -> J_2).  Only cells inside it go through the network; the others
// take the exact inversion (an extrapolating network would fail the residual
// check there anyway).
constexpr float kSurNLo = 0.5f, kSurNHi = 2.0f;
constexpr float kSurDeltaLo = 1.2332948e-4f, kSurDeltaHi = 0.19829931f;

// Offsets into the flat parameter vector.
constexpr int kOW1 = 0, kOB1 = kOW1 + 2 * kH, kOW2 = kOB1 + kH, kOB2 = kOW2 + kH * kH, kOW3 = kOB2 + kH,
              kOB3 = kOW3 + 2 * kH;

// Network weights by value: passed as a kernel parameter (17.9 KB, within the
// 32 KB parameter limit) so that every weight read is a warp-uniform
// constant-bank operand.  Loops over it are fully unrolled.
struct MlpParams {
  float p[kNParam];
};

// The network as FP16 tensor-core B operands (N x K, canonical K-major
// layout without swizzle: element (r, k) of an R-row operand at byte
// ((k/8)(R/8) + r/8) 128 + (r%8) 16 + (k%8) 2), one buffer, byte offsets:
//   kTcB1   64 x 16  layer 1: unit j holds (w_n hi, w_n hi, w_n lo, w_l hi,
//                    w_l hi, w_l lo, b hi, b lo, 0 ...) of W1/2, b1/2, against
//                    the input row (n hi, n lo, n hi, l hi, l lo, l hi, 1, 1,
//                    0 ...), so the products carry the inputs and weights to
//                    about 2^-22
//   kTcB2   64 x 64  W2/2
//   kTcB2b  64 x 16  b2/2 (hi, lo) in columns 6, 7 (against the input row)
//   kTcB3   16 x 64  W3 rows 0, 1 (hi) and 2, 3 (lo); rows 4..15 zero
//   kTcB3b  16 x 16  b3 (hi, lo) in columns 6, 7 of rows 0, 1
// The halving makes layers 1 and 2 produce z/2, the argument of
// silu(z) = (z/2)(1 + tanh(z/2)).
constexpr int kTcB1 = 0, kTcB2 = kTcB1 + kH * 16 * 2, kTcB2b = kTcB2 + kH * kH * 2, kTcB3 = kTcB2b + kH * 16 * 2,
              kTcB3b = kTcB3 + 16 * kH * 2, kTcBytes = kTcB3b + 16 * 16 * 2;  // 14848

__host__ __device__ constexpr int tc_operand_byte(int r, int k, int R) {
  return ((k / 8) * (R / 8) + r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2;
}

// The network as warp-level MMA fragments (mma.sync m16n8k8 / m16n8k16, FP16
// operands; FP16 accumulators for layers 1 and 2, FP32 for layer 3), one
// buffer in the order the lanes read it.
// Lane l has group g = l/4 and index t = l%4; a B fragment of an 8-column
// n-tile holds element (k, n = g) for k = 2t, 2t+1 (and 2t+8, 2t+9 when
// K = 16), packed low element first.  Byte offsets:
//   kMmB1  [p 0..3][lane] 2 x u32  layer 1 (K = 8), n-tiles 2p and 2p+1: the
//                                  8-feature rows of kTcB1 (W1/2, b1/2 hi/lo)
//   kMmB2  [c 0..3][p 0..3][lane] 4 x u32  layer 2 (K = 16 chunk c), n-tiles
//                                  2p and 2p+1 of W2/2 (element (k, n) =
//                                  W2[n][k]/2)
//   kMmC2  [p 0..3][t] 2 x u32     b2/2 for columns 8 nt + 2t, 8 nt + 2t + 1
//                                  as FP16 pairs, nt = 2p then 2p + 1 (the
//                                  FP16 accumulators' initial values)
//   kMmB3  [c 0..3][lane] 4 x u32  layer 3, K = 16 chunk c: the fragment of
//                                  W3 hi, then of W3 lo (columns 0, 1; the
//                                  other six zero); both accumulate into the
//                                  same two columns
//   kMmC3  2 x f32                 b3
// The halving makes layers 1 and 2 produce z/2, as for the tcgen05 operands.
constexpr int kMmB1 = 0, kMmB2 = kMmB1 + 4 * 32 * 8, kMmC2 = kMmB2 + 16 * 32 * 16, kMmB3 = kMmC2 + 4 * 4 * 8,
              kMmC3 = kMmB3 + 4 * 32 * 16, kMmBytes = kMmC3 + 16;  // 11408

__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// Network output (y_0, y_1) for one cell given n and delta = 3/2 - J_2
// (= 3/2 - 3 e/(2 n)); W lives in parameter space.
__device__ __forceinline__ void mlp_forward_f(const MlpParams& W, float n, float delta, float& y0, float& y1) {
  const float x0 = (n - kSurNMid) * (1.0f / kSurNHalf);
  const float x1 = (__logf(delta) - kSurLdMid) * (1.0f / kSurLdHalf);
  float h1[kH];
#pragma unroll
  for (int k = 0; k < kH; ++k) {
    const float z = fmaf(W.p[kOW1 + 2 * k], x0, fmaf(W.p[kOW1 + 2 * k + 1], x1, W.p[kOB1 + k]));
    h1[k] = silu_f(z);
  }
  float a0 = W.p[kOB3], a1 = W.p[kOB3 + 1];
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    float z = W.p[kOB2 + j];
#pragma unroll
    for (int k = 0; k < kH; ++k) z = fmaf(W.p[kOW2 + kH * j + k], h1[k], z);
    const float h = silu_f(z);
    a0 = fmaf(W.p[kOW3 + j], h, a0);
    a1 = fmaf(W.p[kOW3 + kH + j], h, a1);
  }
  y0 = a0;
  y1 = a1;
}

__device__ __forceinline__ void mlp_outputs_to_state(float y0, float y1, float& T, float& mu) {
  T = __expf(fmaf(kSurLnTHalf, y0, kSurLnTMid));
  mu = fmaf(kSurMuHalf, y1, kSurMuMid);
}

}  // namespace lbm
