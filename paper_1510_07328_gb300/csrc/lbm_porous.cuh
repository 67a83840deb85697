// The d2v9 step with rigid obstacles and a constant body force (the paper's
// porous-medium experiment, Sect. "Numerical simulations for electrons in
// metals").  Obstacles: a fluid cell whose pull source is solid (or beyond a
// wall) takes the opposite population of its own cell (halfway bounce-back);
// solid cells are not updated.  Force: exact difference method (Kupershtokh,
// Medvedev and Karpov 2009): after BGK every fluid cell receives
// f_eq(n, u_0 + F/n) - f_eq(n, u_0) on the same moments (same J_2, J_4), which
// adds exactly F of momentum and no mass.
#pragma once
#include "lbm_dev32.cuh"

namespace lbm {

__device__ __forceinline__ bool is_solid(const ProbDev& P, int64_t c) { return P.solid != nullptr && P.solid[c] != 0; }

// Pull of the nine populations of cell (x, y) with obstacles.
template <class T>
__device__ __forceinline__ void pull9_obst(const T* __restrict__ fin, int64_t plane, const ProbDev& P, int x, int y,
                                           T v[9]) {
  const PullIdx q = pull_index(P, x, y);
  auto ld = [&](int a, int64_t r, int xs, int opp) -> T {
    return (r < 0 || xs < 0 || is_solid(P, r + xs)) ? fin[opp * plane + q.row + x] : fin[a * plane + r + xs];
  };
  v[0] = fin[q.row + x];
  v[1] = ld(1, q.row, q.xm, 3);
  v[2] = ld(2, q.rm, x, 4);
  v[3] = ld(3, q.row, q.xp, 1);
  v[4] = ld(4, q.rp, x, 2);
  v[5] = ld(5, q.rm, q.xm, 7);
  v[6] = ld(6, q.rm, q.xp, 8);
  v[7] = ld(7, q.rp, q.xp, 5);
  v[8] = ld(8, q.rp, q.xm, 6);
}

// Pull code of one cell, for the FP32 / BF16 step with obstacles: bit a
// (a = 1..8) is set when the pull source x - e_a of population a is solid or
// beyond a wall, so that the population is the opposite one of the cell
// itself (halfway bounce-back, the rule of pull9_obst); bit 0 when the cell
// is solid.  Computed once per lbm_set_obstacles, 2 bytes per cell.
__global__ void pull_code_kernel(ProbDev P, uint16_t* __restrict__ code) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)P.nx * P.ny) return;
  const int y = (int)(i / P.nx), x = (int)(i % P.nx);
  const PullIdx q = pull_index(P, x, y);
  auto bad = [&](int64_t r, int xs) -> unsigned { return (r < 0 || xs < 0 || P.solid[r + xs] != 0) ? 1u : 0u; };
  unsigned c = P.solid[q.row + x] != 0 ? 1u : 0u;
  c |= bad(q.row, q.xm) << 1 | bad(q.rm, x) << 2 | bad(q.row, q.xp) << 3 | bad(q.rp, x) << 4;
  c |= bad(q.rm, q.xm) << 5 | bad(q.rm, q.xp) << 6 | bad(q.rp, q.xp) << 7 | bad(q.rp, q.xm) << 8;
  code[q.row + x] = (uint16_t)c;
}

// Pulled deviations of cell (x, y) through its pull code: every population's
// address is chosen (neighbour or own opposite) before its single load, so
// the pull has no branch and no mask scan.  `interior`: the row and its tile
// have every neighbour on the lattice without wrapping (the offsets are then
// constants); otherwise the wrapped offsets of pull_index32, whose
// off-lattice entries are never used (their code bits are set).
template <class T>
__device__ __forceinline__ void gather_code(const T* __restrict__ fin, int64_t plane, const ProbDev& P, int x, int y,
                                            bool interior, unsigned code, float g[9]) {
  const int pt = P.pitch, off = (int)P.base + y * pt + x;
  int s[9];
  if (interior) {
    s[1] = off - 1; s[2] = off - pt; s[3] = off + 1; s[4] = off + pt;
    s[5] = off - pt - 1; s[6] = off - pt + 1; s[7] = off + pt + 1; s[8] = off + pt - 1;
  } else {
    const PullIdx32 q = pull_index32(P, x, y);
    s[1] = q.row + q.xm; s[2] = q.rm + x; s[3] = q.row + q.xp; s[4] = q.rp + x;
    s[5] = q.rm + q.xm; s[6] = q.rm + q.xp; s[7] = q.rp + q.xp; s[8] = q.rp + q.xm;
  }
  constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
  g[0] = Dev<T>::ld(fin[off]);
#pragma unroll
  for (int a = 1; a < 9; ++a) {
    const int64_t idx = ((code >> a) & 1u) ? (int64_t)opp[a] * plane + off : (int64_t)a * plane + s[a];
    g[a] = Dev<T>::ld(fin[idx]);
  }
}

// FP64: BGK on f_eq(n, u) plus f_eq(n, u + F/n) - f_eq(n, u).
template <int STAT>
__device__ __forceinline__ void collide_force_f64(const ProbDev& P, const double f[9], double* __restrict__ fout,
                                                  int64_t plane, int64_t c, const InvLimits& L, const InvLimitsF& Lf) {
  const double n = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
  const double jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
  const double jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
  const double E = ((f[1] + f[2]) + (f[3] + f[4])) + 2.0 * ((f[5] + f[6]) + (f[7] + f[8]));
  const double in = 1.0 / n;
  const double ux = jx * in, uy = jy * in;
  double J2, J4;
  if (STAT == STAT_FD) {
    J2 = 1.5 * (E * in - (ux * ux + uy * uy));
    int cl;
    double xx;
    J4 = j4_fp64(J2, L, Lf, &xx, &cl);
  } else {
    J2 = FixedJ<STAT>::j2;
    J4 = FixedJ<STAT>::j4;
  }
  double fe[9], ff[9];
  feq_f64(n, ux, uy, J2, J4, fe);
  feq_f64(n, ux + P.fx * in, uy + P.fy * in, J2, J4, ff);
  const double w = P.omega;
#pragma unroll
  for (int a = 0; a < 9; ++a) fout[a * plane + c] = fma(w, fe[a] - f[a], f[a]) + (ff[a] - fe[a]);
}

// FP32 deviations: BGK as in relax_store_dev plus the force term, whose
// difference S(u + d) - S(u) (d = F/n) is expanded exactly, so that a small
// force loses no precision to cancellation.  With p = e.u, q = e.d,
// s = |u|^2, r = 2 u.d + |d|^2 and the class constants of the bracket
// (Q = q_c s, C = c_0 + c_1 s, A = a_1 + b_0 C):
//   S(+-e)(u + d) - S(+-e)(u) = even +- odd,
//   even = q_c r + a_2 q (2 p + q),
//   odd  = q (A + b_0 c_1 r) + b_0 c_1 p r + b_0 k_4 q (p'^2 + p' p + p^2),  p' = p + q;
// the rest population gets q_rest r.
template <class T, int STAT>
__device__ __forceinline__ void relax_force_store_dev(const ProbDev& P, const float g[9], const CellMom& m, float J2,
                                                      float J4, T* __restrict__ fout, int64_t plane, int off) {
  const float dn = m.dn, X = m.X, ux = m.ux, uy = m.uy, u2 = m.u2;
  float dW0, dWs, dWl;
  if (STAT == STAT_FD) {
    dW0 = dn * (1.0f / 6.0f) + (5.0f / 6.0f) * X;
    dWs = (dn - X) * (1.0f / 6.0f);
    dWl = 0.25f * dWs;
  } else {
    dW0 = dn * (1.0f - 5.0f * J2 / 9.0f);
    dWs = dn * J2 / 9.0f;
    dWl = dn * J2 / 36.0f;
  }
  const float W0 = P.f.wref[0] + dW0, Ws = P.f.wref[1] + dWs, Wl = P.f.wref[2] + dWl;
  const float D22 = delta22_f(J2);  // NaN outside 0 < J_2 < 2
  const float D42 = __fdividef(1.0f, 3.0f - 2.0f * J4);
  const float iJ2 = __fdividef(1.0f, J2);
  const float t = J4 * D42, Pt = (1.0f - J2) * t;
  const float b0 = 1.5f * iJ2;
  const float c1s = -fmaf(0.75f, t, 2.25f * J4), c1l = fmaf(1.5f, t, -4.5f * J4);
  const float A1 = iJ2 * fmaf(-fmaf(1.125f, t, 3.375f * J4), u2, fmaf(1.5f, Pt, 3.0f));
  const float A2 = iJ2 * fmaf(fmaf(2.25f, t, -6.75f * J4), u2, fmaf(-3.0f, Pt, 3.0f));
  const float bk = 4.5f * J4 * iJ2, a2 = 4.5f * iJ2;
  const float h = 1.5f * D22, r = (D22 - 1.0f) * iJ2;
  const float q0 = -h, q1 = fmaf(2.25f, r, -h), q2 = fmaf(4.5f, r, -h);
  const float w = P.f.omega;
  // force: d = F/n, rr = 2 u.d + |d|^2
  const float dx = P.f.fx * m.in, dy = P.f.fy * m.in;
  const float rr = fmaf(2.0f, fmaf(ux, dx, uy * dy), fmaf(dx, dx, dy * dy));
  // each population is stored as soon as its equilibrium and force parts
  // are formed (no arrays of nine live across the cell)
  auto put = [&](int a, float ge, float gf) { fout[a * plane + off] = Dev<T>::st(fmaf(w, ge - g[a], g[a]) + gf); };
  put(0, fmaf(W0, q0 * u2, dW0), W0 * (q0 * rr));
  auto pair = [&](float eu, float ed, float A, float qc, float c1, float W, float dW, int ap, int am) {
    const float e2 = eu * eu;
    const float base = fmaf(W, fmaf(a2, e2, qc * u2), dW);
    const float wo = W * (eu * fmaf(bk, e2, A));
    const float pp = eu + ed;
    const float bc1 = b0 * c1;
    const float even = fmaf(qc, rr, a2 * ed * fmaf(2.0f, eu, ed));
    const float odd = fmaf(ed, fmaf(bc1, rr, A), fmaf(bc1 * eu, rr, bk * ed * fmaf(pp, pp + eu, e2)));
    put(ap, base + wo, W * (even + odd));
    put(am, base - wo, W * (even - odd));
  };
  pair(ux, dx, A1, q1, c1s, Ws, dWs, 1, 3);
  pair(uy, dy, A1, q1, c1s, Ws, dWs, 2, 4);
  pair(ux + uy, dx + dy, A2, q2, c1l, Wl, dWl, 5, 7);
  pair(ux - uy, dx - dy, A2, q2, c1l, Wl, dWl, 8, 6);
}

// True when the tile (kTileX cells from x0, rows y0 .. y1 - 1) and its halo of
// one cell hold no solid cell; every thread of the CTA takes part.  Each
// thread scans its column over rows y0 - 1 .. y1, the first and last thread
// also the halo columns left of the first cell and right of the last one
// (wrapped where periodic).
__device__ __forceinline__ bool tile_clean(const ProbDev& P, int x0, int y0, int y1) {
  unsigned any = 0;  // OR of the mask bytes: independent loads, no short circuit
  if (P.solid != nullptr) {
    const int t = (int)threadIdx.x;
    auto col = [&](int x) {
      if (x < 0 || x >= P.nx) {
        if (P.bc_x != BC_PERIODIC) return;
        x = (x + P.nx) % P.nx;
      }
      for (int y = y0 - 1; y <= y1; ++y) {
        int yy = y;
        if (yy < 0 || yy >= P.ny) {
          if (P.bc_y != BC_PERIODIC) continue;
          yy = (yy + P.ny) % P.ny;
        }
        any |= P.solid[P.base + (int64_t)yy * P.pitch + x];
      }
    };
    if (x0 + t < P.nx) col(x0 + t);
    if (t == 0) col(x0 - 1);
    if (t == kTileX - 1) col(min(x0 + kTileX, P.nx));  // right of the tile's last cell
  }
  return __syncthreads_or(any != 0) == 0;
}

// One CTA per tile of 128 cells x TY rows (PERSIST: a smaller grid walks the
// tiles).  T = double: FP64 populations; tiles without solid cells in reach
// take the pull without mask checks.  float / bf16: deviations, every cell
// pulled through its pull code (gather_code; a problem without obstacles has
// none and pulls plainly), with the next row's loads issued before the
// current row's collision, except for BF16 under the fixed closures, which
// loads one row at a time and spends the registers on resident warps.
// Resident CTAs per SM (measured on the 4096^2 porous lattice, MB closure
// with the force): FP32 nine (71.4 GLUPS against 68.8 at eight), BF16 ten
// without the prefetch (79.1 against 69.3 at eight with it); FD six.
template <class T, int STAT>
__host__ __device__ constexpr int porous_ctas() {
  return sizeof(T) == 8 ? 4 : (STAT == STAT_FD ? 6 : (sizeof(T) == 2 ? 10 : 9));
}
template <class T, int STAT, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX, (porous_ctas<T, STAT>())) stream_collide_porous(const T* __restrict__ fin, T* __restrict__ fout,
                                                                const ProbDev* __restrict__ probs, int nprob,
                                                                int ntiles, int64_t plane, InvLimits L,
                                                                InvLimitsF Lf) {
  int tile = (int)blockIdx.x;
#pragma unroll 1
  do {
    const int p = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
    const ProbDev& P = probs[p];
    const int lt = tile - (int)P.tile_begin;
    const int ty = lt / P.tiles_x;
    const int x0 = (lt - ty * P.tiles_x) * kTileX;
    const int x = x0 + (int)threadIdx.x;
    const int y0 = ty * TY, y1 = min(y0 + TY, P.ny);
    const bool xin = x0 >= 1 && x0 + kTileX <= P.nx - 1;
    if constexpr (Stor<T>::dev) {
      if (x < P.nx) {
        // pulled deviations of row y into g; false for a solid cell
        auto load = [&](int y, float g[9]) -> bool {
          if (P.pcode == nullptr) {  // no obstacles: the plain pull (walls included)
            gather_dev(fin, plane, P, x, y, xin, g);
            return true;
          }
          const unsigned code = P.pcode[(int)P.base + y * P.pitch + x];
          gather_code(fin, plane, P, x, y, xin && y >= 1 && y <= P.ny - 2, code, g);
          return (code & 1u) == 0u;
        };
        // collision of a fluid cell of row y from its pulled deviations
        auto collide = [&](int y, const float g[9]) {
          const CellMom m = dev_moments(P, g);
          float J2, J4;
          if (STAT == STAT_FD) {
            J2 = 1.5f - m.delta;
            float xx;
            J4 = j4_from_delta_f(m.delta, Lf, &xx);
          } else {
            J2 = (float)FixedJ<STAT>::j2;
            J4 = (float)FixedJ<STAT>::j4;
          }
          relax_force_store_dev<T, STAT>(P, g, m, J2, J4, fout, plane, (int)(P.base + (int64_t)y * P.pitch + x));
        };
        if constexpr (sizeof(T) == 2 && STAT != STAT_FD) {
#pragma unroll 1
          for (int y = y0; y < y1; ++y) {
            float g[9];
            if (load(y, g)) collide(y, g);
          }
        } else {
          // the next row's loads are issued before the current row's collision
          float gn[9];
          bool fn = load(y0, gn);
#pragma unroll 1
          for (int y = y0; y < y1; ++y) {
            float g[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) g[a] = gn[a];
            const bool fluid = fn;
            if (y + 1 < y1) fn = load(y + 1, gn);
            if (fluid) collide(y, g);
          }
        }
      }
    } else {
      const bool clean = tile_clean(P, x0, y0, y1);
      if (x < P.nx) {
#pragma unroll 1
        for (int y = y0; y < y1; ++y) {
          const int64_t c = P.base + (int64_t)y * P.pitch + x;
          if (!clean && is_solid(P, c)) continue;
          T v[9];
          if (clean) pull9(fin, plane, pull_index(P, x, y), x, v);
          else pull9_obst(fin, plane, P, x, y, v);
          collide_force_f64<STAT>(P, v, fout, plane, c, L, Lf);
        }
      }
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
}

}  // namespace lbm
