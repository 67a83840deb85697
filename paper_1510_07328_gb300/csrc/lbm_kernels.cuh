// Kernels of the d2v9 generalized-polynomial LBGK step (sm_103a).
//
// Layout in HBM: structure of arrays, one plane per velocity a = 0..8 of
// `plane` cells; problem p occupies cells [base_p, base_p + ny_p * pitch_p)
// of every plane, row-major with a row pitch rounded up to 32 cells.  Two
// such buffers alternate (read A, write B).  Velocity order: rest; (1,0),
// (0,1), (-1,0), (0,-1); (1,1), (-1,1), (-1,-1), (1,-1).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fd_device.cuh"
#include "fd_device_f32.cuh"

namespace lbm {

// FD: J_2 from the energy moment, x by inversion; T0: theta = 0 constants;
// MB: Hermite limit; FT: theta fixed per problem, x from the density alone.
enum { STAT_FD = 0, STAT_T0 = 1, STAT_MB = 2, STAT_FT = 3 };
enum { BC_PERIODIC = 0, BC_BOUNCEBACK = 1 };

constexpr int kTileX = 128;      // cells of one row handled by one CTA (one per thread)
constexpr int kTileYDefault = 4; // rows per tile (each thread walks them); tunable: 1, 2, 4, 8

struct ProbDev {
  int32_t nx, ny, pitch, bc_x, bc_y, tiles_x;  // tiles: kTileX cells x (rows per tile) rows
  int64_t base, tile_begin;
  double tau, omega;
  double n_ref, t_ref;               // deviation reference state (n_ref = 0: absolute storage)
  double j2_ref, ndelta_ref;         // J_2(t_ref), n_ref (3/2 - J_2(t_ref))
  double wref[9];                    // W_a^ref = w_a(J_2(t_ref)) n_ref
  double nsum_ref, esum_ref;         // sum W^ref and sum W^ref |e|^2 (the deviations' offsets)
  double theta;                      // fixed-theta closure: theta = n_ref t_ref/(2 pi) of the problem
  struct {
    float omega, n_ref, ndelta_ref;
    float wref[3];  // rest, short, long
    float fx, fy;
    float two_pi_theta;  // 2 pi theta (fixed-theta closure)
  } f;              // FP32 copies for the reduced-precision step
  const uint8_t* solid;              // obstacle mask indexed like the cells (nonzero: solid), or null
  const uint16_t* pcode;             // pull code of each cell (lbm_porous.cuh), set with solid, or null
  double fx, fy;                     // constant body force per cell and step
};

// Closure constants of the statistics without inversion.
template <int STAT>
struct FixedJ {
  static constexpr double j2 = STAT == STAT_T0 ? 1.5 : 1.0;  // 1 + 2/(2 + D) | 1
  static constexpr double j4 = STAT == STAT_T0 ? 4.0 / 3.0 : 1.0;
};

// Delta_2^2 = 2/((D+2) - J_2 D) = 1/(2 - J_2) for D = 2 (definitions under
// Eq. (H4)).  The polynomials need Delta_2 = +sqrt(Delta_2^2) real and the
// lattice scale c_0^2 = 3 I_4/I_2 = 3 I_2/(I_0 J_2) positive, so the K = 3
// equilibrium exists for 0 < J_2 < 2 only.  Outside (reachable only through
// measured moments) there is no equilibrium: NaN is returned, and every
// population of the cell becomes NaN (counted as non-finite by lbm_moments).
__device__ __forceinline__ double delta22(double J2) {
  return (J2 > 0.0 && J2 < 2.0) ? 1.0 / (2.0 - J2) : __longlong_as_double(0x7ff8000000000000ll);
}
__device__ __forceinline__ float delta22_f(float J2) {
  return (J2 > 0.0f && J2 < 2.0f) ? __fdividef(1.0f, 2.0f - J2) : __int_as_float(0x7fc00000);
}

// Locate the problem and the (row, x-tile) of this CTA.
__device__ __forceinline__ int find_problem(const ProbDev* __restrict__ probs, int nprob, int64_t tile) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].tile_begin <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// K = 3 equilibrium in geometric velocities (Sect. "The Gaussian quadrature",
// D = 2), FP64.  W_0 = n(1 - 5J_2/9), W_short = nJ_2/9, W_long = nJ_2/36.
__device__ __forceinline__ void feq_f64(double n, double ux, double uy, double J2, double J4, double fe[9]) {
  const double u2 = ux * ux + uy * uy;
  const double D22 = delta22(J2);             // 2/((D+2) - J_2 D), NaN outside 0 < J_2 < 2
  const double D42 = 1.0 / (3.0 - 2.0 * J4);  // 2/((D+4) - J_4 (D+2))
  const double iJ2 = 1.0 / J2;
  const double a1 = 3.0 * iJ2, a2 = 4.5 * iJ2, b0 = 1.5 * iJ2;
  const double a3 = 2.25 * (D22 - 1.0) * iJ2;  // (9/2)(D22-1)/(J2 D)
  const double a4 = 1.5 * D22;
  const double k0 = 4.0 * (1.0 - J2) * J4 * D42;  // (1-J2) J4 (D+2) D42
  const double k1 = 3.0 * (1.0 - J2) * J4 * D42;
  const double k2 = 3.0 * J4 * D42;
  const double k3 = 2.25 * J4 * (D42 - 1.0);  // 9 J4 (D42-1)/(D+2)
  const double k4 = 3.0 * J4;
  const double W0 = n * (1.0 - 5.0 * J2 / 9.0), Ws = n * J2 / 9.0, Wl = n * J2 / 36.0;
  // class constants: e2 = 0 (rest), 1 (short), 2 (long)
  const double C1 = k0 - k1 + (k3 - k2) * u2, C2 = k0 - 2.0 * k1 + (2.0 * k3 - k2) * u2;
  const double Q0 = -a4 * u2, Q1 = (a3 - a4) * u2, Q2 = (2.0 * a3 - a4) * u2;
  auto S = [&](double eu, double C, double Qc) {
    return 1.0 + Qc + eu * (a1 + a2 * eu + b0 * (C + k4 * eu * eu));
  };
  fe[0] = W0 * (1.0 + Q0);
  fe[1] = Ws * S(ux, C1, Q1);
  fe[2] = Ws * S(uy, C1, Q1);
  fe[3] = Ws * S(-ux, C1, Q1);
  fe[4] = Ws * S(-uy, C1, Q1);
  fe[5] = Wl * S(ux + uy, C2, Q2);
  fe[6] = Wl * S(-ux + uy, C2, Q2);
  fe[7] = Wl * S(-ux - uy, C2, Q2);
  fe[8] = Wl * S(ux - uy, C2, Q2);
}

// J_2, J_4 of a state given by t (FD) or by the closure.
template <int STAT>
__device__ __forceinline__ void closure_from_t(double t, double& J2, double& J4) {
  if (STAT == STAT_FD || STAT == STAT_FT) {
    const FD5 f = fd_eval(x_of_t(t));
    J2 = j2_of(f);
    J4 = j4_of(f);
  } else {
    J2 = FixedJ<STAT>::j2;
    J4 = FixedJ<STAT>::j4;
  }
}

// J_4 in the degenerate regime, FP64, from s = x^2 (tails below 4.3e-18 for
// x >= 40): J_4 = 60 s (s + pi^2)^2 / ((3 s + pi^2)(15 s^2 + 30 pi^2 s + 7 pi^4)).
__device__ __forceinline__ double j4_degenerate(double s) {
  const double sp = s + kPi2;
  return 60.0 * s * sp * sp / ((3.0 * s + kPi2) * (15.0 * s * s + 30.0 * kPi2 * s + 7.0 * kPi2 * kPi2));
}

// The FP64 step's inversion: J_4 (and x) for a measured J_2.
//  * clamp interval, NaN and the degenerate regime x >= 40 (exact quadratic
//    root, closed-form J_4) as in invert_j2;
//  * otherwise the FP32 inversion gives x_f (about 1e-6 relative); at x_f one
//    FP64 evaluation of f_0..f_4 gives the Newton step dx = (J_2 - J_2(x_f))/
//    J_2'(x_f) and J_4 = J_4(x_f) + J_4'(x_f) dx, whose second-order remainder
//    J_4'' dx^2/2 is below 1e-13; the step repeats (at most 4 evaluations)
//    while |dx| > 1e-6 |x|.
__device__ __forceinline__ double j4_fp64(double J2, const InvLimits& L, const InvLimitsF& Lf, double* xout,
                                          int* clamped) {
  *clamped = 0;
  if (!(J2 == J2) || isinf(J2)) {
    *xout = J2 - J2;
    return *xout;
  }
  if (J2 >= L.j2_hi || J2 <= L.j2_lo) {
    *clamped = 1;
    const double x = J2 >= L.j2_hi ? L.x_hi : L.x_lo;
    *xout = x;
    return j4_of(fd_eval(x));
  }
  const double delta = 1.5 - J2;
  if (delta < 0.1) {
    const double A = 6.0 * delta, B = 3.0 * kPi2 - 6.0 * delta * kPi2, C = kPi2 * kPi2;
    const double sq = (B + sqrt(fmax(B * B - 4.0 * A * C, 0.0))) / (2.0 * A);
    if (sq >= kXDeg * kXDeg) {
      *xout = fmin(sqrt(sq), L.x_hi);
      return j4_degenerate(*xout * *xout);
    }
  }
  float xf;
  j4_from_delta_f((float)delta, Lf, &xf);
  double x = (double)xf;
  double J4 = 0.0;
#pragma unroll 1
  for (int it = 0; it < 4; ++it) {
    const FD5 f = fd_eval(x);
    const double i1 = 1.0 / f.f1, i2 = 1.0 / f.f2, i3 = 1.0 / f.f3, i4 = 1.0 / f.f4;
    const double j = f.f2 * f.f2 * i1 * i3;
    const double dj = j * (2.0 * f.f1 * i2 - f.f0 * i1 - f.f2 * i3);
    const double dx = (J2 - j) / dj;
    J4 = f.f3 * f.f3 * i2 * i4;
    if (fabs(dx) <= 1e-6 * fabs(x) || it == 3) {
      const double dJ4 = J4 * (2.0 * f.f2 * i3 - f.f1 * i2 - f.f3 * i4);
      *xout = x + dx;
      return J4 + dJ4 * dx;
    }
    x = fmin(fmax(x + dx, L.x_lo), L.x_hi);
  }
  *xout = x;
  return J4;
}

// Pull indices of the nine populations of cell (x, y); a negative row or
// column marks an off-lattice source (bounce-back from the opposite
// population of the same cell).
struct PullIdx {
  int64_t row, rm, rp;  // rows y, y-1, y+1 (base included), -1 if off-lattice
  int xm, xp;           // columns x-1, x+1, -1 if off-lattice
};

__device__ __forceinline__ PullIdx pull_index(const ProbDev& P, int x, int y) {
  PullIdx q;
  q.row = P.base + (int64_t)y * P.pitch;
  const int ym = y > 0 ? y - 1 : (P.bc_y == BC_PERIODIC ? P.ny - 1 : -1);
  const int yp = y < P.ny - 1 ? y + 1 : (P.bc_y == BC_PERIODIC ? 0 : -1);
  q.rm = ym >= 0 ? P.base + (int64_t)ym * P.pitch : -1;
  q.rp = yp >= 0 ? P.base + (int64_t)yp * P.pitch : -1;
  q.xm = x > 0 ? x - 1 : (P.bc_x == BC_PERIODIC ? P.nx - 1 : -1);
  q.xp = x < P.nx - 1 ? x + 1 : (P.bc_x == BC_PERIODIC ? 0 : -1);
  return q;
}

template <class T>
__device__ __forceinline__ void pull9(const T* __restrict__ fin, int64_t plane, const PullIdx& q, int x, T v[9]) {
  auto ld = [&](int a, int64_t r, int xs, int opp) -> T {
    return (r < 0 || xs < 0) ? fin[opp * plane + q.row + x] : fin[a * plane + r + xs];
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

// ------------------------------------------------------------------ FP64 step

template <int STAT, int TY, bool PERSIST>
__global__ void __launch_bounds__(kTileX) stream_collide_f64(const double* __restrict__ fin, double* __restrict__ fout,
                                                             const ProbDev* __restrict__ probs, int nprob, int ntiles,
                                                             int64_t plane, InvLimits L, InvLimitsF Lf) {
  int tile = (int)blockIdx.x;
#pragma unroll 1
  do {
    const int p = nprob == 1 ? 0 : find_problem(probs, nprob, tile);
    const ProbDev& P = probs[p];
    const int lt = tile - (int)P.tile_begin;
    const int ty = lt / P.tiles_x;
    const int x = (lt - ty * P.tiles_x) * kTileX + (int)threadIdx.x;
    if (x >= P.nx) continue;
    const int y1 = min(ty * TY + TY, P.ny);
#pragma unroll 1
    for (int y = ty * TY; y < y1; ++y) {
      const PullIdx q = pull_index(P, x, y);
      double f[9];
      pull9(fin, plane, q, x, f);
      // moments (the moment update after the LBGK equation, plus the energy)
      const double n = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7])) + f[8];
      const double jx = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
      const double jy = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
      const double E = ((f[1] + f[2]) + (f[3] + f[4])) + 2.0 * ((f[5] + f[6]) + (f[7] + f[8]));
      const double in = 1.0 / n;
      const double ux = jx * in, uy = jy * in;
      double J2, J4;
      if (STAT == STAT_FD) {
        J2 = 1.5 * (E * in - (ux * ux + uy * uy));  // 3 (E/n - u^2)/D
        int cl;
        double xx;
        J4 = j4_fp64(J2, L, Lf, &xx, &cl);
      } else if (STAT == STAT_FT) {
        // fixed theta: 2 pi theta f_1(x) = n, so the cell's t = 1/f_1(x) = 2 pi theta/n
        closure_from_t<STAT_FT>(2.0 * kPi * P.theta * in, J2, J4);
      } else {
        J2 = FixedJ<STAT>::j2;
        J4 = FixedJ<STAT>::j4;
      }
      double fe[9];
      feq_f64(n, ux, uy, J2, J4, fe);
      const double w = P.omega;
#pragma unroll
      for (int a = 0; a < 9; ++a) fout[a * plane + q.row + x] = fma(w, fe[a] - f[a], f[a]);
    }
  } while (PERSIST && (tile += (int)gridDim.x) < ntiles);
}

// ------------------------------------------------------------------ storage traits

template <class T>
struct Stor;
template <>
struct Stor<double> {
  static constexpr bool dev = false;
  __device__ static double to_f64(double v, double) { return v; }
  __device__ static double from_f64(double f, double) { return f; }
};
template <>
struct Stor<float> {
  static constexpr bool dev = true;
  __device__ static double to_f64(float v, double w) { return w + (double)v; }
  __device__ static float from_f64(double f, double w) { return (float)(f - w); }
};
template <>
struct Stor<__nv_bfloat16> {
  static constexpr bool dev = true;
  __device__ static double to_f64(__nv_bfloat16 v, double w) { return w + (double)__bfloat162float(v); }
  __device__ static __nv_bfloat16 from_f64(double f, double w) { return __float2bfloat16_rn((float)(f - w)); }
};

// ------------------------------------------------------------------ init

struct InitDesc {
  int32_t kind, x0, y0;  // kind 0 HALF, 1 QUADRANT, 2 FIELD (double arrays), 3 FIELD (float arrays)
  double s[4][4];  // n, ux, uy, t of up to four regions
  const double *n, *ux, *uy, *t;  // device arrays for FIELD
  const float *nf, *uxf, *uyf, *tf;  // device arrays for FIELD with float values (deviation storage only)
};

template <class T, int STAT>
__global__ void init_kernel(T* __restrict__ f, ProbDev P, int64_t plane, InitDesc d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cells = (int64_t)P.nx * P.ny;
  if (i >= cells) return;
  const int y = (int)(i / P.nx), x = (int)(i % P.nx);
  double n, ux, uy, t;
  if (d.kind == 2) {
    n = d.n[i]; ux = d.ux[i]; uy = d.uy[i]; t = d.t[i];
  } else {
    const int r = d.kind == 0 ? (x >= d.x0) : (x >= d.x0) + 2 * (y >= d.y0);
    n = d.s[r][0]; ux = d.s[r][1]; uy = d.s[r][2]; t = d.s[r][3];
  }
  double J2, J4;
  closure_from_t<STAT>(t, J2, J4);
  double fe[9];
  feq_f64(n, ux, uy, J2, J4, fe);
  const int64_t c = P.base + (int64_t)y * P.pitch + x;
#pragma unroll
  for (int a = 0; a < 9; ++a) f[a * plane + c] = Stor<T>::from_f64(fe[a], Stor<T>::dev ? P.wref[a] : 0.0);
}

// ------------------------------------------------------------------ populations in / out

template <class T>
__global__ void get_pop_kernel(const T* __restrict__ f, ProbDev P, int64_t plane, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cells = (int64_t)P.nx * P.ny;
  if (i >= cells) return;
  const int y = (int)(i / P.nx), x = (int)(i % P.nx);
  const int64_t c = P.base + (int64_t)y * P.pitch + x;
#pragma unroll
  for (int a = 0; a < 9; ++a) out[a * cells + i] = Stor<T>::to_f64(f[a * plane + c], Stor<T>::dev ? P.wref[a] : 0.0);
}

template <class T>
__global__ void set_pop_kernel(T* __restrict__ f, ProbDev P, int64_t plane, const double* __restrict__ in) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cells = (int64_t)P.nx * P.ny;
  if (i >= cells) return;
  const int y = (int)(i / P.nx), x = (int)(i % P.nx);
  const int64_t c = P.base + (int64_t)y * P.pitch + x;
#pragma unroll
  for (int a = 0; a < 9; ++a) f[a * plane + c] = Stor<T>::from_f64(in[a * cells + i], Stor<T>::dev ? P.wref[a] : 0.0);
}

// ------------------------------------------------------------------ moments

constexpr int kMomThreads = 256;
constexpr int kNPartial = 6;  // sum n, jx, jy, E, clamped, nonfinite
constexpr int kMomDevCells = 4;  // cells per thread of moments_dev_kernel

// FP64 storage (deviation storage has moments_dev_kernel): n, u, the sums
// and the FP64 inversion for x, t, theta, mu.
template <class T, int STAT>
__global__ void __launch_bounds__(kMomThreads) moments_kernel(const T* __restrict__ f, ProbDev P, int64_t plane,
                                                              InvLimits L, InvLimitsF Lf, double* __restrict__ on,
                                                              double* __restrict__ oux, double* __restrict__ ouy,
                                                              double* __restrict__ oT, double* __restrict__ omu,
                                                              double* __restrict__ ot, double* __restrict__ partials) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t cells = (int64_t)P.nx * P.ny;
  double acc[kNPartial] = {0, 0, 0, 0, 0, 0};
  const int64_t c = i < cells ? P.base + (int64_t)(i / P.nx) * P.pitch + (int)(i % P.nx) : 0;
  if (i < cells && P.solid != nullptr && P.solid[c] != 0) {  // obstacle: no fluid
    if (on) on[i] = 0.0;
    if (oux) oux[i] = 0.0;
    if (ouy) ouy[i] = 0.0;
    if (oT) oT[i] = 0.0;
    if (omu) omu[i] = 0.0;
    if (ot) ot[i] = 0.0;
  } else if (i < cells) {
    double v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = Stor<T>::to_f64(f[a * plane + c], Stor<T>::dev ? P.wref[a] : 0.0);
    const double n = ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
    const double jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
    const double jy = (v[2] - v[4]) + (v[5] + v[6]) - (v[7] + v[8]);
    const double E = ((v[1] + v[2]) + (v[3] + v[4])) + 2.0 * ((v[5] + v[6]) + (v[7] + v[8]));
    const double ux = jx / n, uy = jy / n;
    double theta = 0.0, mu = 0.0, t = 0.0;
    int cl = 0;
    if (STAT == STAT_FD) {
      const double J2 = 1.5 * (E / n - (ux * ux + uy * uy));
      double xx;
      j4_fp64(J2, L, Lf, &xx, &cl);
      t = 1.0 / (fmax(xx, 0.0) + log1p(exp(-fabs(xx))));  // t = T/T_F = 1/f_1(x)
      theta = n * t / (2.0 * kPi);     // theta = n t/(2 pi), T_F = n/(2 pi)
      mu = theta * xx;
    } else if (STAT == STAT_FT) {
      // fixed theta: t = 2 pi theta/n, x = ln(e^{1/t} - 1) = a + ln(1 - e^{-a}), a = 1/t
      theta = P.theta;
      t = 2.0 * kPi * theta / n;
      const double a = 1.0 / t;
      mu = theta * (a + log(-expm1(-a)));
    } else if (STAT == STAT_T0) {
      theta = 0.0; t = 0.0; mu = n / (2.0 * kPi);
    } else {
      theta = mu = t = __longlong_as_double(0x7ff8000000000000LL);
    }
    if (on) on[i] = n;
    if (oux) oux[i] = (jx + 0.5 * P.fx) / n;  // velocity at the time level under a body force
    if (ouy) ouy[i] = (jy + 0.5 * P.fy) / n;
    if (oT) oT[i] = theta;
    if (omu) omu[i] = mu;
    if (ot) ot[i] = t;
    acc[0] = n; acc[1] = jx; acc[2] = jy; acc[3] = E;
    acc[4] = cl;
    bool fin = isfinite(n) && isfinite(jx) && isfinite(jy) && isfinite(E);
#pragma unroll
    for (int a = 0; a < 9; ++a) fin = fin && isfinite(v[a]);
    acc[5] = fin ? 0.0 : 1.0;
  }
  // fixed-order block reduction: warp shuffle tree, then warps in order
  __shared__ double sh[kMomThreads / 32][kNPartial];
#pragma unroll
  for (int k = 0; k < kNPartial; ++k) {
    double s = acc[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    acc[k] = s;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < kNPartial; ++k) sh[wid][k] = acc[k];
  }
  __syncthreads();
  if (threadIdx.x < kNPartial) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kMomThreads / 32; ++w) s += sh[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * kNPartial + threadIdx.x] = s;
  }
}

}  // namespace lbm
