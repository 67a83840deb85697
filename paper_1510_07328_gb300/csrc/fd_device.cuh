// Device Fermi-Dirac functions for D = 2 and the inversion J_2 -> x.
//
// f_n(x) = -Li_n(-e^x) is the normalised complete Fermi-Dirac integral (the
// g_nu of Sect. "Generalized polynomials in D dimensions" divided by
// Gamma(nu)); for the FD weight in D = 2, I_2N = 2 pi theta^{N+1} f_{N+1}(x)
// with x = mu/theta, so J_2 = f_2^2/(f_1 f_3) and J_4 = f_3^2/(f_2 f_4).
//
// Evaluation (integer orders; a = |x|, y = e^{-a}):
//  * f_0 = 1/(1 + e^{-x}) and f_1 = max(x,0) + log1p(e^{-a}) in closed form;
//  * S_n(y) = sum_{k>=1} (-1)^{k+1} y^k / k^n, n = 2..4, directly for a >= 2
//    (ratio <= e^-2, early exit), else by Algorithm 1 of Cohen, Rodriguez
//    Villegas and Zagier, "Convergence acceleration of alternating series"
//    (Experimental Math. 9, 2000), whose error is below 2 S/(3+sqrt 8)^N for a
//    moment sequence such as y^{k+1}/(k+1)^n, y in (0, 1];
//  * x <= 0: f_n(x) = S_n(e^x); x > 0: the inversion formula
//    f_n(x) = P_n(x) - (-1)^n S_n(e^{-x}), P_2 = x^2/2 + pi^2/6,
//    P_3 = x^3/6 + pi^2 x/6, P_4 = x^4/24 + pi^2 x^2/12 + 7 pi^4/360; for
//    x >= 40 the S_n tails are below 4.3e-18 relative and dropped.  The first
//    two terms of P_n are the Sommerfeld expansion, Eq. (sommerfeld).
//
// Inversion of J_2 (strictly increasing in x): in the degenerate regime the
// polynomial form gives 3/2 - J_2 = pi^2 (3 s - pi^2) / (6 s (s + pi^2)),
// s = x^2, a quadratic in s whose large root is exact for x >= 40 and a
// starting value elsewhere; then Newton with dJ_2/dx = J_2 (2 f_1/f_2 -
// f_0/f_1 - f_2/f_3) (d f_n/dx = f_{n-1}), safeguarded by bisection on the
// bracket, stopped at the rounding floor of the residual.  x is clamped to
// [x(t = 10), x(t = 1e-3)].
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace lbm {

constexpr double kPi = 3.14159265358979323846;
constexpr double kPi2 = kPi * kPi;
constexpr double kXDeg = 40.0;  // S_n tails dropped beyond this
constexpr double kTMin = 1e-3;  // clamp interval of the inversion in t = T/T_F
constexpr double kTMax = 10.0;

struct FD5 {
  double f0, f1, f2, f3, f4;
};

// Limits of the inversion, filled once per context by a setup kernel.
struct InvLimits {
  double x_lo, x_hi;    // x(t_max), x(t_min)
  double j2_lo, j2_hi;  // J_2 at those x
  double j4_lo, j4_hi;  // J_4 at those x
};

__device__ __forceinline__ void fd_poly(double x, double& p2, double& p3, double& p4) {
  const double s = x * x;
  p2 = 0.5 * s + kPi2 / 6.0;
  p3 = x * (s + kPi2) * (1.0 / 6.0);
  p4 = s * s * (1.0 / 24.0) + kPi2 * s * (1.0 / 12.0) + 7.0 * kPi2 * kPi2 / 360.0;
}

// 1/k, k = 1..48, for the series terms (warp-uniform reads).
static __constant__ double c_inv_k64[49] = {
    0.0,       1.0 / 1,  1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,  1.0 / 6,  1.0 / 7,  1.0 / 8,  1.0 / 9,
    1.0 / 10,  1.0 / 11, 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17, 1.0 / 18, 1.0 / 19,
    1.0 / 20,  1.0 / 21, 1.0 / 22, 1.0 / 23, 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29,
    1.0 / 30,  1.0 / 31, 1.0 / 32, 1.0 / 33, 1.0 / 34, 1.0 / 35, 1.0 / 36, 1.0 / 37, 1.0 / 38, 1.0 / 39,
    1.0 / 40,  1.0 / 41, 1.0 / 42, 1.0 / 43, 1.0 / 44, 1.0 / 45, 1.0 / 46, 1.0 / 47, 1.0 / 48};

// S_2, S_3, S_4 at y = e^{-a}, a >= 0.
static __device__ __noinline__ void fd_alt_series(double a, double& s2, double& s3, double& s4) {
  const double y = exp(-a);
  s2 = s3 = s4 = 0.0;
  if (a >= 2.0) {
    double yk = y, sg = 1.0;
#pragma unroll 1
    for (int k = 1; k <= 48; ++k) {
      const double ik = c_inv_k64[k];
      const double t2 = yk * ik * ik, t3 = t2 * ik, t4 = t3 * ik;
      s2 = fma(sg, t2, s2);
      s3 = fma(sg, t3, s3);
      s4 = fma(sg, t4, s4);
      yk *= y;
      sg = -sg;
      if (yk < 1e-18 * y) break;
    }
  } else {
    const int N = 24;  // (3 + sqrt 8)^24 ~ 2.3e18
    double d = pow(3.0 + sqrt(8.0), (double)N);
    d = 0.5 * (d + 1.0 / d);
    double b = -1.0, c = -d, yk = y;
#pragma unroll 1
    for (int k = 0; k < N; ++k) {
      c = b - c;
      const double ik = 1.0 / (double)(k + 1);
      const double a2 = yk * ik * ik, a3 = a2 * ik, a4 = a3 * ik;
      s2 = fma(c, a2, s2);
      s3 = fma(c, a3, s3);
      s4 = fma(c, a4, s4);
      b = (double)(k + N) * (double)(k - N) * b / (((double)k + 0.5) * (double)(k + 1));
      yk *= y;
    }
    s2 /= d;
    s3 /= d;
    s4 /= d;
  }
}

__device__ __forceinline__ FD5 fd_eval(double x) {
  FD5 r;
  const double a = fabs(x);
  const double em = exp(-a);
  r.f0 = x >= 0.0 ? 1.0 / (1.0 + em) : em / (1.0 + em);
  r.f1 = fmax(x, 0.0) + log1p(em);
  if (x >= kXDeg) {
    fd_poly(x, r.f2, r.f3, r.f4);
    return r;
  }
  double s2, s3, s4;
  fd_alt_series(a, s2, s3, s4);
  if (x > 0.0) {
    double p2, p3, p4;
    fd_poly(x, p2, p3, p4);
    r.f2 = p2 - s2;
    r.f3 = p3 + s3;
    r.f4 = p4 - s4;
  } else {
    r.f2 = s2;
    r.f3 = s3;
    r.f4 = s4;
  }
  return r;
}

// x = mu/theta from t = T/T_F (D = 2): t = 1/f_1(x) => x = 1/t + log(1 - e^{-1/t}).
__device__ __forceinline__ double x_of_t(double t) {
  const double v = 1.0 / t;
  return v + log(-expm1(-v));
}

__device__ __forceinline__ double j2_of(const FD5& f) { return f.f2 * f.f2 / (f.f1 * f.f3); }
__device__ __forceinline__ double j4_of(const FD5& f) { return f.f3 * f.f3 / (f.f2 * f.f4); }

// Solve J_2^FD(x) = J2.  *clamped is set when x hits an end of the interval.
// A non-finite J2 returns NaN without iterating.
static __device__ __noinline__ double invert_j2(double J2, const InvLimits& L, int* clamped) {
  *clamped = 0;
  if (!(J2 == J2) || isinf(J2)) return J2 - J2;  // NaN
  if (J2 >= L.j2_hi) {
    *clamped = 1;
    return L.x_hi;
  }
  if (J2 <= L.j2_lo) {
    *clamped = 1;
    return L.x_lo;
  }
  const double delta = 1.5 - J2;
  double x = 2.0;
  if (delta < 0.1) {
    // 6 delta s^2 - (3 pi^2 - 6 delta pi^2) s + pi^4 = 0, large root
    const double A = 6.0 * delta, B = 3.0 * kPi2 - 6.0 * delta * kPi2, C = kPi2 * kPi2;
    const double s = (B + sqrt(fmax(B * B - 4.0 * A * C, 0.0))) / (2.0 * A);
    x = sqrt(s);
    if (x >= kXDeg) return fmin(x, L.x_hi);
  }
  double lo = L.x_lo, hi = L.x_hi;
#pragma unroll 1
  for (int it = 0; it < 80; ++it) {
    const FD5 f = fd_eval(x);
    const double j = j2_of(f);
    const double g = j - J2;
    if (g == 0.0 || fabs(g) <= 2.5e-16 * J2) break;
    if (g < 0.0) lo = x; else hi = x;
    const double dj = j * (2.0 * f.f1 / f.f2 - f.f0 / f.f1 - f.f2 / f.f3);
    double xn = x - g / dj;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    const bool done = fabs(xn - x) <= 2e-16 * fabs(x);
    x = xn;
    if (done || hi - lo <= 4e-16 * fabs(x)) break;
  }
  return x;
}

}  // namespace lbm
