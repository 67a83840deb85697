"""Generator of the starting value of the FP32 inversion's Newton branch
(csrc/fd_device_f32.cuh, x_start_general): a degree-8 least-squares fit of x
as a polynomial in v = ln((J_2 - 1)/(3/2 - J_2)) over the branch's interval.

The branch serves J_2 in (J_2(x_lo), J_2(7)], x_lo = x(t = 10); above x = 7
the degenerate root with tail passes is exact.  The fit runs over x in
[x_lo - 0.05, 7.3].  v follows both ends:
ln(J_2 - 1) ~ x - ln 8 in the Maxwell-Boltzmann limit, and 3/2 - J_2 ~ x^-2
toward the degenerate side.  J_2 = f_2^2/(f_1 f_3), with the normalised
complete Fermi-Dirac integrals f_n(x) = -Li_n(-e^x) taken from mpmath's
polylogarithm (independent of the library and of the test oracle).

A second fit (fit_degenerate) gives x directly for 7 < x < 17 from
ln(3/2 - J_2), in place of the tail passes.

Two more give J_4 straight from delta = 3/2 - J_2, so that the step, which
needs J_4 and not x, skips x in both degenerate branches:
- fit_j4_degenerate: x >= 17, a degree-4 polynomial in delta over
  [0, 1.02 delta(17)], fitted to the degenerate closed form (the e^{-x}
  tails it drops are below 3.4e-9 of J_4 there);
- fit_j4_mid: 7 < x < 17, a degree-7 polynomial in (delta - m)/h over
  [0.98 delta(17), 1.02 delta(7)], fitted to J_4 = f_3^2/(f_2 f_4);
- fit_j4_low: x_lo < x <= 7, a degree-12 polynomial in (delta - m)/h over
  [delta(7.1), delta(x_lo - 0.05)], fitted to J_4 = f_3^2/(f_2 f_4), in place
  of the Newton iteration (which then runs only for callers that need x).

Run: python paper_1510_07328_gb300/fit_x_of_j2.py  (prints the coefficients,
highest degree first, and the largest errors of the fits).
"""
import mpmath as mp
import numpy as np


def j2(x):
    f = [-mp.polylog(n, -mp.e ** x) for n in (1, 2, 3)]
    return f[1] ** 2 / (f[0] * f[2])


def j4(x):
    f = [-mp.polylog(n, -mp.e ** x) for n in (2, 3, 4)]
    return f[1] ** 2 / (f[0] * f[2])


def j4_closed_form(delta):
    """J_4 of the degenerate regime (e^{-x} tails dropped) at delta = 3/2 -
    J_2: s = x^2 is the large root of 6 delta s^2 - (3 pi^2 - 6 delta pi^2) s
    + pi^4 = 0, and J_4 = P_3^2/(P_2 P_4) = 60 s (s + pi^2)^2 / ((3 s + pi^2)
    (15 s^2 + 30 pi^2 s + 7 pi^4)); 4/3 at delta = 0."""
    d = mp.mpf(delta)
    if d == 0:
        return mp.mpf(4) / 3
    p2 = mp.pi ** 2
    a, b, c = 6 * d, 3 * p2 - 6 * d * p2, p2 ** 2
    s = (b + mp.sqrt(b * b - 4 * a * c)) / (2 * a)
    sp = s + p2
    return 60 * s * sp * sp / ((3 * s + p2) * (15 * s * s + 30 * p2 * s + 7 * p2 ** 2))


def fit_j4_degenerate(deg: int = 4, samples: int = 600):
    """J_4 for x >= 17 as a polynomial in delta over [0, 1.02 delta(17)].
    Returns (coefficients, largest relative error against the closed form,
    delta(17))."""
    mp.mp.dps = 30
    d17 = float(1.5 - j2(17))
    d = np.linspace(0.0, 1.02 * d17, samples)
    J = np.array([float(j4_closed_form(v)) for v in d])
    c = np.polyfit(d, J, deg)
    err = float((np.abs(np.polyval(c, d) - J) / J).max())
    return c, err, d17


def fit_j4_mid(deg: int = 7, samples: int = 700):
    """J_4 for 7 < x < 17 as a polynomial in v = (delta - m)/h, v in [-1, 1]
    over [0.98 delta(17), 1.02 delta(7)]; fitted over x in [6.95, 17.1].
    Returns (coefficients, m, h, largest relative error)."""
    mp.mp.dps = 30
    d7, d17 = float(1.5 - j2(7)), float(1.5 - j2(17))
    xs = np.linspace(6.95, 17.1, samples)
    d = np.array([float(1.5 - j2(x)) for x in xs])
    J = np.array([float(j4(x)) for x in xs])
    lo, hi = 0.98 * d17, 1.02 * d7
    m, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
    v = (d - m) / h
    c = np.polyfit(v, J, deg)
    err = float((np.abs(np.polyval(c, v) - J) / J).max())
    return c, m, h, err


def fit_j4_low(deg: int = 12, samples: int = 1500):
    """J_4 for x_lo < x <= 7 (x_lo = x(t = 10)) as a polynomial in
    v = (delta - m)/h, v in [-1, 1] over [delta(7.1), delta(x_lo - 0.05)]; a
    Chebyshev least-squares fit over x in [x_lo - 0.05, 7.1], returned as
    monomial coefficients of v.  Returns (coefficients, m, h, largest relative
    error)."""
    mp.mp.dps = 30
    x_lo = float(mp.log(mp.e ** mp.mpf("0.1") - 1))
    xs = np.linspace(x_lo - 0.05, 7.1, samples)
    d = np.array([float(1.5 - j2(x)) for x in xs])
    J = np.array([float(j4(x)) for x in xs])
    lo, hi = float(1.5 - j2(7.1)), float(1.5 - j2(x_lo - 0.05))
    m, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
    v = (d - m) / h
    c = np.polynomial.chebyshev.cheb2poly(np.polynomial.chebyshev.chebfit(v, J, deg))[::-1]
    err = float((np.abs(np.polyval(c, v) - J) / J).max())
    return c, m, h, err


def fit(deg: int = 8, samples: int = 800):
    mp.mp.dps = 30
    x_lo = float(mp.log(mp.e ** mp.mpf("0.1") - 1))  # t = 10: 1/f_1(x) = 10
    xs = np.linspace(x_lo - 0.05, 7.3, samples)
    J = np.array([float(j2(x)) for x in xs])
    v = np.log((J - 1.0) / (1.5 - J))
    c = np.polyfit(v, xs, deg)
    err = float(np.abs(np.polyval(c, v) - xs).max())
    return c, err


def fit_degenerate(deg: int = 8, samples: int = 700):
    """x for 7 < x < 17 (delta = 3/2 - J_2 between delta(17) and delta(7)) as a
    degree-8 polynomial in u = (ln delta - m)/h, u in [-1, 1] over
    [0.98 delta(17), 1.02 delta(7)]; fitted over x in [6.95, 17.1].  The
    inversion uses it in place of the tail passes.  Returns (coefficients,
    m, h, largest relative error, delta(7), delta(17))."""
    mp.mp.dps = 30
    d7, d17 = float(1.5 - j2(7)), float(1.5 - j2(17))
    xs = np.linspace(6.95, 17.1, samples)
    d = np.array([float(1.5 - j2(x)) for x in xs])
    lo, hi = np.log(d17 * 0.98), np.log(d7 * 1.02)
    m, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
    u = (np.log(d) - m) / h
    c = np.polyfit(u, xs, deg)
    err = float((np.abs(np.polyval(c, u) - xs) / xs).max())
    return c, m, h, err, d7, d17


if __name__ == "__main__":
    c, err = fit()
    print("coefficients (highest degree first):", ", ".join(f"{v:.9e}f" for v in c))
    print(f"max |x_fit - x| = {err:.2e}")
    mp.mp.dps = 30
    print(f"3/2 - J_2(7) = {float(1.5 - j2(7)):.9f}")
    c, m, h, err, d7, d17 = fit_degenerate()
    print("degenerate-range coefficients:", ", ".join(f"{v:.9e}f" for v in c))
    print(f"m = {m:.9f}, 1/h = {1.0 / h:.9f}, max relative error {err:.2e}, 3/2 - J_2(17) = {d17:.9f}")
    c, err, _ = fit_j4_degenerate()
    print("J_4 for x >= 17, polynomial in delta:", ", ".join(f"{v:.9e}f" for v in c))
    print(f"max relative error against the closed form {err:.2e}")
    c, m, h, err = fit_j4_mid()
    print("J_4 for 7 < x < 17, polynomial in (delta - m)/h:", ", ".join(f"{v:.9e}f" for v in c))
    print(f"m = {m:.9e}, 1/h = {1.0 / h:.9e}, max relative error {err:.2e}")
    c, m, h, err = fit_j4_low()
    print("J_4 for x <= 7, polynomial in (delta - m)/h:", ", ".join(f"{v:.9e}f" for v in c))
    print(f"m = {m:.9e}, 1/h = {1.0 / h:.9e}, max relative error {err:.2e}")
