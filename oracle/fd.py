"""Complete Fermi-Dirac integrals and the FD moment ratios, in FP64.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain CPU oracle that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it;
the library under ``paper_1510_07328_gb300`` never does, and this package never
imports that library.

Definitions (paper, Sect. "Generalized polynomials in D dimensions", the FD
weight and its moments ``I_2N = (2 pi)^{D/2} theta^{N+D/2} g_{N+D/2}(e^{mu/theta})``):

    f_n(x) = 1/Gamma(n) * int_0^inf t^(n-1) / (exp(t - x) + 1) dt ,   x = mu/theta

The paper prints ``g_nu`` without the ``1/Gamma(nu)``; only the normalised form
is consistent with Eq. (i2n-cont2) and with the Sommerfeld expansion, Eq.
(sommerfeld), so that is the reading used here (f_n = -Li_n(-e^x)).

Evaluation, three regions, each a direct consequence of the definition:

* x <= -1: expand 1/(e^{t-x}+1) = sum_k (-1)^(k+1) e^{k(x-t)} and integrate term
  by term: f_n(x) = sum_k (-1)^(k+1) e^{kx} / k^n.
* x >= +1: the polylogarithm inversion formula for integer order,
  f_n(x) = P_n(x) - (-1)^n f_n(-x), P_n(x) = 2 sum_j eta(2j) x^(n-2j)/(n-2j)!,
  with eta(0)=1/2, eta(2)=pi^2/12, eta(4)=7 pi^4/720.  Its first two terms are
  the paper's Sommerfeld expansion, Eq. (sommerfeld).
* |x| < 1: Gauss-Legendre quadrature of the defining integral on [0, 60] in
  panels of width 2 (the integrand is analytic in a strip of half-width pi
  about the real axis, so 16 nodes per panel reach well below 1e-20).

f_0(x) = 1/(1+e^{-x}) is the n -> 0 member (d f_n/dx = f_{n-1}).

Pinned in tests/test_oracle_fd.py against mpmath's polylog, against the
closed forms f_0 and f_1 = ln(1+e^x), against the derivative identity, and at
the region seams.
"""
from __future__ import annotations

import math

import numpy as np

NMAX = 5  # orders 0..5: I_0..I_8 for D = 2 need f_1..f_5

_ETA_EVEN = (0.5, math.pi ** 2 / 12.0, 7.0 * math.pi ** 4 / 720.0)

# Gauss-Legendre panels for the |x| < 1 region.
_GL_X, _GL_W = np.polynomial.legendre.leggauss(16)
_PANEL = 2.0
_TMAX = 60.0
_nodes = []
_weights = []
for a in np.arange(0.0, _TMAX, _PANEL):
    _nodes.append(a + 0.5 * _PANEL * (_GL_X + 1.0))
    _weights.append(0.5 * _PANEL * _GL_W)
_QT = np.concatenate(_nodes)
_QW = np.concatenate(_weights)


def _series_neg(n: int, x: np.ndarray) -> np.ndarray:
    """sum_{k>=1} (-1)^(k+1) e^{kx}/k^n for x <= -1 (ratio <= e^-1)."""
    y = np.exp(x)
    out = np.zeros_like(x)
    yk = np.ones_like(x)
    for k in range(1, 80):  # e^-80 ~ 2e-35: far past double precision
        yk = yk * y
        term = yk / float(k) ** n
        out = out + term if (k % 2 == 1) else out - term
    return out


def _poly_pos(n: int, x: np.ndarray) -> np.ndarray:
    """P_n(x) of the inversion formula (degenerate part of f_n)."""
    out = np.zeros_like(x)
    for j, eta in enumerate(_ETA_EVEN):
        p = n - 2 * j
        if p < 0:
            break
        out = out + 2.0 * eta * x ** p / math.factorial(p)
    return out


def _quad(n: int, x: np.ndarray) -> np.ndarray:
    """Gauss-Legendre quadrature of the defining integral (|x| < 1)."""
    t = _QT[None, :]
    fermi = 1.0 / (np.exp(t - x[:, None]) + 1.0)
    integrand = t ** (n - 1) * fermi
    return (integrand * _QW[None, :]).sum(axis=1) / math.gamma(n)


def fd(n: int, x) -> np.ndarray:
    """Normalised complete FD integral f_n(x) for integer n in 0..NMAX."""
    x = np.asarray(x, dtype=np.float64)
    shape = x.shape
    x = x.reshape(-1)
    if n == 0:
        return (1.0 / (1.0 + np.exp(-x))).reshape(shape)
    if n < 0 or n > NMAX:
        raise ValueError("order out of range")
    out = np.empty_like(x)
    neg = x <= -1.0
    pos = x >= 1.0
    mid = ~(neg | pos)
    if neg.any():
        out[neg] = _series_neg(n, x[neg])
    if pos.any():
        xp = x[pos]
        sign = -1.0 if n % 2 == 0 else 1.0  # -(-1)^n
        out[pos] = _poly_pos(n, xp) + sign * _series_neg(n, -xp)
    if mid.any():
        out[mid] = _quad(n, x[mid])
    return out.reshape(shape)


def fd_all(x, nmax: int = 4) -> list:
    """[f_0(x), ..., f_nmax(x)]."""
    return [fd(n, x) for n in range(nmax + 1)]


def j2_of_x(x) -> np.ndarray:
    """J_2 = I_2^2/(I_4 I_0) for the D = 2 FD weight = f_2^2/(f_1 f_3)
    (definition of J_L under Eq. (H4); I_2N in terms of f_{N+1})."""
    f1, f2, f3 = fd(1, x), fd(2, x), fd(3, x)
    return f2 * f2 / (f1 * f3)


def j4_of_x(x) -> np.ndarray:
    """J_4 = I_4^2/(I_6 I_2) = f_3^2/(f_2 f_4) for D = 2."""
    f2, f3, f4 = fd(2, x), fd(3, x), fd(4, x)
    return f3 * f3 / (f2 * f4)


def x_of_t(t) -> np.ndarray:
    """Log-fugacity x = mu/theta from t = T/T_F (D = 2).

    With T_F the zero-temperature chemical potential at the same density,
    I_0 = 2 pi theta f_1(x) and I_0 = 2 pi T_F give t = 1/f_1(x) = 1/ln(1+e^x),
    hence x = ln(e^{1/t} - 1) = 1/t + ln(1 - e^{-1/t}).
    """
    t = np.asarray(t, dtype=np.float64)
    return 1.0 / t + np.log(-np.expm1(-1.0 / t))


def t_of_x(x) -> np.ndarray:
    """t = T/T_F = 1/f_1(x) (D = 2)."""
    return 1.0 / fd(1, x)
