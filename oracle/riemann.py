"""Exact solution of the Riemann problem for the isothermal Euler equations.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper validates its zero-temperature method against the exact solution of
the Riemann problem of an isothermal gas (Sect. "Numerical simulations for
electrons in metals", Fig. 1): at theta = 0 the FD gas has pressure
P = c^2 rho with c^2 = J_2/3 in lattice units (J_2 = 1 + 2/(2 + D)).  The
solution is written here from textbook gas dynamics (two waves around a
contact-free star state):

* across a shock into state K: u* - u_K = -/+ c (rho* - rho_K)/sqrt(rho* rho_K)
  (Rankine-Hugoniot for P = c^2 rho), shock speed
  S = (rho* u* - rho_K u_K)/(rho* - rho_K);
* across a rarefaction: u* - u_K = -/+ c ln(rho*/rho_K) (Riemann invariant
  u +/- c ln rho), fan between the characteristic speeds u_K -/+ c and
  u* -/+ c, inside the fan u = x/t +/- c and rho = rho_K exp(-/+(u - u_K)/c)
  (upper signs: left wave, lower signs: right wave);
* rho* solves f_L(rho*) + f_R(rho*) + u_R - u_L = 0 by bisection, with
  f_K(rho) = c (rho - rho_K)/sqrt(rho rho_K) for rho > rho_K (shock) and
  c ln(rho/rho_K) otherwise (rarefaction).
"""
from __future__ import annotations

import math

import numpy as np


def _f(rho, rk, c):
    if rho > rk:
        return c * (rho - rk) / math.sqrt(rho * rk)
    return c * math.log(rho / rk)


def star_state(rl, ul, rr, ur, c):
    """(rho*, u*) of the isothermal Riemann problem."""
    lo, hi = 1e-12, 10.0 * max(rl, rr) + 10.0 * abs(ur - ul) / c + 1.0
    g = lambda r: _f(r, rl, c) + _f(r, rr, c) + ur - ul
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if g(mid) > 0.0:
            hi = mid
        else:
            lo = mid
    rs = 0.5 * (lo + hi)
    us = 0.5 * (ul + ur) + 0.5 * (_f(rs, rr, c) - _f(rs, rl, c))
    return rs, us


def sample(xi, rl, ul, rr, ur, c):
    """(rho, u) at similarity coordinate xi = x/t (arrays allowed)."""
    rs, us = star_state(rl, ul, rr, ur, c)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    for i, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact: left wave
            if rs > rl:  # shock
                S = (rs * us - rl * ul) / (rs - rl)
                rho[i], u[i] = (rl, ul) if s < S else (rs, us)
            else:  # rarefaction
                head, tail = ul - c, us - c
                if s < head:
                    rho[i], u[i] = rl, ul
                elif s > tail:
                    rho[i], u[i] = rs, us
                else:
                    uu = s + c
                    rho[i], u[i] = rl * math.exp(-(uu - ul) / c), uu
        else:  # right wave
            if rs > rr:
                S = (rs * us - rr * ur) / (rs - rr)
                rho[i], u[i] = (rs, us) if s < S else (rr, ur)
            else:
                tail, head = us + c, ur + c
                if s > head:
                    rho[i], u[i] = rr, ur
                elif s < tail:
                    rho[i], u[i] = rs, us
                else:
                    uu = s - c
                    rho[i], u[i] = rr * math.exp((uu - ur) / c), uu
    return rho, u
