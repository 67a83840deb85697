"""Plain FP64 lattice Boltzmann-BGK step on the d1v3 lattice (D = 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's second lattice (Sect. "The Gaussian quadrature"): velocities
e_0 = 0, e_+1 = +1, e_-1 = -1 (stored in that order), weights
w_0 = I_0 (1 - J_2/3), w_+-1 = I_0 J_2/6, velocity scale c_0 = sqrt(3 I_4/I_2).
The state is the post-collision population array ``f[a, x]``.  One step:

1. stream: f_a(x, t+1) is pulled from x - e_a; x is periodic or closed by
   halfway bounce-back walls at x = -1/2 and x = nx - 1/2 (a pulled source
   beyond a wall is replaced by the opposite population of the same cell);
2. moments: n = I_0 = sum_a f_a, j = f_+1 - f_-1, u_0 = j/n;
3. equilibrium: ``gpoly.equilibrium`` (the tensor contraction of
   Eq. (expansao0), D = 1) from the closure's moments I_0..I_6;
4. BGK: f* = f - (f - f_eq)/tau.

Closures:
* "t0": theta = 0 (the paper's zero-temperature runs): I_2N from
  Eq. (sommerfeld) at theta = 0 with D = 1, mu fixed by n through
  I_0 = (2 pi mu)^{1/2}/Gamma(3/2), i.e. mu = n^2/8; then J_N = 1 + 2/(N + 1)
  (J_2 = 5/3, J_4 = 7/5) and the lattice sound speed squared is J_2/3 = 5/9;
* "mb": Maxwell-Boltzmann with theta = 1/3 (J_N = 1): the standard D1Q3
  lattice.
There is no finite-temperature closure through the energy on d1v3: with
three velocities the moments n, j and E fix all three populations, so a
collision that conserves them leaves f unchanged.
"""
from __future__ import annotations

import numpy as np

from . import gpoly as _g

D = 1
Q = 3
E = _g.E_D1V3[:, 0]
OPP = _g.OPP_D1V3


def stream(f: np.ndarray, bc_x: str = "periodic") -> np.ndarray:
    """Pull streaming of f[a, x]."""
    out = np.empty_like(f)
    out[0] = f[0]
    if bc_x == "periodic":
        out[1] = np.roll(f[1], 1)    # e = +1: from x - 1
        out[2] = np.roll(f[2], -1)   # e = -1: from x + 1
    elif bc_x == "bounceback":
        out[1, 1:] = f[1, :-1]
        out[1, 0] = f[2, 0]          # source x = -1 is beyond the wall
        out[2, :-1] = f[2, 1:]
        out[2, -1] = f[1, -1]        # source x = nx is beyond the wall
    else:
        raise ValueError(bc_x)
    return out


def moments(f: np.ndarray):
    """n and j of f[a, ...]."""
    n = f.sum(axis=0)
    j = f[1] - f[2]
    return n, j


def moment_set(n, stat: str) -> dict:
    n = np.asarray(n, dtype=np.float64)
    if stat == "t0":
        return _g.moments_t0(n * n / 8.0, D, nmax=3)
    if stat == "mb":
        return _g.moments_mb(n, 1.0 / 3.0, nmax=3)
    raise ValueError(f"d1v3 has no {stat!r} closure")


def equilibrium(n, u0, stat: str) -> np.ndarray:
    """f_eq[a, ...] for states n, u0 (arrays of equal shape)."""
    n = np.asarray(n, dtype=np.float64)
    shape = n.shape
    I = moment_set(n.reshape(-1), stat)
    feq = _g.equilibrium(I, np.asarray(u0, dtype=np.float64).reshape(-1, 1), D)
    return feq.T.reshape((Q,) + shape)


def init_equilibrium(n, u0, stat: str) -> np.ndarray:
    return equilibrium(n, u0, stat)


def collide(fin: np.ndarray, tau: float, stat: str) -> np.ndarray:
    n, j = moments(fin)
    feq = equilibrium(n, j / n, stat)
    return fin - (fin - feq) / tau


def step(f: np.ndarray, tau: float, stat: str, bc_x: str = "periodic") -> np.ndarray:
    return collide(stream(f, bc_x), tau, stat)


def run(f: np.ndarray, tau: float, stat: str, nsteps: int, bc_x: str = "periodic") -> np.ndarray:
    for _ in range(nsteps):
        f = step(f, tau, stat, bc_x)
    return f


def fields(f: np.ndarray, stat: str) -> dict:
    """n, u0 and, at theta = 0, the chemical potential mu = n^2/8."""
    n, j = moments(f)
    out = {"n": n, "ux": j / n}
    if stat == "t0":
        out["mu"] = n * n / 8.0
    return out
