"""Plain FP64 d2v9 step with rigid obstacles and a constant body force.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's second experiment (Sect. "Numerical simulations for electrons in
metals", the porous-medium figures): electrons driven by a constant external
force through rigid obstacles, bounce-back on the obstacles, periodic borders.
The paper names no forcing scheme; this oracle uses the exact difference
method (Kupershtokh, Medvedev and Karpov, Comput. Math. Appl. 58 (2009) 965):
after the BGK relaxation each cell receives

    f_eq(n, u_0 + F/n) - f_eq(n, u_0),   u_0 = j/n,

with both equilibria built from the same moments I_0..I_6 (the same J_2 and
J_4), so the force changes momentum by exactly F per cell and step and leaves
the mass unchanged.  The velocity of the fluid at the time level is
(j + F/2)/n.

Obstacles: cell (x, y) is solid where ``solid[y, x]`` is true.  A fluid cell
whose pull source is solid (or beyond a wall) takes the opposite population of
its own cell (halfway bounce-back, as at the walls); solid cells keep their
populations and take no part in the step.
"""
from __future__ import annotations

import numpy as np

from . import fd as _fd
from . import gpoly as _g
from . import lbm as _l


def stream(f: np.ndarray, solid: np.ndarray, bc_x: str = "periodic", bc_y: str = "periodic") -> np.ndarray:
    """Pull streaming of f[a, y, x] with solid cells treated like walls."""
    ny, nx = f.shape[1:]
    out = np.empty_like(f)
    ys, xs = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for a in range(_l.Q):
        sx, sy = xs - _l.EX[a], ys - _l.EY[a]
        off = np.zeros((ny, nx), dtype=bool)
        if bc_x == "periodic":
            sx = sx % nx
        else:
            off |= (sx < 0) | (sx >= nx)
        if bc_y == "periodic":
            sy = sy % ny
        else:
            off |= (sy < 0) | (sy >= ny)
        sxc, syc = np.clip(sx, 0, nx - 1), np.clip(sy, 0, ny - 1)
        off |= solid[syc, sxc]
        out[a] = np.where(off, f[_l.OPP[a]], f[a][syc, sxc])
    return out


def collide(fin: np.ndarray, tau: float, stat: str, force) -> np.ndarray:
    """BGK plus the exact-difference force term, for fluid cells fin[a, c]."""
    n, j, En = _l.moments(fin)
    u0 = (j / n).T
    F = np.asarray(force, dtype=np.float64)
    if stat == "fd":
        j2 = _l.j2_from_moments(n, j, En)
        x = _l.invert_j2(j2)
        I = _l.moment_set(n, j2, _fd.j4_of_x(x), "fd", x)
    else:
        I = _l.moment_set(n, None, None, stat)
    feq = _g.equilibrium(I, u0, _l.D).T
    feq_f = _g.equilibrium(I, u0 + F[None, :] / n[:, None], _l.D).T
    return fin - (fin - feq) / tau + (feq_f - feq)


def step(f: np.ndarray, solid: np.ndarray, tau: float, stat: str, force, bc_x="periodic", bc_y="periodic"):
    fin = stream(f, solid, bc_x, bc_y)
    out = f.copy()  # solid cells keep their populations
    fl = ~solid
    out[:, fl] = collide(fin[:, fl], tau, stat, force)
    return out


def run(f, solid, tau, stat, force, nsteps, bc_x="periodic", bc_y="periodic"):
    for _ in range(nsteps):
        f = step(f, solid, tau, stat, force, bc_x, bc_y)
    return f


def velocity(f: np.ndarray, force) -> tuple:
    """(n, u_x, u_y) with u = (j + F/2)/n per cell."""
    n, j, _ = _l.moments(f)
    F = np.asarray(force, dtype=np.float64)
    return n, (j[0] + 0.5 * F[0]) / n, (j[1] + 0.5 * F[1]) / n

