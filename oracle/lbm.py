"""Plain FP64 lattice Boltzmann-BGK step on the d2v9 lattice.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The state is the post-collision population array ``f[a, y, x]`` (a = 0..8,
velocity order: rest; (1,0),(0,1),(-1,0),(0,-1); (1,1),(-1,1),(-1,-1),(1,-1)).
One step, in the paper's order (Sect. "The Gaussian quadrature", the LBGK
equation and the moment update that follows it):

1. stream: f_a(x, t+1) is pulled from x - e_a.  y is periodic; x is periodic or
   closed by halfway bounce-back walls at x = -1/2 and x = nx - 1/2 (a pulled
   source beyond a wall is replaced by the opposite population of the same
   cell, diagonals included).
2. moments: n = I_0 = sum_a f_a; j = sum_a f_a e_a, u_0 = j/n; and the
   geometric energy E = sum_a f_a |e_a|^2.  The paper updates only I_0 and u_0;
   the finite-temperature method also needs the second moment, which by the
   quadrature of the equilibrium equals n (u_0^2 + D J_2/3), so
   J_2 = 3 (E/n - u_0^2)/D is read directly off the moments.
3. inversion: x = mu/theta solves J_2^FD(x) = J_2, by plain bisection on
   [x(t_max), x(t_min)] (J_2^FD is strictly increasing in x).  x is clamped to
   that interval; the measured J_2 is kept unclamped in the equilibrium so the
   collision conserves n, j and E exactly.  Then J_4 = J_4^FD(x).
4. equilibrium: ``gpoly.equilibrium`` (tensor contraction, Eq. (expansao0))
   built from moments I_0..I_6 whose ratios are the measured J_2 and J_4.
5. BGK: f* = f - (f - f_eq)/tau.

Statistics: "fd" (above), "t0" (theta = 0 closure: J_N = 1 + 2/(N+D) constant,
the paper's zero-temperature runs) and "mb" (Maxwell-Boltzmann: J_N = 1,
the standard Hermite D2Q9 limit).  In "t0" and "mb" J_2 is a constant and
energy is not a collision invariant.

"ft" is the fixed-temperature reading of the moment update, which names only
I_0 and u_0: theta is a constant of the problem (Params.theta), x follows
from the density alone, n = I_0 = 2 pi theta f_1(x) (the FD form of I_2N with
N = 0, D = 2), in closed form x = a + ln(1 - e^{-a}), a = n/(2 pi theta), and
J_2, J_4 are the FD values at that x.  Energy is not a collision invariant.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import fd as _fd
from . import gpoly as _g

D = 2
Q = 9
E = _g.E_D2V9
OPP = _g.OPP_D2V9
EX = E[:, 0].astype(int)
EY = E[:, 1].astype(int)

T_MIN = 1e-3   # clamp interval of the inversion, in t = T/T_F
T_MAX = 10.0
X_HI = float(_fd.x_of_t(T_MIN))
X_LO = float(_fd.x_of_t(T_MAX))


@dataclass
class Params:
    tau: float
    bc_x: str = "periodic"  # or "bounceback"
    bc_y: str = "periodic"  # or "bounceback"
    stat: str = "fd"        # "fd", "t0", "mb", "ft"
    theta: float | None = None  # the constant theta of the "ft" closure


# ---------------------------------------------------------------- streaming


def stream(f: np.ndarray, bc_x: str, bc_y: str = "periodic") -> np.ndarray:
    """Pull streaming with periodic or halfway bounce-back boundaries."""
    _, ny, nx = f.shape
    out = np.empty_like(f)
    ys, xs = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    for a in range(Q):
        sx = xs - EX[a]
        sy = ys - EY[a]
        off = np.zeros((ny, nx), dtype=bool)
        if bc_x == "periodic":
            sx = sx % nx
        else:
            off |= (sx < 0) | (sx >= nx)
            sx = np.clip(sx, 0, nx - 1)
        if bc_y == "periodic":
            sy = sy % ny
        else:
            off |= (sy < 0) | (sy >= ny)
            sy = np.clip(sy, 0, ny - 1)
        pulled = f[a, sy, sx]
        out[a] = np.where(off, f[OPP[a]], pulled)
    return out


# ---------------------------------------------------------------- moments


def moments(f: np.ndarray):
    """n, j (2, ...), E = sum f |e|^2 over the velocity axis 0."""
    n = f.sum(axis=0)
    jx = np.tensordot(E[:, 0], f, axes=(0, 0))
    jy = np.tensordot(E[:, 1], f, axes=(0, 0))
    e2 = (E * E).sum(axis=1)
    En = np.tensordot(e2, f, axes=(0, 0))
    return n, np.stack([jx, jy]), En


def j2_from_moments(n, j, En):
    """J_2 = 3 (E/n - |u_0|^2)/D."""
    u0 = j / n
    return 3.0 * (En / n - (u0 * u0).sum(axis=0)) / D


# ---------------------------------------------------------------- inversion


def invert_j2(j2: np.ndarray) -> np.ndarray:
    """Bisection for J_2^FD(x) = j2 on [X_LO, X_HI], clamped at the ends."""
    j2 = np.asarray(j2, dtype=np.float64)
    lo = np.full(j2.shape, X_LO)
    hi = np.full(j2.shape, X_HI)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        done = (mid == lo) | (mid == hi)
        if done.all():
            break
        up = _fd.j2_of_x(mid) < j2
        lo = np.where(up & ~done, mid, lo)
        hi = np.where(~up & ~done, mid, hi)
    x = 0.5 * (lo + hi)
    x = np.where(j2 >= _fd.j2_of_x(np.full(j2.shape, X_HI)), X_HI, x)
    x = np.where(j2 <= _fd.j2_of_x(np.full(j2.shape, X_LO)), X_LO, x)
    return x


def x_of_n_theta(n, theta):
    """x with 2 pi theta f_1(x) = n, f_1(x) = ln(1 + e^x): x = ln(e^a - 1),
    a = n/(2 pi theta), written as a + ln(1 - e^{-a}) (no overflow)."""
    a = np.asarray(n, dtype=np.float64) / (2.0 * math.pi * theta)
    return a + np.log(-np.expm1(-a))


# ---------------------------------------------------------------- equilibrium


def moment_set(n, j2, j4, stat: str = "fd", x=None) -> dict:
    """I_0..I_6 for the equilibrium.

    fd: I_0 = n and I_2 the FD value at the inverted x (theta = n t/(2 pi),
        t = 1/f_1(x)); I_4 and I_6 then follow from the measured J_2 and the
        inverted J_4 by the definition of J_L.  For an unclamped state these
        are the FD moments 2 pi theta^{N+1} f_{N+1}(x) themselves.
    t0: the theta = 0 limit of Eq. (sommerfeld), mu = n/(2 pi) for D = 2.
    mb: I_2N = n theta^N with theta = 1/3 (unit lattice velocity scale).
    """
    n = np.asarray(n, dtype=np.float64)
    if stat == "t0":
        mu = n / (2.0 * math.pi)
        return _g.moments_t0(mu, D, nmax=3)
    if stat == "mb":
        return _g.moments_mb(n, 1.0 / 3.0, nmax=3)
    theta = n / (2.0 * math.pi * _fd.fd(1, x))
    I0 = n
    I2 = 2.0 * math.pi * theta ** 2 * _fd.fd(2, x)
    I4 = I2 * I2 / (I0 * j2)
    I6 = I4 * I4 / (I2 * j4)
    return {0: I0, 2: I2, 4: I4, 6: I6}


def equilibrium_state(n, u0, j2, stat: str = "fd", x=None) -> np.ndarray:
    """f_eq for cells given n (C,), u0 (C, 2) and, for fd, j2 and x (C,)."""
    if stat == "fd":
        j4 = _fd.j4_of_x(x)
    else:
        j4 = None
    I = moment_set(n, j2, j4, stat, x)
    return _g.equilibrium(I, u0, D)


def init_equilibrium(n, ux, uy, t, stat: str = "fd") -> np.ndarray:
    """f[a, y, x] = f_eq(n, u0, t) on a field of (ny, nx) states."""
    n = np.asarray(n, dtype=np.float64)
    shape = n.shape
    nn = n.reshape(-1)
    u0 = np.stack([np.asarray(ux, dtype=np.float64).reshape(-1),
                   np.asarray(uy, dtype=np.float64).reshape(-1)], axis=-1)
    if stat in ("fd", "ft"):  # an FD equilibrium at the given t either way
        x = _fd.x_of_t(np.asarray(t, dtype=np.float64).reshape(-1))
        j2 = _fd.j2_of_x(x)
        feq = equilibrium_state(nn, u0, j2, "fd", x)
    else:
        feq = equilibrium_state(nn, u0, None, stat)
    return feq.T.reshape((Q,) + shape)


def collide(fin: np.ndarray, tau: float, stat: str = "fd", theta: float | None = None):
    """BGK collision of pulled populations fin[a, ...]; returns (f*, x).
    theta: the problem's constant theta for stat "ft"."""
    shape = fin.shape[1:]
    fl = fin.reshape(Q, -1)
    n, j, En = moments(fl)
    u0 = (j / n).T
    if stat == "fd":
        j2 = j2_from_moments(n, j, En)
        x = invert_j2(j2)
        feq = equilibrium_state(n, u0, j2, "fd", x)
    elif stat == "ft":
        x = x_of_n_theta(n, theta)
        feq = equilibrium_state(n, u0, _fd.j2_of_x(x), "fd", x)
    else:
        x = np.full(n.shape, np.nan)
        feq = equilibrium_state(n, u0, None, stat)
    fout = fl - (fl - feq.T) / tau
    return fout.reshape((Q,) + shape), x.reshape(shape)


def step(f: np.ndarray, p: Params) -> np.ndarray:
    fin = stream(f, p.bc_x, p.bc_y)
    out, _ = collide(fin, p.tau, p.stat, p.theta)
    return out


def run(f: np.ndarray, p: Params, nsteps: int) -> np.ndarray:
    for _ in range(nsteps):
        f = step(f, p)
    return f


# ---------------------------------------------------------------- reported fields


def fields(f: np.ndarray, stat: str = "fd") -> dict:
    """Macroscopic fields of a stored state: n, u0 (lattice units), J_2, x,
    t = T/T_F, T = theta and mu (dimensionless units of the paper).

    t = 1/f_1(x) (T_F is the theta = 0 chemical potential at the same n,
    T_F = n/(2 pi) for D = 2); theta = n t/(2 pi); mu = theta x.
    """
    n, j, En = moments(f)
    u0 = j / n
    j2 = j2_from_moments(n, j, En)
    out = {"n": n, "ux": u0[0], "uy": u0[1], "j2": j2}
    if stat == "fd":
        x = invert_j2(j2.reshape(-1)).reshape(n.shape)
        t = _fd.t_of_x(x)
        T = n * t / (2.0 * math.pi)
        out.update(x=x, t=t, T=T, mu=T * x)
    return out
