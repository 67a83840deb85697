"""Seeded synthetic workloads: the initial macroscopic states of the Riemann
problems, and nothing of the method.

This module is the only code that the CUDA library's callers and the CPU
oracle share.  It draws random numbers and lays out initial fields (density n,
lattice velocity u0 and t = T/T_F per cell); turning them into populations is
done separately by each side.

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style:
value(seed, i) = mix(seed + (i + 1) * 0x9E3779B97F4A7C15), and a double in
[0, 1) from the top 53 bits.

Workloads (the paper's experiments are synthetic: a stepwise Riemann problem
and a porous medium; these stand in for the benchmark cases built on them):

* ``riemann_1d``   quasi-1D step, 400 x 4, n = 1.0 | 0.8, t = 0.05, tau = 0.8,
                   bounce-back walls at the x ends, periodic in y;
* ``quadrants``    1024^2 four-quadrant problem, n ~ U[0.7, 1.0],
                   t ~ U[0.02, 0.1] per quadrant, tau = 0.6, periodic;
* ``smooth_t``     4096^2 density step at x = L/2 (1.0 | 0.8) with a smooth
                   temperature field from 8 random Fourier modes mapped
                   linearly onto t in [0.01, 0.2], periodic;
* ``batched``      256 quasi-1D problems, lengths log-uniform in [256, 8192],
                   widths uniform in 4..64, density ratio U[1.05, 2.0]
                   (right state n = 1), t ~ U[0.01, 0.2], tau ~ U[0.55, 1.0];
* ``surrogate_set`` (n, t) training pairs, n ~ U[0.5, 2], t log-uniform in
                   [0.005, 0.3].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """count SplitMix64 outputs for counters offset .. offset+count-1."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class Problem:
    """One lattice and its initial state (all arrays (ny, nx), float64)."""
    nx: int
    ny: int
    tau: float
    bc_x: str            # "periodic" | "bounceback"
    bc_y: str
    n: np.ndarray = field(repr=False)
    ux: np.ndarray = field(repr=False)
    uy: np.ndarray = field(repr=False)
    t: np.ndarray = field(repr=False)
    name: str = ""
    # compact description for the library's region-based initialisation
    kind: str = "field"  # "half" | "quadrant" | "field"
    states: list = field(default_factory=list)  # [(n, ux, uy, t), ...]
    split: tuple = (0, 0)                       # (x0, y0) of the regions

    @property
    def cells(self) -> int:
        return self.nx * self.ny


def _half(nx, ny, x0, left, right, tau, bc_x, bc_y, name) -> Problem:
    xs = np.arange(nx)
    L = xs < x0
    n = np.where(L, left[0], right[0])[None, :].repeat(ny, 0)
    ux = np.where(L, left[1], right[1])[None, :].repeat(ny, 0)
    uy = np.where(L, left[2], right[2])[None, :].repeat(ny, 0)
    t = np.where(L, left[3], right[3])[None, :].repeat(ny, 0)
    return Problem(nx, ny, tau, bc_x, bc_y, n.astype(np.float64), ux.astype(np.float64),
                   uy.astype(np.float64), t.astype(np.float64), name=name, kind="half",
                   states=[tuple(left), tuple(right)], split=(x0, 0))


def riemann_1d(nx: int = 400, ny: int = 4, n_left: float = 1.0, n_right: float = 0.8,
               t: float = 0.05, tau: float = 0.8, bc_x: str = "bounceback") -> Problem:
    """Quasi-1D Riemann step: left half n_left, right half n_right, u = 0."""
    return _half(nx, ny, nx // 2, (n_left, 0.0, 0.0, t), (n_right, 0.0, 0.0, t), tau,
                 bc_x, "periodic", f"riemann_1d_{nx}x{ny}")


def quadrants(L: int = 1024, seed: int = 1, tau: float = 0.6) -> Problem:
    """Four quadrants, n ~ U[0.7, 1.0], t ~ U[0.02, 0.1]; quadrant q has
    x >= L/2 for q in {1, 3} and y >= L/2 for q in {2, 3}."""
    r = uniform(seed, 8)
    ns = 0.7 + 0.3 * r[0:4]
    ts = 0.02 + 0.08 * r[4:8]
    xs = np.arange(L)
    qx = (xs >= L // 2).astype(int)
    q = qx[None, :] + 2 * qx[:, None]
    n = ns[q]
    t = ts[q]
    z = np.zeros((L, L))
    states = [(float(ns[k]), 0.0, 0.0, float(ts[k])) for k in range(4)]
    return Problem(L, L, tau, "periodic", "periodic", n, z, z.copy(), t,
                   name=f"quadrants_{L}", kind="quadrant", states=states, split=(L // 2, L // 2))


def fourier_modes(seed: int, count: int = 8):
    """Mode table (m, l, a, phi): integer wave numbers 1..4, a ~ U[0.5, 1],
    phi ~ U[0, 2 pi)."""
    r = uniform(seed, 4 * count)
    m = 1 + np.floor(4 * r[0:count]).astype(int)
    l = 1 + np.floor(4 * r[count:2 * count]).astype(int)
    a = 0.5 + 0.5 * r[2 * count:3 * count]
    phi = 2 * math.pi * r[3 * count:4 * count]
    return m, l, a, phi


def smooth_t_field(L: int, seed: int = 2, t_lo: float = 0.01, t_hi: float = 0.2,
                   rows: slice | None = None) -> np.ndarray:
    """t(y, x) = t_lo + (t_hi - t_lo)(s - min s)/(max s - min s),
    s = sum_k a_k cos(2 pi (m_k x + l_k y)/L + phi_k).  ``rows`` selects a
    band of rows (the normalisation always uses the whole lattice)."""
    m, l, a, phi = fourier_modes(seed)
    xs = np.arange(L, dtype=np.float64)
    # separable evaluation: cos(A + B) = cos A cos B - sin A sin B
    ys = xs if rows is None else xs[rows]

    def field_rows(yv):
        s = np.zeros((len(yv), L))
        for k in range(len(a)):
            ax = 2 * math.pi * m[k] * xs / L + phi[k]
            by = 2 * math.pi * l[k] * yv / L
            s += a[k] * (np.cos(by)[:, None] * np.cos(ax)[None, :] - np.sin(by)[:, None] * np.sin(ax)[None, :])
        return s

    # global extrema from the full field, evaluated in bands to bound memory
    smin, smax = np.inf, -np.inf
    for y0 in range(0, L, 512):
        s = field_rows(xs[y0:y0 + 512])
        smin = min(smin, s.min())
        smax = max(smax, s.max())
    s = field_rows(ys)
    return t_lo + (t_hi - t_lo) * (s - smin) / (smax - smin)


def smooth_t(L: int = 4096, seed: int = 2, tau: float = 0.8, t_lo: float = 0.01,
             t_hi: float = 0.2) -> Problem:
    """Density step at x = L/2 (1.0 | 0.8), smooth t field, u = 0, periodic."""
    t = smooth_t_field(L, seed, t_lo, t_hi)
    xs = np.arange(L)
    n = np.where(xs < L // 2, 1.0, 0.8)[None, :].repeat(L, 0)
    z = np.zeros((L, L))
    return Problem(L, L, tau, "periodic", "periodic", n, z, z.copy(), t,
                   name=f"smooth_t_{L}", kind="field")


@dataclass
class BatchSpec:
    nx: int
    ny: int
    n_left: float
    n_right: float
    t: float
    tau: float


def batched_specs(count: int = 256, seed: int = 3, lmin: int = 256, lmax: int = 8192,
                  wmin: int = 4, wmax: int = 64) -> list:
    """Per-problem sizes and states of the batched workload."""
    r = uniform(seed, 5 * count)
    out = []
    for p in range(count):
        u = r[5 * p:5 * p + 5]
        nx = int(round(math.exp(math.log(lmin) + u[0] * (math.log(lmax) - math.log(lmin)))))
        ny = wmin + int(math.floor(u[1] * (wmax - wmin + 1)))
        ratio = 1.05 + 0.95 * u[2]
        t = 0.01 + 0.19 * u[3]
        tau = 0.55 + 0.45 * u[4]
        out.append(BatchSpec(nx, min(ny, wmax), ratio, 1.0, t, tau))
    return out


def batched(count: int = 256, seed: int = 3, **kw) -> list:
    """The batched workload as Problem objects (quasi-1D steps split at nx/2,
    bounce-back at the x ends, periodic in y)."""
    probs = []
    for s in batched_specs(count, seed, **kw):
        probs.append(_half(s.nx, s.ny, s.nx // 2, (s.n_left, 0.0, 0.0, s.t),
                           (s.n_right, 0.0, 0.0, s.t), s.tau, "bounceback", "periodic",
                           f"batch_{s.nx}x{s.ny}"))
    return probs


def surrogate_set(count: int, seed: int = 4, n_lo: float = 0.5, n_hi: float = 2.0,
                  t_lo: float = 0.005, t_hi: float = 0.3):
    """(n, t) pairs: n ~ U[n_lo, n_hi], t log-uniform in [t_lo, t_hi]."""
    r = uniform(seed, 2 * count)
    n = n_lo + (n_hi - n_lo) * r[:count]
    t = np.exp(math.log(t_lo) + (math.log(t_hi) - math.log(t_lo)) * r[count:])
    return n, t


def random_field(nx: int, ny: int, seed: int, tau: float = 0.7, bc_x: str = "periodic",
                 bc_y: str = "periodic", n_lo: float = 0.7, n_hi: float = 1.2, u_max: float = 0.1,
                 t_lo: float = 0.02, t_hi: float = 0.3) -> Problem:
    """Per-cell random state: n ~ U[n_lo, n_hi], u0 ~ U[-u_max, u_max]^2,
    t ~ U[t_lo, t_hi] (test inputs spanning several tiles and ragged edges)."""
    c = nx * ny
    r = uniform(seed, 4 * c)
    n = (n_lo + (n_hi - n_lo) * r[:c]).reshape(ny, nx)
    ux = (u_max * (2 * r[c:2 * c] - 1)).reshape(ny, nx)
    uy = (u_max * (2 * r[2 * c:3 * c] - 1)).reshape(ny, nx)
    t = (t_lo + (t_hi - t_lo) * r[3 * c:]).reshape(ny, nx)
    return Problem(nx, ny, tau, bc_x, bc_y, n, ux, uy, t, name=f"random_{nx}x{ny}", kind="field")


def disc_centres(nx: int, ny: int, count: int, radius: int, seed: int) -> list:
    """Integer centres of `count` discs in an nx x ny periodic box, drawn
    uniformly (SplitMix64, seed) and rejected when closer than 2 radius + 1 to
    an earlier centre (periodic distance), so the discs neither overlap nor
    touch."""
    cx = np.empty(count, dtype=np.int64)
    cy = np.empty(count, dtype=np.int64)
    m = 0
    k = 0
    dmin2 = (2 * radius + 1) ** 2
    while m < count:
        if k > 10000 * count:
            raise ValueError("no room for the discs")
        r = uniform(seed, 2, offset=2 * k)
        k += 1
        x, y = min(int(r[0] * nx), nx - 1), min(int(r[1] * ny), ny - 1)
        if m:
            dx = np.abs(cx[:m] - x)
            dy = np.abs(cy[:m] - y)
            dx = np.minimum(dx, nx - dx)
            dy = np.minimum(dy, ny - dy)
            if np.any(dx * dx + dy * dy < dmin2):
                continue
        cx[m], cy[m] = x, y
        m += 1
    return list(zip(cx.tolist(), cy.tolist()))


def disc_mask(nx: int, ny: int, centres, radius: float) -> np.ndarray:
    """Solid mask (ny, nx) of discs: cell (x, y) is solid when its periodic
    distance to a centre is at most the radius."""
    solid = np.zeros((ny, nx), dtype=bool)
    R = int(np.floor(radius))
    oy, ox = np.meshgrid(np.arange(-R, R + 1), np.arange(-R, R + 1), indexing="ij")
    inside = ox * ox + oy * oy <= radius * radius
    oy, ox = oy[inside], ox[inside]
    for cx, cy in centres:
        solid[(cy + oy) % ny, (cx + ox) % nx] = True
    return solid


def porous_medium(nx: int = 700, ny: int = 150, count: int = 30, radius: int = 3, seed: int = 12,
                  tau: float = 0.7, n0: float = 1.0, t: float = 0.5):
    """The paper's porous sample: `count` discs of the given radius at seeded
    random positions in a periodic nx x ny box, fluid at rest with density
    n0 (and t = T/T_F for the FD closure).  Returns (Problem, solid mask)."""
    solid = disc_mask(nx, ny, disc_centres(nx, ny, count, radius, seed), radius)
    n = np.full((ny, nx), n0)
    z = np.zeros((ny, nx))
    p = Problem(nx, ny, tau, "periodic", "periodic", n, z, z.copy(), np.full((ny, nx), t),
                name=f"porous_{nx}x{ny}_{count}discs", kind="field")
    return p, solid


def perturb_populations(f: np.ndarray, seed: int, amp: float) -> np.ndarray:
    """Multiply populations by (1 + amp * U[-1, 1]) to leave equilibrium."""
    r = uniform(seed, f.size).reshape(f.shape)
    return f * (1.0 + amp * (2.0 * r - 1.0))


def surrogate_init(seed: int = 11, hidden: int = 64) -> np.ndarray:
    """Initial weights of the 2 -> H -> H -> 2 network (Glorot-uniform
    weights, zero biases), order W1, b1, W2, b2, W3, b3."""
    sizes = [(hidden, 2), (hidden, hidden), (2, hidden)]
    out = []
    off = 0
    for (fo, fi) in sizes:
        a = math.sqrt(6.0 / (fi + fo))
        out.append(a * (2.0 * uniform(seed, fo * fi, offset=off) - 1.0))
        off += fo * fi
        out.append(np.zeros(fo))
    return np.concatenate(out).astype(np.float32)
