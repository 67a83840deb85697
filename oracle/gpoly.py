"""Generalized orthonormal polynomials, expansion coefficients and the
discrete K = 3 equilibrium, in FP64 tensor form.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Everything here is written from the paper's definitions, term by term, with
full index tensors (no closed-form shortcuts):

* isotropic moments ``I_2N`` of the weight, Eqs. (i2n-cont), (i2n-cont2), and
  for FD ``I_2N = (2 pi)^{D/2} theta^{N+D/2} f_{N+D/2}(x)``;
* ``J_L = I_L^2/(I_{L+2} I_{L-2})``, ``Delta_L^2 = 2/[(D+L) - J_L (D+L-2)]``,
  ``delta_L = 2 I_{L+2} I_{L-2}/Delta_L^2`` (definitions under Eq. (H4));
* polynomial coefficients ``c_K = I_2K^{-1/2}``,
  ``c'_K = -c_K (I_{2K-2}/I_{2K-4}) Delta_{2K-2}``,
  ``cbar_K = c_K (Delta_{2K-2} - 1)/(D + 2K - 4)`` and ``d_4, d'_4, dbar_4``;
* polynomials ``P_0 .. P_4``, Eqs. (H0)-(H4);
* expansion coefficients ``A_0 .. A_3``, Eqs. (A0)-(A3);
* the d1v3 / d2v9 Gaussian-quadrature lattices and weights, Sect. "The
  Gaussian quadrature";
* the discrete equilibrium ``f_eq,a = w_a sum_{N<=3} (1/N!) A(u) . P(xi_a)``,
  Eq. (expansao0) evaluated at the lattice nodes ``xi_a = c_0 e_a``,
  ``c_0 = sqrt(3 I_4/I_2)``.

Readings of garbled or ambiguous passages:

* ``Delta_L`` is the positive square root of ``Delta_L^2``.
* The polynomials, and with them the expansion, exist only where every
  ``Delta_L^2`` used is positive and finite and ``c_0^2 = 3 I_4/I_2`` is
  positive.  For the K = 3 equilibrium built from moments with ratios J_2 and
  J_4 this is 0 < J_2 < 2 and J_4 < 3/2 (D = 2).  A state outside (reachable
  only through measured moments, never from an FD weight) has no real
  polynomials: ``equilibrium`` returns NaN for it, explicitly, and
  ``in_expansion_domain`` says which states those are.
* ``c'_1 = cbar_1 = 0`` (Eq. (H1) has no lower-order part).
* The constant ``c_0`` of Eq. (H0) is ``c_{K=0} = I_0^{-1/2}``; the velocity
  scale of the lattice is the separate ``c_0 = sqrt(3 I_4/I_2)``.
* ``delta_{i1..i2N}`` is the sum over all (2N-1)!! pairings of the indices.
* The d2v9 long vectors are the four diagonals (1,1), (-1,1), (-1,-1), (1,-1).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import fd as _fd

# ---------------------------------------------------------------- lattices

# d2v9: rest; short (1,0),(0,1),(-1,0),(0,-1); long (1,1),(-1,1),(-1,-1),(1,-1)
E_D2V9 = np.array(
    [[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]],
    dtype=np.float64,
)
OPP_D2V9 = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])
E_D1V3 = np.array([[0], [1], [-1]], dtype=np.float64)
OPP_D1V3 = np.array([0, 2, 1])


def lattice(D: int):
    """(e_a, opposite index) of the paper's lattice for dimension D."""
    if D == 2:
        return E_D2V9, OPP_D2V9
    if D == 1:
        return E_D1V3, OPP_D1V3
    raise ValueError("only d1v3 and d2v9 are defined in the paper")


def weights(D: int, I0, J2):
    """Quadrature weights w_a(I_0, J_2), Sect. "The Gaussian quadrature".

    d1v3: w_0 = I_0 (1 - J_2/3), w_{+-1} = I_0 J_2/6.
    d2v9: w_0 = I_0 (1 - 5 J_2/9), w_short = I_0 J_2/9, w_long = I_0 J_2/36.
    Returns an array with the velocity index last.
    """
    I0 = np.asarray(I0, dtype=np.float64)
    J2 = np.asarray(J2, dtype=np.float64)
    if D == 1:
        ws = I0 * J2 / 6.0
        return np.stack([I0 * (1.0 - J2 / 3.0), ws, ws], axis=-1)
    w0 = I0 * (1.0 - 5.0 * J2 / 9.0)
    wsh = I0 * J2 / 9.0
    wl = I0 * J2 / 36.0
    return np.stack([w0, wsh, wsh, wsh, wsh, wl, wl, wl, wl], axis=-1)


# ---------------------------------------------------------------- moments


def moments_fd(theta, x, D: int = 2, nmax: int = 4) -> dict:
    """I_0, I_2, ..., I_{2 nmax} of the FD weight (D = 2: integer orders)."""
    if D != 2:
        raise ValueError("the integer-order FD moments here are for D = 2")
    theta = np.asarray(theta, dtype=np.float64)
    return {
        2 * N: 2.0 * math.pi * theta ** (N + 1) * _fd.fd(N + 1, x)
        for N in range(nmax + 1)
    }


def moments_mb(rho0, theta, nmax: int = 4) -> dict:
    """MB weight: I_2N = I_0 theta^N (Sect. "Generalized polynomials")."""
    rho0 = np.asarray(rho0, dtype=np.float64)
    return {2 * N: rho0 * np.asarray(theta, dtype=np.float64) ** N for N in range(nmax + 1)}


def moments_t0(mu, D: int, nmax: int = 4) -> dict:
    """theta = 0 limit of Eq. (sommerfeld): I_2N = (2pi)^{D/2} mu^{N+D/2} / Gamma(N+D/2+1)."""
    mu = np.asarray(mu, dtype=np.float64)
    return {
        2 * N: (2.0 * math.pi) ** (D / 2.0) * mu ** (N + D / 2.0) / math.gamma(N + D / 2.0 + 1.0)
        for N in range(nmax + 1)
    }


def J(I: dict, L: int):
    """J_L = I_L^2 / (I_{L+2} I_{L-2})."""
    return I[L] ** 2 / (I[L + 2] * I[L - 2])


def Delta2(I: dict, L: int, D: int):
    """Delta_L^2 = 2 / [(D+L) - J_L (D+L-2)]."""
    return 2.0 / ((D + L) - J(I, L) * (D + L - 2))


def sqrt_domain(d2):
    """Delta_L = +sqrt(Delta_L^2) where Delta_L^2 is positive and finite; NaN
    where it is not (no real polynomial exists there), without a warning."""
    d2 = np.asarray(d2, dtype=np.float64)
    ok = np.isfinite(d2) & (d2 > 0.0)
    return np.sqrt(np.where(ok, d2, 1.0)) * np.where(ok, 1.0, np.nan)


def in_expansion_domain(I: dict, D: int, kmax: int = 3):
    """True where the K = kmax expansion exists: Delta_2^2 .. Delta_{2 kmax - 2}^2
    positive and finite, and I_4/I_2 > 0 (a real lattice scale c_0)."""
    ok = np.ones(np.shape(I[0]), dtype=bool)
    with np.errstate(divide="ignore", invalid="ignore"):
        for K in range(2, kmax + 1):
            d2 = Delta2(I, 2 * K - 2, D)
            ok &= np.isfinite(d2) & (d2 > 0.0)
        ok &= np.asarray(I[4] / I[2]) > 0.0
    return ok


def small_delta(I: dict, L: int, D: int):
    """delta_L = 2 I_{L+2} I_{L-2} / Delta_L^2."""
    return 2.0 * I[L + 2] * I[L - 2] / Delta2(I, L, D)


# ---------------------------------------------------------------- coefficients


def coefficients(I: dict, D: int, kmax: int = 3, d4_sign: float = 1.0) -> dict:
    """c_K, c'_K, cbar_K (K <= kmax) and, for kmax = 4, d_4, d'_4, dbar_4."""
    c = {}
    for K in range(kmax + 1):
        c[("c", K)] = 1.0 / sqrt_domain(I[2 * K])
    c[("cp", 1)] = 0.0 * c[("c", 1)]
    c[("cb", 1)] = 0.0 * c[("c", 1)]
    for K in range(2, kmax + 1):
        with np.errstate(divide="ignore"):
            Dl = sqrt_domain(Delta2(I, 2 * K - 2, D))
        c[("cp", K)] = -c[("c", K)] * (I[2 * K - 2] / I[2 * K - 4]) * Dl
        c[("cb", K)] = c[("c", K)] * (Dl - 1.0) / (D + 2 * K - 4)
    if kmax >= 4:
        d2 = small_delta(I, 2, D)
        d4 = small_delta(I, 4, D)
        d6 = small_delta(I, 6, D)
        D6 = np.sqrt(Delta2(I, 6, D))
        c4 = c[("c", 4)]
        dd4 = d4_sign * np.sqrt(8.0 * d4 ** 2 * I[4] / (d2 * (d2 * d6 * (D + 4) - d4 ** 2 * D)))
        c[("d", 4)] = dd4
        c[("dp", 4)] = -(dd4 / D) * (I[0] / I[2] + I[4] * d2 / (I[2] * d4)) + 2.0 * c4 * I[6] * D6 / (D * I[4])
        c[("db", 4)] = dd4 * d2 / (D * (D + 2) * d4) + c4 * (D - 2 * (D + 2) * D6) / (D * (D + 2) * (D + 4))
    return c


# ---------------------------------------------------------------- tensors


def kron(D: int) -> np.ndarray:
    return np.eye(D)


def delta_all_pairings(D: int, order: int) -> np.ndarray:
    """delta_{i1..i_order}: sum over all pairings of products of Kronecker deltas."""
    shape = (D,) * order
    out = np.zeros(shape)
    for idx in itertools.product(range(D), repeat=order):
        out[idx] = _count_pairings(list(idx))
    return out


def _count_pairings(idx: list) -> int:
    if not idx:
        return 1
    first, rest = idx[0], idx[1:]
    total = 0
    for k in range(len(rest)):
        if rest[k] == first:
            total += _count_pairings(rest[:k] + rest[k + 1:])
    return total


def sym_vec_delta(v: np.ndarray, D: int) -> np.ndarray:
    """v_i delta_jk + v_j delta_ik + v_k delta_ij for v of shape (..., D)."""
    d = kron(D)
    return (
        np.einsum("...i,jk->...ijk", v, d)
        + np.einsum("...j,ik->...ijk", v, d)
        + np.einsum("...k,ij->...ijk", v, d)
    )


def sym_vv_delta(v: np.ndarray, D: int) -> np.ndarray:
    """The six-term v v delta tensor of Eq. (H4)."""
    d = kron(D)
    return (
        np.einsum("...i,...j,kl->...ijkl", v, v, d)
        + np.einsum("...i,...k,jl->...ijkl", v, v, d)
        + np.einsum("...i,...l,jk->...ijkl", v, v, d)
        + np.einsum("...j,...k,il->...ijkl", v, v, d)
        + np.einsum("...j,...l,ik->...ijkl", v, v, d)
        + np.einsum("...k,...l,ij->...ijkl", v, v, d)
    )


def _b(a, nextra: int):
    """Broadcast a per-state coefficient against nextra trailing tensor axes."""
    a = np.asarray(a, dtype=np.float64)
    return a.reshape(a.shape + (1,) * nextra)


def polynomials(xi: np.ndarray, coef: dict, D: int, kmax: int = 3) -> list:
    """[P_0, P_{i}, P_{ij}, P_{ijk}(, P_{ijkl})] at xi (shape (..., D)),
    Eqs. (H0)-(H4).  Coefficient arrays broadcast against xi's leading axes."""
    xi = np.asarray(xi, dtype=np.float64)
    lead = xi.shape[:-1]
    xi2 = np.sum(xi * xi, axis=-1)
    d = kron(D)
    P = [np.broadcast_to(_b(coef[("c", 0)], 0), lead).copy()]
    P.append(_b(coef[("c", 1)], 1) * xi)
    P.append(
        _b(coef[("c", 2)], 2) * np.einsum("...i,...j->...ij", xi, xi)
        + _b(coef[("cb", 2)] * xi2 + coef[("cp", 2)], 2) * d
    )
    P.append(
        _b(coef[("c", 3)], 3) * np.einsum("...i,...j,...k->...ijk", xi, xi, xi)
        + _b(coef[("cb", 3)] * xi2 + coef[("cp", 3)], 3) * sym_vec_delta(xi, D)
    )
    if kmax >= 4:
        d4t = delta_all_pairings(D, 4)
        P.append(
            _b(coef[("c", 4)], 4) * np.einsum("...i,...j,...k,...l->...ijkl", xi, xi, xi, xi)
            + _b(coef[("cb", 4)] * xi2 + coef[("cp", 4)], 4) * sym_vv_delta(xi, D)
            + _b(coef[("db", 4)] * xi2 ** 2 + coef[("dp", 4)] * xi2 + coef[("d", 4)], 4) * d4t
        )
    return P


def expansion_coefficients(u: np.ndarray, I: dict, coef: dict, D: int) -> list:
    """[A_0, A_i, A_ij, A_ijk](u), Eqs. (A0)-(A3); u has shape (..., D)."""
    u = np.asarray(u, dtype=np.float64)
    u2 = np.sum(u * u, axis=-1)
    I0 = np.asarray(I[0], dtype=np.float64)
    J2 = J(I, 2)
    d = kron(D)
    A0 = I0 * coef[("c", 0)] * np.ones_like(u2)
    A1 = _b(I0 * coef[("c", 1)], 1) * u
    A2 = _b(I0, 2) * (
        _b(coef[("c", 2)], 2) * np.einsum("...i,...j->...ij", u, u) + _b(coef[("cb", 2)] * u2, 2) * d
    )
    A3 = _b(I0, 3) * (
        _b(coef[("c", 3)], 3) * np.einsum("...i,...j,...k->...ijk", u, u, u)
        + _b(coef[("cp", 3)] * (1.0 - J2) + coef[("cb", 3)] * u2, 3) * sym_vec_delta(u, D)
    )
    return [A0, A1, A2, A3]


def equilibrium(I: dict, u0: np.ndarray, D: int) -> np.ndarray:
    """Discrete K = 3 equilibrium f_eq,a for a batch of states.

    I: dict of arrays I_0..I_6 with shape (C,); u0: lattice velocity u/c_0,
    shape (C, D).  Returns (C, Q).

    Eq. (expansao0) with the weight replaced by the quadrature weights at the
    nodes: f_eq,a = w_a * sum_{N=0}^{3} (1/N!) A_{i1..iN}(u) P_{i1..iN}(xi_a),
    xi_a = c_0 e_a, u = c_0 u0, c_0 = sqrt(3 I_4/I_2).
    """
    e, _ = lattice(D)
    coef = coefficients(I, D, kmax=3)
    c0 = sqrt_domain(3.0 * I[4] / I[2])  # (C,); NaN outside the expansion's domain
    u = c0[:, None] * np.asarray(u0, dtype=np.float64)
    xi = c0[:, None, None] * e[None, :, :]  # (C, Q, D)
    # broadcast coefficients over the velocity axis
    coef_q = {k: np.asarray(v)[:, None] if np.ndim(v) else v for k, v in coef.items()}
    P = polynomials(xi, coef_q, D, kmax=3)
    A = expansion_coefficients(u, I, coef, D)
    S = A[0][:, None] * P[0]
    S = S + np.einsum("ci,cqi->cq", A[1], P[1])
    S = S + 0.5 * np.einsum("cij,cqij->cq", A[2], P[2])
    S = S + (1.0 / 6.0) * np.einsum("cijk,cqijk->cq", A[3], P[3])
    w = weights(D, I[0], J(I, 2))
    out = w * S
    # a state outside the domain gets NaN in every population, explicitly
    out[~in_expansion_domain(I, D, kmax=3)] = np.nan
    return out


def feq_closed_form(n, u0, J2, J4, D: int) -> np.ndarray:
    """The K = 3 equilibrium in geometric velocities as printed in Sect. "The
    Gaussian quadrature" (used ONLY by tests, to check it against the tensor
    contraction above)."""
    e, _ = lattice(D)
    n = np.asarray(n, dtype=np.float64)[:, None]
    u0 = np.asarray(u0, dtype=np.float64)
    J2 = np.asarray(J2, dtype=np.float64)[:, None]
    J4 = np.asarray(J4, dtype=np.float64)[:, None]
    D22 = 2.0 / ((D + 2) - J2 * D)
    D42 = 2.0 / ((D + 4) - J4 * (D + 2))
    eu = u0 @ e.T  # (C, Q)
    u2 = np.sum(u0 * u0, axis=-1)[:, None]
    e2 = np.sum(e * e, axis=-1)[None, :]
    w = weights(D, n[:, 0], J2[:, 0])
    br = (
        (1 - J2) * J4 * (D + 2) * D42
        - 3 * (1 - J2) * J4 * D42 * e2
        - 3 * J4 * D42 * u2
        + 9 * J4 * (D42 - 1) / (D + 2) * u2 * e2
        + 3 * J4 * eu ** 2
    )
    S = (
        1
        + 3 / J2 * eu
        + 9 / (2 * J2) * eu ** 2
        + 4.5 * (D22 - 1) / (J2 * D) * u2 * e2
        - 1.5 * D22 * u2
        + 3 / (2 * J2) * eu * br
    )
    return w * S
