"""Pins for oracle/gpoly.py: generalized polynomials, expansion coefficients,
quadrature and the K = 3 equilibrium.

The checks use brute-force 2D quadrature of the FD weight (polar coordinates,
Gauss-Legendre in xi^2/2 and a trapezoid rule in angle), textbook Hermite
polynomials for the Maxwell-Boltzmann limit, and the paper's printed closed
form of the d2v9 equilibrium.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import fd, gpoly as g

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_limits.json")
D = 2


def fd_weight_nodes(x, theta=1.0, M=32, panel=2.0, width=60.0, nodes=20):
    """Nodes xi (K, 2) and weights omega(xi) dA for the 2D FD weight
    omega = 1/(exp((xi^2/2 - mu)/theta) + 1), mu = x theta."""
    mu = x * theta
    gx, gw = np.polynomial.legendre.leggauss(nodes)
    smax = max(mu, 0.0) + width * theta
    s_nodes, s_w = [], []
    a = 0.0
    while a < smax:
        b = min(a + panel * theta, smax)
        s_nodes.append(a + 0.5 * (b - a) * (gx + 1))
        s_w.append(0.5 * (b - a) * gw)
        a = b
    s = np.concatenate(s_nodes)
    sw = np.concatenate(s_w)
    r = np.sqrt(2 * s)
    phi = 2 * math.pi * np.arange(M) / M
    R, PHI = np.meshgrid(r, phi, indexing="ij")
    W = (sw / (np.exp((s - mu) / theta) + 1.0))[:, None] * (2 * math.pi / M) * np.ones_like(PHI)
    xi = np.stack([R * np.cos(PHI), R * np.sin(PHI)], axis=-1).reshape(-1, 2)
    return xi, W.reshape(-1)


def moments_at(x, theta=1.0):
    return g.moments_fd(theta, np.array(x), D=2, nmax=4)


def perm_delta(a, b):
    """delta_{a|b}: the number of permutations matching index tuple a onto b."""
    if len(a) != len(b):
        return 0
    return sum(all(a[k] == b[p[k]] for k in range(len(a))) for p in itertools.permutations(range(len(a))))


@pytest.mark.parametrize("x", [-2.0, 0.5, 3.0, 20.0])
def test_gram_orthonormality_through_order_4(x):
    """Eq. (omeg-feq): int omega P_a P_b = delta_NM delta_{a|b}, P_0..P_4 with
    the coefficients printed after Eq. (H4) and Delta_L = +sqrt(Delta_L^2)."""
    I = moments_at(x)
    I[8] = 2 * math.pi * fd.fd(5, np.array(x))  # theta = 1
    coef = g.coefficients(I, D, kmax=4)
    xi, W = fd_weight_nodes(x)
    P = g.polynomials(xi, coef, D, kmax=4)
    comps = []
    for N in range(5):
        for idx in itertools.product(range(D), repeat=N):
            comps.append((idx, P[N][(slice(None),) + idx]))
    worst = 0.0
    for (ia, pa), (ib, pb) in itertools.combinations_with_replacement(comps, 2):
        val = np.sum(W * pa * pb)
        want = perm_delta(ia, ib) if len(ia) == len(ib) else 0
        worst = max(worst, abs(val - want))
    assert worst < 1e-11, worst


def test_gram_fails_with_wrong_reading():
    """The same check with Delta_L^2 in place of Delta_L in c'_K, cbar_K fails:
    the Gram test discriminates between the two readings of the printed formula."""
    x = 3.0
    I = moments_at(x)
    coef = g.coefficients(I, D, kmax=3)
    Dl2 = g.Delta2(I, 2, D)
    coef[("cp", 2)] = -coef[("c", 2)] * (I[2] / I[0]) * Dl2
    coef[("cb", 2)] = coef[("c", 2)] * (Dl2 - 1.0) / D
    xi, W = fd_weight_nodes(x)
    P = g.polynomials(xi, coef, D, kmax=3)
    # P_0 stays orthogonal to P_ij for any Delta; the norm of P_xx does not
    assert abs(np.sum(W * P[2][:, 0, 0] ** 2) - 2.0) > 1e-3
    good = g.polynomials(xi, g.coefficients(I, D, kmax=3), D, kmax=3)
    assert abs(np.sum(W * good[2][:, 0, 0] ** 2) - 2.0) < 1e-11


@pytest.mark.parametrize("x", [-1.5, 3.0, 20.0])
def test_expansion_coefficients_by_quadrature(x):
    """Eqs. (A0)-(A3) against A(u) = int omega(eta) P(eta + u) d eta, Eq. (expansao1)."""
    I = moments_at(x)
    coef = g.coefficients(I, D, kmax=3)
    xi, W = fd_weight_nodes(x)
    rng = np.random.default_rng(7)
    for _ in range(3):
        u = rng.uniform(-0.6, 0.6, 2)
        P = g.polynomials(xi + u, coef, D, kmax=3)
        num = [np.tensordot(W, p, axes=(0, 0)) for p in P]
        A = g.expansion_coefficients(u, I, coef, D)
        for N in range(4):
            np.testing.assert_allclose(num[N], A[N], rtol=1e-11, atol=1e-12 * float(np.sqrt(I[0])))


def test_expansion_at_zero_velocity():
    """Eq. (expansao2): A_N(0) = 0 for N > 0 and A_0 P_0 = 1."""
    I = moments_at(5.0)
    coef = g.coefficients(I, D, kmax=3)
    A = g.expansion_coefficients(np.zeros(2), I, coef, D)
    assert abs(A[0] * coef[("c", 0)] - 1.0) < 1e-15
    for N in (1, 2, 3):
        assert np.abs(A[N]).max() == 0.0


@pytest.mark.parametrize("x", [-2.0, 0.5, 3.0, 20.0, 200.0])
def test_quadrature_exact_to_degree_5(x):
    """Eq. (i2n-disc) with the d2v9 weights and c_0 = sqrt(3 I_4/I_2): exact for
    every monomial xi_x^p xi_y^q, p + q <= 5, and not for xi_x^6."""
    I = moments_at(x)
    J2 = g.J(I, 2)
    c0 = math.sqrt(3 * I[4] / I[2])
    w = g.weights(D, I[0], J2)
    xi = c0 * g.E_D2V9
    xq, Wq = fd_weight_nodes(x)
    for p in range(6):
        for q in range(6 - p):
            lat = np.sum(w * xi[:, 0] ** p * xi[:, 1] ** q)
            cont = np.sum(Wq * xq[:, 0] ** p * xq[:, 1] ** q)
            scale = I[2 * ((p + q + 1) // 2)] if p + q > 0 else I[0]
            assert abs(lat - cont) <= 1e-11 * scale, (p, q, lat, cont)
    lat6 = np.sum(w * xi[:, 0] ** 6)
    cont6 = np.sum(Wq * xq[:, 0] ** 6)
    assert abs(lat6 - cont6) > 1e-3 * cont6


def test_weights_formula_printed_in_paper():
    gold = json.load(open(GOLD))["weights"]
    assert gold["d2v9"]["w0"] == "I0 (1 - 5 J2/9)"
    w = g.weights(2, 2.0, 1.2)
    np.testing.assert_allclose(w, [2 * (1 - 5 * 1.2 / 9)] + [2 * 1.2 / 9] * 4 + [2 * 1.2 / 36] * 4)
    w1 = g.weights(1, 2.0, 1.2)
    np.testing.assert_allclose(w1, [2 * (1 - 1.2 / 3), 2 * 1.2 / 6, 2 * 1.2 / 6])


def hermite(xi):
    """Textbook D-dimensional Hermite tensors H_0..H_4 (Grad)."""
    d = np.eye(2)
    H0 = np.ones(xi.shape[:-1])
    H1 = xi
    H2 = np.einsum("...i,...j->...ij", xi, xi) - d
    H3 = np.einsum("...i,...j,...k->...ijk", xi, xi, xi) - g.sym_vec_delta(xi, 2)
    H4 = (np.einsum("...i,...j,...k,...l->...ijkl", xi, xi, xi, xi) - g.sym_vv_delta(xi, 2)
          + g.delta_all_pairings(2, 4))
    return [H0, H1, H2, H3, H4]


def test_mb_limit_gives_hermite_polynomials():
    """MB weight, I_2N = I_0 theta^N: P = H(xi/sqrt(theta))/sqrt(I_0)."""
    gold = json.load(open(GOLD))["gaussian_limit_coefficients"]
    I0, theta = 1.7, 0.6
    I = g.moments_mb(I0, theta, nmax=5)
    coef = g.coefficients(I, D, kmax=4)
    rng = np.random.default_rng(3)
    xi = rng.normal(size=(10, 2))
    P = g.polynomials(xi, coef, D, kmax=4)
    H = hermite(xi / math.sqrt(theta))
    for N in range(5):
        np.testing.assert_allclose(P[N], H[N] / math.sqrt(I0), rtol=1e-13, atol=1e-13)
    # Gaussian limit I_2N = 1: the printed coefficient values
    c = g.coefficients(g.moments_mb(1.0, 1.0, nmax=5), D, kmax=4)
    for K in range(5):
        assert abs(c[("c", K)] - gold["c_K"]) < 1e-15
    for K in range(2, 5):
        assert abs(abs(c[("cp", K)]) - gold["abs_cprime_K"]) < 1e-15
        assert abs(c[("cb", K)] - gold["cbar_K"]) < 1e-15
    assert abs(abs(c[("d", 4)]) - gold["abs_d4"]) < 1e-15
    assert abs(c[("db", 4)] - gold["dbar_4"]) < 1e-15
    assert abs(c[("dp", 4)] - gold["dprime_4"]) < 1e-15


def test_mb_limit_equilibrium_is_standard_d2q9():
    """J_2 = J_4 = 1: f_eq = w (1 + 3eu + 9/2 eu^2 - 3/2 u^2 + 9/2 eu^3 - 9/2 eu u^2)
    with w = (4/9, 1/9, 1/36) n, the third-order Hermite D2Q9 equilibrium."""
    rng = np.random.default_rng(11)
    C = 16
    n = rng.uniform(0.5, 2, C)
    u0 = rng.uniform(-0.3, 0.3, (C, 2))
    I = g.moments_mb(n, 1.0 / 3.0, nmax=3)
    f = g.equilibrium(I, u0, D)
    e = g.E_D2V9
    eu = u0 @ e.T
    u2 = (u0 * u0).sum(1)[:, None]
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[None, :] * n[:, None]
    ref = w * (1 + 3 * eu + 4.5 * eu ** 2 - 1.5 * u2 + 4.5 * eu ** 3 - 4.5 * eu * u2)
    np.testing.assert_allclose(f, ref, rtol=1e-13)


def fd_states(C, seed=5, xlo=-2.0, xhi=60.0, umax=0.25):
    rng = np.random.default_rng(seed)
    x = rng.uniform(xlo, xhi, C)
    n = rng.uniform(0.5, 2.0, C)
    theta = n / (2 * math.pi * fd.fd(1, x))
    I = g.moments_fd(theta, x, D=2, nmax=3)
    u0 = rng.uniform(-umax, umax, (C, 2))
    return n, x, I, u0


def test_closed_form_equals_tensor_contraction():
    """The printed geometric-velocity K = 3 equilibrium equals the tensor
    contraction of Eq. (expansao0) with Eqs. (H0)-(H3), (A0)-(A3)."""
    n, x, I, u0 = fd_states(64)
    ft = g.equilibrium(I, u0, D)
    fc = g.feq_closed_form(n, u0, g.J(I, 2), g.J(I, 4), D)
    np.testing.assert_allclose(ft, fc, rtol=1e-13, atol=1e-15)


def test_equilibrium_moments():
    """Sum f_eq = n, sum f_eq e = n u0, sum f_eq e e = n (u0 u0 + J_2 delta/3) for
    any u0 (moments of the continuous f_eq(xi - u) up to second order; the
    quadrature is exact to degree 5 and S is of degree 3)."""
    n, x, I, u0 = fd_states(64, seed=9)
    f = g.equilibrium(I, u0, D)
    e = g.E_D2V9
    J2 = g.J(I, 2)
    np.testing.assert_allclose(f.sum(1), n, rtol=1e-14)
    np.testing.assert_allclose(f @ e, n[:, None] * u0, rtol=1e-13, atol=1e-15)
    for i in range(2):
        for j in range(2):
            m = (f * e[None, :, i] * e[None, :, j]).sum(1)
            np.testing.assert_allclose(m, n * (u0[:, i] * u0[:, j] + (i == j) * J2 / 3), rtol=1e-13)


def test_equilibrium_at_rest_is_weights():
    n, x, I, _ = fd_states(16)
    f = g.equilibrium(I, np.zeros((16, 2)), D)
    np.testing.assert_allclose(f, g.weights(D, n, g.J(I, 2)), rtol=1e-15)


def test_zero_temperature_weights_printed_vs_formula():
    """At theta = 0 the paper prints d2v9 weights (3/5, 1/30, 2/15) I_0 and
    d1v3 weights (7/12, 5/24) I_0; these do not follow from its own weight
    formulas at J_2 = 1 + 2/(2 + D) (they do not even sum to I_0 for d2v9).
    The formulas give (1/6, 1/24, 1/6) and (1/2, 1/4); the formulas are used."""
    gold = json.load(open(GOLD))["zero_temperature"]
    pw = gold["printed_weights_d2v9"]
    assert abs(pw["w0_over_I0"] + 4 * pw["wl_over_I0"] + 4 * pw["ws_over_I0"] - 1.0) > 0.2
    I = g.moments_t0(1.0, 2, nmax=3)
    J2 = g.J(I, 2)
    assert abs(J2 - 1.5) < 1e-15
    w = g.weights(2, 1.0, J2)
    np.testing.assert_allclose(w[[0, 5, 1]], [1 / 6, 1 / 24, 1 / 6], rtol=1e-15)
    I1 = g.moments_t0(1.0, 1, nmax=3)
    J21 = g.J(I1, 2)
    assert abs(J21 - (1 + 2 / 3)) < 1e-15
    np.testing.assert_allclose(g.weights(1, 1.0, J21)[:2], [4 / 9, 5 / 18], rtol=1e-15)
    # the printed d1v3 weights are the formula at J_2 = 5/4 instead
    np.testing.assert_allclose(g.weights(1, 1.0, 1.25)[:2],
                               [gold["printed_weights_d1v3"]["w0_over_I0"],
                                gold["printed_weights_d1v3"]["w1_over_I0"]], rtol=1e-15)


def test_zero_temperature_velocity_scale():
    """theta = 0: c_0 = sqrt(3 I_4/I_2) = sqrt(6 mu/(D + 4)) and I_0 = (2 pi mu)^{D/2}/Gamma(D/2+1)."""
    for Dd in (1, 2):
        mu = 0.37
        I = g.moments_t0(mu, Dd, nmax=3)
        assert abs(math.sqrt(3 * I[4] / I[2]) - math.sqrt(6 * mu / (Dd + 4))) < 1e-15
        assert abs(I[0] - (2 * math.pi * mu) ** (Dd / 2) / math.gamma(Dd / 2 + 1)) < 1e-15


def test_expansion_domain_is_where_delta2_is_positive():
    """The polynomials need Delta_L = +sqrt(Delta_L^2) real (definitions under
    Eq. (H4)) and a real lattice scale c_0 = sqrt(3 I_4/I_2) (Sect. "The
    Gaussian quadrature").  With I_4 = I_2^2/(I_0 J_2), Delta_2^2 = 1/(2 - J_2)
    for D = 2, so the K = 3 equilibrium exists for 0 < J_2 < 2 only.  Inside:
    every coefficient and population is finite over the FD range the tests and
    workloads use; outside: every population is NaN, set explicitly (no
    floating-point warning is raised on the way)."""
    import warnings

    from oracle import lbm as olbm

    rng = np.random.default_rng(7)
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        # FD states: n in [0.5, 2], t from the clamp's low end to its high end
        for t in (1e-3, 5e-3, 0.02, 0.05, 0.1, 0.3, 1.0, 10.0):
            n = rng.uniform(0.5, 2.0, 16)
            x = fd.x_of_t(np.full(16, t))
            j2 = fd.j2_of_x(x)
            I = olbm.moment_set(n, j2, fd.j4_of_x(x), "fd", x)
            coef = g.coefficients(I, D, kmax=3)
            assert all(np.isfinite(v).all() for v in coef.values())
            assert g.in_expansion_domain(I, D).all()
            u0 = rng.uniform(-0.3, 0.3, (16, 2))
            assert np.isfinite(g.equilibrium(I, u0, D)).all()
        # measured J_2 on either side of the boundaries (x of a mid-range FD state)
        x = fd.x_of_t(np.full(6, 0.05))
        j2 = np.array([1.999, 1.9, 2.0, 2.3, 5.0, -0.1])
        I = olbm.moment_set(np.ones(6), j2, fd.j4_of_x(x), "fd", x)
        feq = g.equilibrium(I, np.full((6, 2), 0.01), D)
    inside = np.array([True, True, False, False, False, False])
    assert np.array_equal(g.in_expansion_domain(I, D), inside)
    assert np.isfinite(feq[inside]).all()
    assert np.isnan(feq[~inside]).all()
    # just inside, the tensor form still equals the printed closed form
    ref = g.feq_closed_form(np.ones(2), np.full((2, 2), 0.01), j2[:2], fd.j4_of_x(x[:2]), D)
    np.testing.assert_allclose(feq[:2], ref, rtol=1e-12, atol=0)
