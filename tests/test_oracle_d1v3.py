"""Pins of the d1v3 oracle (oracle/lbm1d.py) against what the paper and the
mathematics fix: the zero-temperature weight's moments by direct integration,
quadrature exactness to degree 5, the equilibrium's moments, the printed
closed form against the tensor contraction, the Maxwell-Boltzmann limit as the
textbook D1Q3 equilibrium, conservation, and the paper's Riemann run (Fig. 1)
on d1v3 against the exact isothermal solution."""
import math

import numpy as np
import pytest

from oracle import gpoly as g
from oracle import lbm1d, riemann


def test_zero_temperature_moments_by_integration():
    """At theta = 0 the D = 1 FD weight is uniform on |xi| < a, a = sqrt(2 mu).
    With I_2N the coefficient of the isotropic tensor (Eq. (i2n-cont2)),
    int omega xi^{2N} dxi = (2N - 1)!! I_2N.  The uniform weight of mass n
    gives int xi^{2N} = n a^{2N}/(2N + 1); mu = n^2/8 makes I_0 = n."""
    for n in (0.85, 1.0, 1.7):
        mu = n * n / 8.0
        a2 = 2.0 * mu
        I = lbm1d.moment_set(np.array([n]), "t0")
        for N, dfact in ((0, 1), (1, 1), (2, 3), (3, 15)):
            assert abs(dfact * I[2 * N][0] - n * a2 ** N / (2 * N + 1)) < 1e-15 * n


def test_quadrature_exact_to_degree_5():
    """sum_a w_a (c_0 e_a)^p equals the uniform weight's p-th moment for
    p <= 5 and misses p = 6."""
    n = 0.93
    I = lbm1d.moment_set(np.array([n]), "t0")
    J2 = I[2] ** 2 / (I[0] * I[4])
    w = g.weights(1, I[0], J2)[0]
    c0 = math.sqrt(3.0 * I[4][0] / I[2][0])
    a = math.sqrt(n * n / 4.0)
    for p in range(6):
        lat = float(np.sum(w * (c0 * lbm1d.E) ** p))
        cont = 0.0 if p % 2 else n * a ** p / (p + 1)
        assert abs(lat - cont) < 1e-14, p
    lat6 = float(np.sum(w * (c0 * lbm1d.E) ** 6))
    assert abs(lat6 - n * a ** 6 / 7) > 1e-3 * n * a ** 6


def test_zero_temperature_constants():
    """J_N = 1 + 2/(N + D) and Delta_N^2 = (D + N)/2 for D = 1 (Sect.
    "Numerical simulations")."""
    I = lbm1d.moment_set(np.array([1.3]), "t0")
    assert abs(g.J(I, 2)[0] - 5.0 / 3.0) < 1e-14
    assert abs(g.J(I, 4)[0] - 7.0 / 5.0) < 1e-14
    assert abs(g.Delta2(I, 2, 1)[0] - 1.5) < 1e-13
    assert abs(g.Delta2(I, 4, 1)[0] - 2.5) < 1e-13


def states(count, seed):
    r = np.random.default_rng(seed)
    return r.uniform(0.6, 1.6, count), r.uniform(-0.2, 0.2, count)


@pytest.mark.parametrize("stat", ["t0", "mb"])
def test_equilibrium_moments(stat):
    """sum f_eq = n, sum f_eq e = n u0, sum f_eq e^2 = n (u0^2 + J_2/3)."""
    n, u = states(64, 1)
    f = lbm1d.equilibrium(n, u, stat)
    J2 = 5.0 / 3.0 if stat == "t0" else 1.0
    np.testing.assert_allclose(f.sum(0), n, rtol=1e-14)
    np.testing.assert_allclose(f[1] - f[2], n * u, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(f[1] + f[2], n * (u * u + J2 / 3.0), rtol=1e-13)


@pytest.mark.parametrize("stat", ["t0", "mb"])
def test_closed_form_equals_tensor_contraction(stat):
    n, u = states(64, 2)
    J2, J4 = (5.0 / 3.0, 7.0 / 5.0) if stat == "t0" else (1.0, 1.0)
    ft = lbm1d.equilibrium(n, u, stat).T
    fc = g.feq_closed_form(n, u[:, None], np.full(64, J2), np.full(64, J4), 1)
    np.testing.assert_allclose(ft, fc, rtol=1e-13, atol=1e-15)


def test_mb_limit_is_textbook_d1q3():
    """theta = 1/3, J = Delta = 1: weights (2/3, 1/6, 1/6) and
    f_eq = w n (1 + 3 e u + 9/2 (e u)^2 - 3/2 u^2); the third-order Hermite
    term (e^3 - e) u^3 vanishes on the nodes e in {0, +1, -1}."""
    n, u = states(32, 3)
    f = lbm1d.equilibrium(n, u, "mb")
    for a, (e, w) in enumerate(zip(lbm1d.E, (2 / 3, 1 / 6, 1 / 6))):
        ref = w * n * (1 + 3 * e * u + 4.5 * (e * u) ** 2 - 1.5 * u * u)
        np.testing.assert_allclose(f[a], ref, rtol=1e-13)


@pytest.mark.parametrize("stat", ["t0", "mb"])
def test_collision_conserves_mass_and_momentum(stat):
    r = np.random.default_rng(4)
    n, u = states(200, 4)
    f = lbm1d.equilibrium(n, u, stat) * (1 + 0.05 * r.standard_normal((3, 200)))
    fc = lbm1d.collide(f, 0.7, stat)
    n0, j0 = lbm1d.moments(f)
    n1, j1 = lbm1d.moments(fc)
    np.testing.assert_allclose(n1, n0, rtol=1e-14)
    np.testing.assert_allclose(j1, j0, rtol=1e-12, atol=1e-15)


def test_uniform_state_is_fixed_and_walls_keep_mass():
    f = lbm1d.equilibrium(np.full(50, 0.9), np.full(50, 0.05), "t0")
    np.testing.assert_allclose(lbm1d.step(f, 0.8, "t0"), f, rtol=1e-14)
    xs = np.arange(60)
    f = lbm1d.equilibrium(np.where(xs < 20, 1.0, 0.8), np.zeros(60), "t0")
    m0 = f.sum()
    f = lbm1d.run(f, 0.8, "t0", 200, "bounceback")
    assert abs(f.sum() - m0) < 1e-12 * m0


def test_paper_riemann_run_d1v3():
    """Fig. 1 on d1v3: 3001 nodes periodic, n = 1.0 for L/4 < x < 3L/4 and 0.85
    elsewhere, u = 0, tau = 0.58, 500 steps, against the exact isothermal
    Riemann solution with c^2 = J_2/3 = 5/9 (lattice units).  The paper prints
    no tolerance; 0.1 % on the plateau, 2 cells on the shock."""
    L, steps, tau = 3001, 500, 0.58
    C = math.sqrt(5.0 / 9.0)
    xs = np.arange(L)
    n0 = np.where((xs > L / 4) & (xs < 3 * L / 4), 1.0, 0.85)
    f = lbm1d.run(lbm1d.init_equilibrium(n0, np.zeros(L), "t0"), tau, "t0", steps)
    fl = lbm1d.fields(f, "t0")
    x0 = 0.75 * L
    rs, us = riemann.star_state(1.0, 0.0, 0.85, 0.0, C)
    S = rs * us / (rs - 0.85)
    plateau = slice(int(x0 + (us - C) * steps) + 20, int(x0 + S * steps) - 20)
    assert abs(fl["n"][plateau].mean() - rs) < 1e-3 * rs
    assert abs(fl["ux"][plateau].mean() - us) < 1e-3
    half = 0.5 * (rs + 0.85)
    k = 2300 + int(np.argmax(fl["n"][2300:2900] < half))
    assert abs(k - (x0 + S * steps)) <= 2.0
