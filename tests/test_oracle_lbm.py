"""Pins for oracle/lbm.py: the LBGK step.

Invariants that any correct pull-stream + BGK step must satisfy: per-collision
conservation of n, j and E (the K = 3 equilibrium reproduces the moments to
second order exactly); a uniform state is a fixed point; the centre of mass
moves by the total momentum each step (fixes the streaming direction); walls
conserve mass and energy and mirror symmetry holds; a shear wave decays at the
Navier-Stokes rate set by the lattice's own third moment (see
test_shear_wave_decay); and the inversion round-trips.
"""
import math

import numpy as np
import pytest

from oracle import fd, gpoly as g, lbm


def random_near_eq(ny, nx, seed, t=0.1, amp=0.05, stat="fd"):
    rng = np.random.default_rng(seed)
    n = 1.0 + 0.1 * rng.standard_normal((ny, nx))
    ux = 0.05 * rng.standard_normal((ny, nx))
    uy = 0.05 * rng.standard_normal((ny, nx))
    tt = np.full((ny, nx), t)
    f = lbm.init_equilibrium(n, ux, uy, tt, stat)
    return f * (1.0 + amp * rng.standard_normal(f.shape))


@pytest.mark.parametrize("stat", ["fd", "t0", "mb"])
def test_collision_conserves_mass_momentum(stat):
    f = random_near_eq(3, 5, 1, stat=stat)
    out, _ = lbm.collide(f, 0.63, stat)
    n0, j0, E0 = lbm.moments(f)
    n1, j1, E1 = lbm.moments(out)
    np.testing.assert_allclose(n1, n0, rtol=2e-15)
    np.testing.assert_allclose(j1, j0, rtol=1e-13, atol=1e-15)
    if stat == "fd":  # the energy closure: E is a collision invariant
        np.testing.assert_allclose(E1, E0, rtol=2e-15)
    else:             # fixed J_2: E relaxes towards n (u0^2 + 2 J_2/3)
        assert np.abs(E1 - E0).max() > 1e-6


def test_uniform_state_is_fixed_point():
    ny, nx = 4, 6
    for t, ux, uy in [(0.05, 0.0, 0.0), (0.2, 0.07, -0.03)]:
        f = lbm.init_equilibrium(np.full((ny, nx), 1.3), np.full((ny, nx), ux),
                                 np.full((ny, nx), uy), np.full((ny, nx), t))
        f1 = lbm.run(f, lbm.Params(tau=0.7), 3)
        np.testing.assert_allclose(f1, f, rtol=1e-13)


def test_centre_of_mass_moves_by_total_momentum():
    """With pull streaming f_a(x) <- f*_a(x - e_a): sum_x x n(t+1) = sum_x x n(t) + sum j."""
    nx, ny = 64, 3
    xs = np.arange(nx)
    n = np.ones((ny, nx)) + 0.3 * np.exp(-((xs - 32) / 4.0) ** 2)[None, :]
    ux = 0.1 * np.exp(-((xs - 32) / 4.0) ** 2)[None, :] * np.ones((ny, 1))
    f = lbm.init_equilibrium(n, ux, np.zeros((ny, nx)), np.full((ny, nx), 0.2), "mb")
    p = lbm.Params(tau=0.9, stat="mb")
    for _ in range(3):
        nb, jb, _ = lbm.moments(f)
        f = lbm.step(f, p)
        na, _, _ = lbm.moments(f)
        dx = (xs[None, :] * (na - nb)).sum()
        assert abs(dx - jb[0].sum()) < 1e-12


def test_bounceback_walls_conserve_mass_and_energy():
    f = random_near_eq(4, 12, 2, t=0.2)
    n0, j0, E0 = lbm.moments(f)
    out = lbm.run(f, lbm.Params(tau=0.9, bc_x="bounceback"), 4)
    n1, j1, E1 = lbm.moments(out)
    assert abs(n1.sum() - n0.sum()) < 1e-12 * n0.sum()
    assert abs(E1.sum() - E0.sum()) < 1e-12 * E0.sum()
    closed = lbm.run(f, lbm.Params(tau=0.9, bc_x="bounceback", bc_y="bounceback"), 4)
    assert abs(lbm.moments(closed)[0].sum() - n0.sum()) < 1e-12 * n0.sum()


def test_mirror_symmetry_with_walls():
    """Reflecting x (e_a -> mirrored velocity, u_x -> -u_x) commutes with the step."""
    f = random_near_eq(3, 9, 4, t=0.15)
    mirror = np.array([0, 3, 2, 1, 4, 6, 5, 8, 7])  # a -> index of (-e_x, e_y)
    fm = f[mirror][:, :, ::-1]
    p = lbm.Params(tau=0.8, bc_x="bounceback")
    a = lbm.run(f, p, 2)
    b = lbm.run(fm, p, 2)
    np.testing.assert_allclose(b, a[mirror][:, :, ::-1], rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("stat,tau", [("mb", 0.8), ("t0", 0.8), ("t0", 0.58)])
def test_shear_wave_decay(stat, tau):
    """u_y = A sin(2 pi x/L) decays as exp(-nu k^2 t) with the Chapman-Enskog
    viscosity of BGK, nu = (Q_xxy/(n u_y)) (tau - 1/2), Q_xxy = sum f_eq e_x^2 e_y.

    For the printed d2v9 equilibrium at linear order in u this third moment is
    (1 - (1 - J_2) J_4 Delta_4^2)/3 (only the diagonals carry e_x^2 e_y, and the
    J_4 bracket of the third-order term contributes through them).  In the MB
    limit this is 1/3, the paper's eta = I_2 (tau - 1/2) (Sect. "Numerical
    simulations for electrons in metals") in lattice units.  In the theta = 0
    closure it is 1, twice the paper's J_2/3 = 1/2: the quadrature is exact
    only to degree 5 and this moment is of degree 6.  The test pins the lattice
    value and records the factor against the paper's formula.
    """
    L, steps, A = 48, 150, 1e-4
    xs = np.arange(L)
    uy = A * np.sin(2 * math.pi * xs / L)[None, :]
    z = np.zeros((1, L))
    f = lbm.init_equilibrium(np.ones((1, L)), z, uy, z, stat)
    p = lbm.Params(tau=tau, stat=stat)
    s = np.sin(2 * math.pi * xs / L)
    amps = []
    for k in range(steps + 1):
        if k in (50, steps):
            fl = lbm.fields(f, stat)
            amps.append((fl["uy"][0] * s).sum() * 2 / L)
        f = lbm.step(f, p)
    J2, J4 = (1.0, 1.0) if stat == "mb" else (1.5, 4.0 / 3.0)
    D42 = 2.0 / (6.0 - 4.0 * J4)
    nu = (1.0 - (1.0 - J2) * J4 * D42) / 3.0 * (tau - 0.5)
    k2 = (2 * math.pi / L) ** 2
    rate = -math.log(amps[1] / amps[0]) / (steps - 50)
    assert abs(rate / (nu * k2) - 1.0) < 0.01, (rate, nu * k2)
    paper_nu = J2 / 3.0 * (tau - 0.5)
    assert abs(nu / paper_nu - (1.0 if stat == "mb" else 2.0)) < 1e-12


def test_inversion_round_trip():
    x = np.array([-2.0, -0.3, 0.4, 1.7, 3.3, 5.0, 10.0, 20.0, 40.0])
    x2 = lbm.invert_j2(fd.j2_of_x(x))
    np.testing.assert_allclose(x2, x, rtol=1e-12, atol=1e-13)
    # degenerate end: conditioning dx = dJ_2 x^3/pi^2; J_4 stays well determined
    xd = np.array([100.0, 300.0])
    xr = lbm.invert_j2(fd.j2_of_x(xd))
    np.testing.assert_allclose(fd.j4_of_x(xr), fd.j4_of_x(xd), rtol=1e-14)
    np.testing.assert_allclose(xr, xd, rtol=1e-9)


def test_inversion_clamps():
    xs = lbm.invert_j2(np.array([1.6, 1.5, 1.0, 0.5]))
    assert xs[0] == lbm.X_HI and xs[1] == lbm.X_HI
    assert xs[2] == lbm.X_LO and xs[3] == lbm.X_LO


def test_init_is_equilibrium_at_given_t():
    ny, nx = 2, 3
    t = np.array([[0.01, 0.05, 0.1], [0.2, 0.3, 1.0]])
    f = lbm.init_equilibrium(np.full((ny, nx), 0.9), np.zeros((ny, nx)), np.zeros((ny, nx)), t)
    fl = lbm.fields(f)
    np.testing.assert_allclose(fl["t"], t, rtol=1e-9)
    np.testing.assert_allclose(fl["j2"], fd.j2_of_x(fd.x_of_t(t)), rtol=1e-15)
    # T_F = n/(2 pi) for D = 2: T = t n/(2 pi)
    np.testing.assert_allclose(fl["T"], t * 0.9 / (2 * math.pi), rtol=1e-9)
