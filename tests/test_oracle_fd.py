"""Pins for oracle/fd.py: the complete Fermi-Dirac integrals and J_2, J_4.

Each check fixes the oracle against something other than itself: mpmath's
polylogarithm (brute force at 40 digits), closed forms of the low orders, the
derivative identity d f_n/dx = f_{n-1}, the Sommerfeld expansion of the paper
(Eq. (sommerfeld)) and the zero-temperature and Maxwell-Boltzmann limits of the
J_L that the paper prints (Sect. "Numerical simulations for electrons in
metals"; Sect. "Generalized polynomials in D dimensions", MB weight).
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import fd

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_limits.json")

XS = [-30.0, -5.0, -2.25, -1.0000001, -1.0, -0.9999999, -0.5, 0.0, 0.3,
      0.9999999, 1.0, 1.0000001, 2.0, 3.3, 10.0, 20.0, 40.0, 100.0, 1000.0]


def test_fd_against_mpmath_polylog():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for x in XS:
        for n in range(1, fd.NMAX + 1):
            ref = float(-mp.polylog(n, -mp.e ** mp.mpf(x)))
            v = float(fd.fd(n, np.array([x]))[0])
            assert abs(v - ref) <= 2e-15 * abs(ref), (n, x, v, ref)


def test_low_orders_closed_form():
    x = np.linspace(-40, 60, 1001)
    np.testing.assert_allclose(fd.fd(0, x), 1.0 / (1.0 + np.exp(-x)), rtol=1e-15)
    f1 = np.where(x > 0, x + np.log1p(np.exp(-np.abs(x))), np.log1p(np.exp(x)))
    np.testing.assert_allclose(fd.fd(1, x), f1, rtol=4e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_derivative_identity(n):
    x = np.array([-3.0, -1.0, -0.4, 0.0, 0.7, 1.0, 2.5, 8.0, 30.0])
    h = 1e-4
    d = (fd.fd(n, x + h) - fd.fd(n, x - h)) / (2 * h)
    np.testing.assert_allclose(d, fd.fd(n - 1, x), rtol=2e-8, atol=1e-12)


def test_seams_continuous():
    for s in (-1.0, 1.0):
        x = np.array([s - 1e-12, s, s + 1e-12])
        for n in range(1, fd.NMAX + 1):
            v = fd.fd(n, x)
            slope = fd.fd(n - 1, x[1:2])[0]
            # across each seam the change must be the derivative times the step
            assert abs((v[1] - v[0]) - 1e-12 * slope) <= 5e-15 * abs(v[1])
            assert abs((v[2] - v[1]) - 1e-12 * slope) <= 5e-15 * abs(v[1])


def test_sommerfeld_expansion():
    """Eq. (sommerfeld), D = 2, theta = 1: I_2N/(2 pi) = f_{N+1}(mu)
    = mu^{N+1}/(N+1)! [1 + (pi^2/6)(N+1)N/mu^2 + O(mu^-4)]."""
    for N in range(0, 4):
        errs = []
        for mu in (20.0, 40.0):
            exact = fd.fd(N + 1, np.array([mu]))[0]
            som = mu ** (N + 1) / math.factorial(N + 1) * (1 + math.pi ** 2 / 6 * (N + 1) * N / mu ** 2)
            errs.append(abs(exact / som - 1.0))
        if N == 3:  # the dropped (theta/mu)^4 term: halving theta/mu divides it by 16
            assert 12.0 < errs[0] / errs[1] < 20.0
        if N <= 2:  # two terms are exact for f_1..f_3 up to exponentially small tails
            assert errs[1] < 1e-14
        assert errs[1] < 50.0 / 40.0 ** 4  # 7 pi^4 24/360 = 45.5 is the N = 3 coefficient


def test_zero_temperature_limits_printed_in_paper():
    """theta -> 0: J_N = 1 + 2/(N + D) and Delta_N^2 = (D + N)/2 (D = 2)."""
    gold = json.load(open(GOLD))["zero_temperature"]
    assert gold["J_N"] == "1 + 2/(N + D)"
    x = np.array([1e5])
    D = 2
    j2 = fd.j2_of_x(x)[0]
    j4 = fd.j4_of_x(x)[0]
    assert abs(j2 - (1 + 2 / (2 + D))) < 1e-9
    assert abs(j4 - (1 + 2 / (4 + D))) < 1e-9
    d22 = 2.0 / ((D + 2) - j2 * D)
    d42 = 2.0 / ((D + 4) - j4 * (D + 2))
    assert abs(d22 - (D + 2) / 2) < 1e-8
    assert abs(d42 - (D + 4) / 2) < 1e-8


def test_maxwell_boltzmann_limit():
    """x -> -inf: f_n -> e^x for every n, so J_2, J_4 -> 1 (the MB weight
    I_2N = I_0 theta^N gives J_L = 1)."""
    x = np.array([-40.0])
    assert abs(fd.j2_of_x(x)[0] - 1.0) < 1e-15
    assert abs(fd.j4_of_x(x)[0] - 1.0) < 1e-15


def test_j2_strictly_increasing_and_t_roundtrip():
    x = np.linspace(-2.25, 200.0, 4001)
    j2 = fd.j2_of_x(x)
    assert np.all(np.diff(j2) > 0)
    t = np.array([0.005, 0.01, 0.05, 0.1, 0.2, 0.3, 1.0, 10.0])
    np.testing.assert_allclose(fd.t_of_x(fd.x_of_t(t)), t, rtol=1e-14)


def test_fd_values_degenerate_quadratic():
    """For large x, f_n reduce to the polynomials of the inversion formula and
    3/2 - J_2 = pi^2 (3 s - pi^2)/(6 s (s + pi^2)), s = x^2."""
    x = np.array([40.0, 100.0, 300.0])
    s = x * x
    delta = math.pi ** 2 * (3 * s - math.pi ** 2) / (6 * s * (s + math.pi ** 2))
    np.testing.assert_allclose(1.5 - fd.j2_of_x(x), delta, rtol=1e-9)


@pytest.mark.parametrize("t", [0.005, 0.05, 0.1, 0.2, 0.3])
def test_inversion_at_reference_states(t):
    """The inversion end to end at the states used across the workloads:
    x(t), J_2(x) and J_4(x) against mpmath's polylogarithm (solved
    independently), and the oracle's J_2 -> x bisection recovering x."""
    mp = pytest.importorskip("mpmath")
    from oracle import lbm as olbm

    mp.mp.dps = 40

    def f(n, x):
        return -mp.polylog(n, -mp.e ** x)

    x_ref = mp.findroot(lambda x: 1 / f(1, x) - t, 1 / mp.mpf(t))
    j2_ref = f(2, x_ref) ** 2 / (f(1, x_ref) * f(3, x_ref))
    j4_ref = f(3, x_ref) ** 2 / (f(2, x_ref) * f(4, x_ref))
    x = float(fd.x_of_t(np.array([t]))[0])
    assert abs(x - float(x_ref)) <= 1e-13 * abs(float(x_ref))
    assert abs(float(fd.j2_of_x(np.array([x]))[0]) - float(j2_ref)) <= 1e-14
    assert abs(float(fd.j4_of_x(np.array([x]))[0]) - float(j4_ref)) <= 1e-14
    x_back = float(olbm.invert_j2(np.array([float(j2_ref)]))[0])
    # J_2 is flat in x as t -> 0 (3/2 - J_2 ~ x^-2): the round trip's x error
    # is the FP64 rounding of J_2 divided by dJ_2/dx
    dj2 = 2 * (1.5 - float(j2_ref)) / float(x_ref)
    assert abs(x_back - float(x_ref)) <= 4 * 2.2e-16 * 1.5 / dj2 + 1e-12 * abs(float(x_ref))
