"""Linear stability of the LBGK step around a uniform state at rest.

The growth factor of a Fourier mode k is the spectral radius of
S(k) J, with J the Jacobian of the oracle's collision (central differences)
and S(k) = diag(exp(-i k . e_a)) the pull-streaming shift.  These tests record
what the paper's scheme does:

* theta = 0 closure (the paper's own runs, Sect. "Numerical simulations for
  electrons in metals"): every 1D mode (k_y = 0, the 3001 x 1 lattice of the
  paper's Riemann test) is stable for tau = 0.57 .. 0.95, consistent with the
  tau-independence the paper reports; 2D modes on d2v9 grow at tau = 0.6.
* energy closure (J_2 read from the energy moment, the finite-temperature
  reading): 1D modes grow at t = T/T_F = 0.05, tau = 0.8.
"""
import math

import numpy as np
import pytest

from oracle import gpoly as g, lbm

E = g.E_D2V9


def jacobian(stat, t, tau, h=1e-6):
    z = np.zeros((1, 1))
    f0 = lbm.init_equilibrium(np.ones((1, 1)), z, z, np.full((1, 1), t), stat)[:, 0, 0]
    Jc = np.zeros((9, 9))
    for b in range(9):
        d = np.zeros(9)
        d[b] = h
        hi, _ = lbm.collide((f0 + d)[:, None], tau, stat)
        lo, _ = lbm.collide((f0 - d)[:, None], tau, stat)
        Jc[:, b] = (hi[:, 0] - lo[:, 0]) / (2 * h)
    return Jc


def growth(stat, t, tau, ks):
    Jc = jacobian(stat, t, tau)
    worst = 0.0
    for kx, ky in ks:
        S = np.diag(np.exp(-1j * (kx * E[:, 0] + ky * E[:, 1])))
        worst = max(worst, np.abs(np.linalg.eigvals(S @ Jc)).max())
    return worst


K1D = [(k, 0.0) for k in np.linspace(1e-3, math.pi, 120)]
K2D = K1D + [(k, k) for k in np.linspace(1e-2, math.pi, 40)] + [(k, k / 2) for k in np.linspace(1e-2, math.pi, 40)]


@pytest.mark.parametrize("tau", [0.57, 0.58, 0.8, 0.95])
def test_zero_temperature_1d_stable(tau):
    assert growth("t0", 0.0, tau, K1D) < 1.0 + 1e-7


def test_zero_temperature_2d_unstable_at_low_tau():
    assert growth("t0", 0.0, 0.6, K2D) > 1.05


def test_energy_closure_1d_unstable():
    assert growth("fd", 0.05, 0.8, K1D) > 1.05


def test_mb_closure_stable():
    assert growth("mb", 0.0, 0.6, K2D) < 1.0 + 1e-7
