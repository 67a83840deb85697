"""The paper's zero-temperature Riemann experiment on the GPU (3001 x 1
periodic, tau = 0.58): FP64 against the oracle cell by cell after 100 steps,
and FP32 and FP64 against the exact isothermal solution after 500 steps.

The remnant of the initial discontinuity, carried with the flow, amplifies
round-off by about 1.06 per step in this setup (a 1e-14 perturbation reaches
2e-2 there by step 500, while the plateau and the shock are unaffected), so
independent runs are compared cell by cell only at step 100, where that
growth is still below 1e-13."""
import math

import numpy as np
import pytest

from oracle import lbm as olbm
from oracle import riemann
from paper_1510_07328_gb300 import inputs

pytestmark = pytest.mark.gpu
C = math.sqrt(0.5)
L, STEPS, TAU = 3001, 500, 0.58


@pytest.fixture(scope="module")
def Lb():
    import torch

    assert torch.cuda.is_available()
    from paper_1510_07328_gb300 import build

    build.build()
    from paper_1510_07328_gb300 import lbm

    return lbm


def problem():
    xs = np.arange(L)
    n = np.where((xs > L / 4) & (xs < 3 * L / 4), 1.0, 0.85)[None, :]
    z = np.zeros((1, L))
    return inputs.Problem(L, 1, TAU, "periodic", "periodic", n, z, z.copy(), z.copy(), name="paper_fig1",
                          kind="field")


@pytest.fixture(scope="module")
def oracle_100():
    p = problem()
    f = olbm.init_equilibrium(p.n, p.ux, p.uy, p.t, "t0")
    return olbm.run(f, olbm.Params(tau=TAU, stat="t0"), 100)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_paper_riemann_run(Lb, oracle_100, prec):
    p = problem()
    lat = Lb.Lattice([p], stat="t0", prec=prec, n_ref=0.9, t_ref=0.05)
    lat.init()
    lat.step(100)
    if prec == "f64":
        f = lat.populations(0)
        assert np.abs(f - oracle_100).max() <= 1e-12 * np.abs(oracle_100).max()
    lat.step(STEPS - 100)
    fl = lat.fields(0)
    lat.close()
    rs, us = riemann.star_state(1.0, 0.0, 0.85, 0.0, C)
    S = rs * us / (rs - 0.85)
    x0 = 0.75 * L
    plateau = slice(int(x0 + (us - C) * STEPS) + 20, int(x0 + S * STEPS) - 20)
    assert abs(fl["n"][0, plateau].mean() - rs) < 1e-3 * rs
    assert abs(fl["ux"][0, plateau].mean() - us) < 1e-3
    k = 2300 + int(np.argmax(fl["n"][0, 2300:2800] < 0.5 * (rs + 0.85)))
    assert abs(k - (x0 + S * STEPS)) <= 2.0
