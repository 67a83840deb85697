"""FP32 and BF16 deviation storage against the FP64 oracle.

Per step, the oracle state f_k goes into the library as g = f - W_ref rounded
to the storage type, takes one CUDA step and is compared with the oracle's
f_{k+1}.  Error budget per step, in absolute terms:
  storage rounding   u_s max|g|  (unit roundoff u_s = 2^-24 FP32, 2^-8 BF16, in and out)
  FP32 arithmetic    ~ a few 2^-24 max|f| (moment sums, equilibrium, J_4
                     from the FP32 inversion to ~1e-6 relative, entering
                     only the third-order term)
The tolerance is 8 u_s max|g| + 4e-6 max|f|.
"""
import numpy as np
import pytest

from oracle import lbm as olbm
from paper_1510_07328_gb300 import inputs

pytestmark = pytest.mark.gpu

U_STORE = {"f32": 2.0 ** -24, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available()
    from paper_1510_07328_gb300 import build

    build.build()
    from paper_1510_07328_gb300 import lbm

    return lbm


def oinit(p, stat="fd"):
    return olbm.init_equilibrium(p.n, p.ux, p.uy, p.t, stat)


def wref(p, stat, n_ref, t_ref):
    """W_a^ref of the library's deviation storage, from the oracle's weights."""
    from oracle import fd, gpoly

    if stat == "fd":
        j2 = float(fd.j2_of_x(fd.x_of_t(np.array([t_ref])))[0])
    else:
        j2 = 1.5 if stat == "t0" else 1.0
    return gpoly.weights(2, n_ref, j2)


CASES = {
    "random_300x5_bb": lambda: inputs.random_field(300, 5, 61, tau=0.7, bc_x="bounceback"),
    "random_129x9": lambda: inputs.random_field(129, 9, 62, tau=0.58, t_lo=0.005, t_hi=0.3),
    "riemann_400x4": lambda: inputs.riemann_1d(),
    # hot states, x from about 3.3 down to the clamp end x(t = 10): the FP32
    # inversion's low-x branch (J_4 from its polynomial in delta) over its range
    "random_130x6_hot": lambda: inputs.random_field(130, 6, 63, tau=0.65, u_max=0.05, t_lo=0.3, t_hi=9.5),
}


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("stat", ["fd", "t0", "mb"])
@pytest.mark.parametrize("name", list(CASES))
def test_step_parity_reduced(L, prec, stat, name):
    p = CASES[name]()
    n_ref, t_ref = 0.95, 0.05
    f = inputs.perturb_populations(oinit(p, stat), 71, 0.01)
    par = olbm.Params(tau=p.tau, bc_x=p.bc_x, bc_y=p.bc_y, stat=stat)
    W = wref(p, stat, n_ref, t_ref)[:, None, None]
    lat = L.Lattice([p], stat=stat, prec=prec, n_ref=n_ref, t_ref=t_ref)
    for _ in range(2):
        lat.set_populations(f)
        lat.step(1)
        got = lat.populations(0)
        g_in = np.abs(f - W).max()
        f = olbm.step(f, par)
        g_out = np.abs(f - W).max()
        tol = 8 * U_STORE[prec] * max(g_in, g_out) + 4e-6 * np.abs(f).max()
        err = np.abs(got - f).max()
        assert err <= tol, (err, tol)
    lat.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("stat", ["fd", "t0", "mb"])
def test_init_reduced(L, prec, stat):
    """The initial equilibrium of a deviation-stored context is computed with
    the step's FP32 arithmetic (closure from t and equilibrium in deviation
    form): storage rounding plus the step's FP32 budget, 4e-6 max|f|."""
    p = CASES["random_129x9"]()  # t from 0.005: the degenerate closed form and the series
    lat = L.Lattice([p], stat=stat, prec=prec, n_ref=0.95, t_ref=0.05)
    lat.init()
    got = lat.populations(0)
    lat.close()
    ref = oinit(p, stat)
    W = wref(p, stat, 0.95, 0.05)[:, None, None]
    err = np.abs(got - ref).max()
    assert err <= U_STORE[prec] * np.abs(ref - W).max() + 4e-6 * np.abs(ref).max(), err


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_moments_reduced(L, prec):
    """Moments of a deviation-stored context against the oracle's fields of
    the same populations.  n and u come from FP64 sums of the stored values
    (storage rounding only).  T, mu and t come from the FP32 inversion:
    relative error 2e-5 at these states, t in [0.005, 0.3].  J_2 carries the
    storage rounding, and x(J_2) is ill-conditioned as t -> 0."""
    p = CASES["random_129x9"]()
    f = inputs.perturb_populations(oinit(p), 72, 0.002)
    lat = L.Lattice([p], stat="fd", prec=prec, n_ref=0.95, t_ref=0.05)
    lat.set_populations(f)
    stored = lat.populations(0)  # the state the library holds, after storage rounding
    got = lat.fields(0)
    lat.close()
    ref = olbm.fields(stored)
    assert np.abs(got["n"] - ref["n"]).max() <= 1e-12 * ref["n"].max()
    assert np.abs(got["ux"] - ref["ux"]).max() <= 1e-12 and np.abs(got["uy"] - ref["uy"]).max() <= 1e-12
    for k in ("T", "t"):
        rel = np.abs(got[k] - ref[k]) / np.abs(ref[k])
        print(prec, k, "max rel", rel.max())
        assert rel.max() <= 2e-5, k
    assert np.abs(got["mu"] - ref["mu"]).max() <= 2e-5 * np.abs(ref["mu"]).max()


def test_fp32_against_fp64_fields_after_20_steps(L):
    """Stated error of the FP32 path against the FP64 GPU path after 20 steps
    on a smooth, stable-for-20-steps state: density, velocity, temperature."""
    p = inputs.random_field(256, 64, 81, tau=0.8, u_max=0.01, n_lo=0.95, n_hi=1.05, t_lo=0.1, t_hi=0.12)
    a = L.Lattice([p], stat="fd", prec="f64")
    b = L.Lattice([p], stat="fd", prec="f32", n_ref=1.0, t_ref=0.11)
    a.init()
    b.init()
    a.step(20)
    b.step(20)
    fa, fb = a.fields(0), b.fields(0)
    a.close()
    b.close()
    assert np.isfinite(fa["n"]).all() and np.isfinite(fb["n"]).all()
    assert np.abs(fb["n"] - fa["n"]).max() < 2e-6
    assert np.abs(fb["ux"] - fa["ux"]).max() < 2e-6
    assert (np.abs(fb["T"] - fa["T"]) / fa["T"]).max() < 1e-3
