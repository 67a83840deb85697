"""FP32 / BF16 deviation storage with the Fermi-Dirac inversion in FP64
(inv="exact_f64") against the FP64 oracle, and beside the same storage with
the FP32 inversion.

The step keeps FP32 populations, moment sums and equilibrium; only the
inversion J_2 -> (x, J_4) of Sect. "Generalized polynomials in D dimensions"
runs in FP64 (J_4 to about 1e-13, rounded once to FP32).  The per-step error
budget is therefore the FP32 step's (storage rounding plus FP32 arithmetic,
8 u_s max|g| + 4e-6 max|f|), and the two inversions give populations within
the FP32 inversion's own share of it.

The 1024^2 four-quadrant lattice (tau = 0.6) is the FP32-storage / FP64-
inversion workload against plain FP64; its FD closure turns non-finite near
step 12 there, so the comparison stops at 10 steps.
"""
import numpy as np
import pytest

from oracle import lbm as olbm
from paper_1510_07328_gb300 import inputs
from parity import finite_pair

pytestmark = pytest.mark.gpu

U_STORE = {"f32": 2.0 ** -24, "bf16": 2.0 ** -8}
N_REF, T_REF = 0.95, 0.05


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available()
    from paper_1510_07328_gb300 import build

    build.build()
    from paper_1510_07328_gb300 import lbm

    return lbm


def wref(n_ref, t_ref):
    """W_a^ref of the deviation storage, from the oracle's weights."""
    from oracle import fd, gpoly

    j2 = float(fd.j2_of_x(fd.x_of_t(np.array([t_ref])))[0])
    return gpoly.weights(2, n_ref, j2)[:, None, None]


CASES = {
    "random_300x5_bb": lambda: inputs.random_field(300, 5, 61, tau=0.7, bc_x="bounceback"),
    "random_129x9": lambda: inputs.random_field(129, 9, 62, tau=0.58, t_lo=0.005, t_hi=0.3),
    "random_130x6_hot": lambda: inputs.random_field(130, 6, 63, tau=0.65, u_max=0.05, t_lo=0.3, t_hi=9.5),
    # cold cells near the clamp end t = 1e-3 (the degenerate closed form of both inversions)
    "random_97x7_cold": lambda: inputs.random_field(97, 7, 64, tau=0.9, u_max=0.02, t_lo=0.0012, t_hi=0.01),
}


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("name", list(CASES))
def test_step_parity_x64(L, prec, name):
    """Two steps, each from the oracle's state, against the oracle's next
    state; and the FP32-inversion step from the same stored state beside it."""
    p = CASES[name]()
    f = inputs.perturb_populations(olbm.init_equilibrium(p.n, p.ux, p.uy, p.t), 71, 0.01)
    par = olbm.Params(tau=p.tau, bc_x=p.bc_x, bc_y=p.bc_y)
    W = wref(N_REF, T_REF)
    a = L.Lattice([p], stat="fd", prec=prec, n_ref=N_REF, t_ref=T_REF, inv="exact_f64")
    b = L.Lattice([p], stat="fd", prec=prec, n_ref=N_REF, t_ref=T_REF)
    for _ in range(2):
        a.set_populations(f)
        b.set_populations(f)
        a.step(1)
        b.step(1)
        got, got32 = a.populations(0), b.populations(0)
        g_in = np.abs(f - W).max()
        f = olbm.step(f, par)
        g_out = np.abs(f - W).max()
        tol = 8 * U_STORE[prec] * max(g_in, g_out) + 4e-6 * np.abs(f).max()
        finite_pair(got, f)
        err = np.abs(got - f).max()
        d = np.abs(got - got32).max()
        print(f"{name} {prec}: FP64 inversion err {err:.3e}, FP32 inversion err {np.abs(got32 - f).max():.3e}, "
              f"difference {d:.3e}, tol {tol:.3e}")
        assert err <= tol, (err, tol)
        # the inversions differ by the FP32 one's share of the budget (plus
        # one storage rounding where a result lands on a rounding boundary)
        assert d <= 4e-6 * np.abs(f).max() + 2 * U_STORE[prec] * g_out, d
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_init_x64(L, prec):
    """The initial equilibrium with the closure J_2(t), J_4(t) in FP64: storage
    rounding plus the FP32 equilibrium's budget."""
    p = CASES["random_129x9"]()
    lat = L.Lattice([p], stat="fd", prec=prec, n_ref=N_REF, t_ref=T_REF, inv="exact_f64")
    lat.init()
    got = lat.populations(0)
    lat.close()
    ref = olbm.init_equilibrium(p.n, p.ux, p.uy, p.t)
    W = wref(N_REF, T_REF)
    err = np.abs(got - ref).max()
    assert err <= U_STORE[prec] * np.abs(ref - W).max() + 4e-6 * np.abs(ref).max(), err


@pytest.mark.parametrize("prec", ["f32", "bf16"])
def test_moments_x64(L, prec):
    """T, t and mu of the FP64 inversion against the oracle's fields of the
    stored state.  The inversion is exact; what remains is the FP32 rounding
    of delta = 3/2 - J_2 in the deviation moments, amplified by the
    conditioning of x(J_2) as t -> 0 (the FP32 inversion's bound, 2e-5)."""
    p = CASES["random_129x9"]()
    f = inputs.perturb_populations(olbm.init_equilibrium(p.n, p.ux, p.uy, p.t), 72, 0.002)
    a = L.Lattice([p], stat="fd", prec=prec, n_ref=N_REF, t_ref=T_REF, inv="exact_f64")
    b = L.Lattice([p], stat="fd", prec=prec, n_ref=N_REF, t_ref=T_REF)
    a.set_populations(f)
    b.set_populations(f)
    stored = a.populations(0)
    got, got32 = a.fields(0), b.fields(0)
    a.close()
    b.close()
    ref = olbm.fields(stored)
    assert np.abs(got["n"] - ref["n"]).max() <= 1e-12 * ref["n"].max()
    for k in ("T", "t"):
        finite_pair(got[k], ref[k])
        rel = np.abs(got[k] - ref[k]) / np.abs(ref[k])
        rel32 = np.abs(got32[k] - ref[k]) / np.abs(ref[k])
        print(prec, k, "max rel: FP64 inversion", rel.max(), "FP32 inversion", rel32.max())
        assert rel.max() <= 2e-5, k
    assert np.abs(got["mu"] - ref["mu"]).max() <= 2e-5 * np.abs(ref["mu"]).max()


def _errors(a, b):
    ok = np.isfinite(a["n"]) & np.isfinite(b["n"])
    rT = (np.abs(a["T"] - b["T"]) / b["T"])[ok]
    return {"finite": float(ok.mean()),
            "n": float((np.abs(a["n"] - b["n"]) / b["n"])[ok].max()),
            "u": float(np.hypot(a["ux"] - b["ux"], a["uy"] - b["uy"])[ok].max()),
            "T_max": float(rT.max()), "T_rms": float(np.sqrt(np.mean(rT ** 2)))}


def test_quadrants_fp32_storage_fp64_inversion_vs_fp64(L):
    """The 1024^2 quadrant lattice: FP32 deviation storage with the FP64
    inversion and with the FP32 one, each against the plain FP64 GPU path
    after 5 and 10 steps.  Both hold the FP32 storage bounds; the printed
    maxima show what the inversion's precision changes."""
    prob = inputs.quadrants(1024, seed=1)
    ref = L.Lattice([prob], stat="fd", prec="f64")
    x64 = L.Lattice([prob], stat="fd", prec="f32", n_ref=0.9, t_ref=0.07, inv="exact_f64")
    f32 = L.Lattice([prob], stat="fd", prec="f32", n_ref=0.9, t_ref=0.07)
    for lat in (ref, x64, f32):
        lat.init()
    done = 0
    for k in (5, 10):
        for lat in (ref, x64, f32):
            lat.step(k - done)
        done = k
        fr = ref.fields(0)
        e64, e32 = _errors(x64.fields(0), fr), _errors(f32.fields(0), fr)
        print(f"quadrants 1024^2 FP32 storage, step {k}: FP64 inversion {e64}; FP32 inversion {e32}")
        for e in (e64, e32):
            assert e["finite"] == 1.0
            assert e["n"] <= 3e-6 and e["u"] <= 3e-6 and e["T_rms"] <= 3e-6, e
    for lat in (ref, x64, f32):
        lat.close()


def test_x64_rejected_where_not_built(L):
    """The FP64 inversion exists for the FD closure on d2v9 only, and not with
    obstacles or forces."""
    p = inputs.random_field(64, 4, 65)
    for stat in ("t0", "mb", "ft"):
        with pytest.raises(L.LbmError) as e:
            L.Lattice([p], stat=stat, prec="f32", n_ref=N_REF, t_ref=T_REF, inv="exact_f64")
        assert e.value.status == L.LBM_EUNSUPPORTED
    lat = L.Lattice([p], stat="fd", prec="f32", n_ref=N_REF, t_ref=T_REF, inv="exact_f64")
    with pytest.raises(L.LbmError) as e:
        lat.set_force(1e-6, 0.0)
    assert e.value.status == L.LBM_EUNSUPPORTED
    lat.close()
