"""Reduced-precision storage against FP64 on the same GPU, over many steps,
on the 1024^2 four-quadrant Riemann lattice (tau = 0.6).

* FD closure at the workload's own states (t in [0.02, 0.1]): the energy
  closure is linearly unstable there and the lattice turns non-finite near
  step 12 (the oracle shows the same), so the comparison stops at 10 steps.
* Maxwell-Boltzmann closure (stable): 1000 and 5000 steps.

Each case states its errors on n, |u| (and T for FD) as maxima over the
lattice; the bounds below hold them with a margin and are printed.
"""
import numpy as np
import pytest

from paper_1510_07328_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available()
    from paper_1510_07328_gb300 import build

    build.build()
    from paper_1510_07328_gb300 import lbm

    return lbm


def errors(a, b, with_T):
    ok = np.isfinite(a["n"]) & np.isfinite(b["n"])
    out = {"finite": float(ok.mean()),
           "n": float((np.abs(a["n"] - b["n"]) / b["n"])[ok].max()),
           "u": float(np.hypot(a["ux"] - b["ux"], a["uy"] - b["uy"])[ok].max())}
    if with_T:
        out["T_rms"] = float(np.sqrt(np.mean(((a["T"] - b["T"]) / b["T"])[ok] ** 2)))
    return out


def run_pair(L, stat, prec, checkpoints):
    prob = inputs.quadrants(1024, seed=1)
    ref = L.Lattice([prob], stat=stat, prec="f64")
    red = L.Lattice([prob], stat=stat, prec=prec, n_ref=0.9, t_ref=0.07)
    ref.init()
    red.init()
    done, res = 0, {}
    for k in checkpoints:
        ref.step(k - done)
        red.step(k - done)
        done = k
        res[k] = errors(red.fields(0), ref.fields(0), stat == "fd")
    ref.close()
    red.close()
    return res


# (stat, prec) -> {steps: (max rel n, max |u|, RMS rel T)}; measured on GB300:
# FD FP32 step 10: 5.0e-7, 3.8e-7, 3.1e-7; FD BF16 step 10: 2.0e-3, 1.5e-3,
# 1.6e-3; MB FP32 step 5000: 2.2e-5, 7.4e-6; MB BF16 step 5000: 4.8e-3, 2.0e-3
BOUNDS = {
    ("fd", "f32"): {5: (3e-6, 3e-6, 3e-6), 10: (3e-6, 3e-6, 3e-6)},
    ("fd", "bf16"): {5: (1e-2, 1e-2, 5e-2), 10: (1e-2, 1e-2, 5e-2)},
    ("mb", "f32"): {1000: (1e-4, 5e-5, None), 5000: (1e-4, 5e-5, None)},
    ("mb", "bf16"): {1000: (2e-2, 1e-2, None), 5000: (2e-2, 1e-2, None)},
}


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("stat", ["fd", "mb"])
def test_reduced_precision_error_vs_fp64(L, stat, prec):
    b = BOUNDS[(stat, prec)]
    res = run_pair(L, stat, prec, sorted(b))
    for k, e in res.items():
        print(f"quadrants 1024^2 {stat} {prec} step {k}: {e}")
        assert e["finite"] == 1.0
        assert e["n"] <= b[k][0] and e["u"] <= b[k][1], (k, e)
        if b[k][2] is not None:
            assert e["T_rms"] <= b[k][2], (k, e)
