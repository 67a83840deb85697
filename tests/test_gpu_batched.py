"""Many problems of uneven sizes in one launch: tilings, persistent grids and
the autotuner give the same populations bit for bit, the autotuner leaves the
state untouched, and each problem matches the oracle."""
import numpy as np
import pytest

from oracle import lbm as olbm
from paper_1510_07328_gb300 import inputs
from parity import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available()
    from paper_1510_07328_gb300 import build

    build.build()
    from paper_1510_07328_gb300 import lbm

    return lbm


def small_batch():
    specs = inputs.batched_specs(count=12, seed=9, lmin=3, lmax=300, wmin=1, wmax=9)
    probs = []
    for s in specs:
        probs.append(inputs._half(s.nx, s.ny, s.nx // 2, (s.n_left, 0.0, 0.0, s.t), (s.n_right, 0.0, 0.0, s.t),
                                  s.tau, "bounceback", "periodic", "b"))
    return probs


def run_tiling(L, probs, prec, rows, ctas, steps=21):
    lat = L.Lattice(probs, prec=prec, n_ref=1.2, t_ref=0.05)
    L.lbm_set_tiling(lat.ctx, rows, ctas)
    assert L.lbm_get_tiling(lat.ctx) == {"rows_per_tile": rows, "ctas": ctas}
    lat.init()
    lat.step(steps)
    got = [lat.populations(i) for i in range(len(probs))]
    lat.close()
    return got


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_tilings_agree_and_each_is_deterministic(L, prec):
    """Each tiling is a separately compiled kernel: for a given tiling two runs
    agree bit for bit; across tilings the FP32 results may differ by rounding
    (the compiler may fuse multiply-adds differently per instantiation), which
    the unstable dynamics amplify (some of these small problems leave the
    equilibrium's domain within about 20 steps), so the comparison across
    tilings is made after 6 steps; FP64 differences stay at round-off.  Cells
    of the smallest problems that leave the expansion's domain are NaN in
    every tiling alike; the comparisons require the same NaN cells."""
    probs = small_batch()
    tol = {"f64": 1e-13, "f32": 2e-6}[prec]
    ref = run_tiling(L, probs, prec, 1, 0, steps=6)
    for rows in (1, 2, 4, 8):
        for ctas in (0, 3, 64):
            got = run_tiling(L, probs, prec, rows, ctas, steps=6)
            for a, r in zip(got, ref):
                assert rel_err(a, r) <= tol, (rows, ctas)
            first = run_tiling(L, probs, prec, rows, ctas, steps=21)  # 16-step graph + 5 launches
            again = run_tiling(L, probs, prec, rows, ctas, steps=21)
            for a, b in zip(first, again):
                assert np.array_equal(a, b, equal_nan=True), (rows, ctas)


def test_autotune_keeps_state_and_picks_valid_tiling(L):
    probs = small_batch()
    lat = L.Lattice(probs, prec="f32", n_ref=1.2, t_ref=0.05)
    lat.init()
    lat.step(3)
    before = [lat.populations(i) for i in range(len(probs))]
    t = L.lbm_autotune(lat.ctx, 2)
    assert t["rows_per_tile"] in (1, 2, 4, 8) and t["ctas"] >= 0 and t["ms_per_step"] > 0
    after = [lat.populations(i) for i in range(len(probs))]
    for a, b in zip(before, after):
        assert np.array_equal(a, b, equal_nan=True)
    lat.step(5)
    lat.close()


def test_batch_matches_oracle_per_problem(L):
    probs = small_batch()
    lat = L.Lattice(probs, prec="f64")
    L.lbm_set_tiling(lat.ctx, 8, 5)
    fs = [olbm.init_equilibrium(p.n, p.ux, p.uy, p.t) for p in probs]
    fs = [inputs.perturb_populations(f, 90 + i, 0.02) for i, f in enumerate(fs)]
    for i, f in enumerate(fs):
        lat.set_populations(f, i)
    lat.step(1)
    for i, (p, f) in enumerate(zip(probs, fs)):
        ref = olbm.step(f, olbm.Params(tau=p.tau, bc_x=p.bc_x, bc_y=p.bc_y))
        assert np.abs(lat.populations(i) - ref).max() <= 1e-12 * np.abs(ref).max()
    lat.close()


def test_set_tiling_rejects_bad_values(L):
    lat = L.Lattice(small_batch()[:2], prec="f64")
    for rows, ctas in ((3, 0), (0, 0), (4, -1)):
        with pytest.raises(L.LbmError) as e:
            L.lbm_set_tiling(lat.ctx, rows, ctas)
        assert e.value.status == L.LBM_EINVAL
    lat.close()
