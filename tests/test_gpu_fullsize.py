"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times, on sampled cells.

The CUDA path runs the whole lattice; for each sampled cell the oracle runs
only the (2k+1) x (2k+1) window around it, built from the same seeded input
fields, for the same k steps.  Cells within k of a window edge feel the
window's artificial boundary; the centre cell does not, so it must match the
full-lattice result.  A window that reaches a wall keeps that wall
(bounce-back).
"""
import numpy as np
import pytest

from oracle import lbm as olbm
from paper_1510_07328_gb300 import inputs

pytestmark = pytest.mark.gpu
K = 3  # steps


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available()
    from paper_1510_07328_gb300 import build

    build.build()
    from paper_1510_07328_gb300 import lbm

    return lbm


def sample_cells(nx, ny, count, seed):
    r = inputs.uniform(seed, 2 * count)
    xs = np.minimum((r[:count] * nx).astype(int), nx - 1)
    ys = np.minimum((r[count:] * ny).astype(int), ny - 1)
    extra = [(0, 0), (nx - 1, ny - 1), (0, ny - 1), (nx - 1, 0), (nx // 2, ny // 2), (nx // 2 - 1, ny // 2)]
    return list(zip(xs, ys)) + [(x, y) for x, y in extra if x < nx and y < ny]


def window_oracle(field, nx, ny, bc_x, bc_y, tau, cx, cy, k, stat="fd"):
    """Oracle populations of cell (cx, cy) after k steps, from a window.
    field(ys, xs) returns (n, ux, uy, t) arrays for index arrays."""
    wx = np.arange(cx - k, cx + k + 1)
    wy = np.arange(cy - k, cy + k + 1)
    wall_x = bc_x == "bounceback" and (wx.min() < 0 or wx.max() >= nx)
    wall_y = bc_y == "bounceback" and (wy.min() < 0 or wy.max() >= ny)
    if bc_x == "bounceback":
        wx = wx[(wx >= 0) & (wx < nx)]
    if bc_y == "bounceback":
        wy = wy[(wy >= 0) & (wy < ny)]
    gx, gy = np.meshgrid(wx % nx, wy % ny)
    n, ux, uy, t = field(gy, gx)
    f = olbm.init_equilibrium(n, ux, uy, t, stat)
    p = olbm.Params(tau=tau, bc_x="bounceback" if wall_x else "periodic",
                    bc_y="bounceback" if wall_y else "periodic", stat=stat)
    f = olbm.run(f, p, k)
    ix = int(np.where(wx == cx)[0][0])
    iy = int(np.where(wy == cy)[0][0])
    return f[:, iy, ix]


def gpu_cells(lbm, lat, index, prob, cells):
    """Populations of the given cells of one problem, gathered on the device."""
    import torch

    f = torch.empty((9, prob.ny, prob.nx), dtype=torch.float64, device="cuda")
    lbm.lbm_get_populations(lat.ctx, index, f, on_device=True)
    torch.cuda.synchronize()
    xs = torch.tensor([c[0] for c in cells], device="cuda")
    ys = torch.tensor([c[1] for c in cells], device="cuda")
    out = f[:, ys, xs].T.cpu().numpy()
    del f
    return out


def tol_for(prec, fmax, gmax):
    if prec == "f64":
        return 1e-12 * K * fmax
    u = {"f32": 2.0 ** -24, "bf16": 2.0 ** -8}[prec]
    return K * (8 * u * gmax + 4e-6 * fmax)


@pytest.mark.parametrize("prec,inv", [("f32", "exact"), ("f64", "exact"), ("bf16", "exact"),
                                      ("f32", "exact_f64")])
def test_smooth_t_4096_sampled(L, prec, inv):
    """The bench's lattice and contexts: FP32, FP64 and BF16 storage with the
    exact inversion, and FP32 storage with the FP64 inversion."""
    import torch

    prob = inputs.smooth_t(4096, tau=0.8)
    dev = {k: torch.from_numpy(getattr(prob, k)).cuda() for k in ("n", "ux", "uy", "t")}
    lat = L.Lattice([prob], stat="fd", prec=prec, n_ref=0.9, t_ref=0.05, inv=inv)  # as bench.py
    lat.init(fields_on_device=dev)
    lat.step(K)
    cells = sample_cells(prob.nx, prob.ny, 48, seed=101)
    got = gpu_cells(L, lat, 0, prob, cells)
    lat.close()
    del dev

    def field(gy, gx):
        return prob.n[gy, gx], prob.ux[gy, gx], prob.uy[gy, gx], prob.t[gy, gx]

    for (cx, cy), g in zip(cells, got):
        ref = window_oracle(field, prob.nx, prob.ny, prob.bc_x, prob.bc_y, prob.tau, cx, cy, K)
        fmax = np.abs(ref).max()
        assert np.abs(g - ref).max() <= tol_for(prec, fmax, fmax), (cx, cy)


def test_quadrants_1024_sampled(L):
    prob = inputs.quadrants(1024, seed=1)
    lat = L.Lattice([prob], stat="fd", prec="f64")
    lat.init()
    lat.step(K)
    cells = sample_cells(prob.nx, prob.ny, 32, seed=102) + [(511, 511), (512, 512), (511, 0), (1023, 512)]
    got = gpu_cells(L, lat, 0, prob, cells)
    lat.close()

    def field(gy, gx):
        return prob.n[gy, gx], prob.ux[gy, gx], prob.uy[gy, gx], prob.t[gy, gx]

    for (cx, cy), g in zip(cells, got):
        ref = window_oracle(field, prob.nx, prob.ny, prob.bc_x, prob.bc_y, prob.tau, cx, cy, K)
        assert np.abs(g - ref).max() <= tol_for("f64", np.abs(ref).max(), 0), (cx, cy)


def test_batched_256_sampled_autotuned(L):
    probs = inputs.batched()
    lat = L.Lattice(probs, stat="fd", prec="f32", n_ref=1.2, t_ref=0.05)  # as bench.py
    lat.init()
    L.lbm_autotune(lat.ctx, 2)
    lat.step(K)
    pick = sorted(set(int(v) for v in (inputs.uniform(103, 12) * len(probs)).astype(int)))
    for i in pick:
        p = probs[i]
        cells = sample_cells(p.nx, p.ny, 6, seed=200 + i) + [(0, 1), (p.nx - 1, p.ny // 2), (p.nx // 2, 0)]
        got = gpu_cells(L, lat, i, p, cells)

        def field(gy, gx, p=p):
            return p.n[gy, gx], p.ux[gy, gx], p.uy[gy, gx], p.t[gy, gx]

        for (cx, cy), g in zip(cells, got):
            ref = window_oracle(field, p.nx, p.ny, p.bc_x, p.bc_y, p.tau, cx, cy, K)
            fmax = np.abs(ref).max()
            # |g| = |f - W_ref| <= |f| + |W_ref| <= 2 max|f| for these states
            assert np.abs(g - ref).max() <= tol_for("f32", fmax, 2 * fmax), (i, cx, cy)
    lat.close()


def test_smooth_t_4096_sampled_learned(L):
    """The learned step (network on tcgen05, polish, check, fallback) on the
    4096^2 lattice in the launch configuration bench.py times (persistent
    grid, network trained as there), against the exact FP64 oracle."""
    import torch

    n_tr, t_tr = inputs.surrogate_set(1_000_000, seed=4)
    net, _ = L.lbm_surrogate_train(inputs.surrogate_init(11), n_tr, t_tr, epochs=32, batch=1024)
    prob = inputs.smooth_t(4096, tau=0.8)
    dev = {k: torch.from_numpy(getattr(prob, k)).cuda() for k in ("n", "ux", "uy", "t")}
    lat = L.Lattice([prob], stat="fd", prec="f32", n_ref=0.9, t_ref=0.05, inv="surrogate", surrogate=net,
                    engine="tensor")
    lat.init(fields_on_device=dev)
    lat.step(K)
    st = L.lbm_surrogate_stats(lat.ctx)
    cells = sample_cells(prob.nx, prob.ny, 48, seed=104)
    got = gpu_cells(L, lat, 0, prob, cells)
    lat.close()
    del dev
    assert st["evaluations"] > 0.9 * K * prob.nx * prob.ny and st["fallbacks"] <= 0.01 * st["evaluations"], st

    def field(gy, gx):
        return prob.n[gy, gx], prob.ux[gy, gx], prob.uy[gy, gx], prob.t[gy, gx]

    for (cx, cy), g in zip(cells, got):
        ref = window_oracle(field, prob.nx, prob.ny, prob.bc_x, prob.bc_y, prob.tau, cx, cy, K)
        fmax = np.abs(ref).max()
        assert np.abs(g - ref).max() <= tol_for("f32", fmax, fmax), (cx, cy)


def test_porous_4096_sampled_autotuned(L):
    """The porous step on the bench's 4096^2 disc lattice (4793 discs of
    radius 3, MB closure, force (1e-6, 0), FP32 pull codes, autotuned
    tiling), from random velocities so that the bounce-back on the discs
    shows; sampled cells include ones next to the discs.  The oracle window
    carries the same piece of the obstacle mask."""
    import bench
    import torch
    from oracle import porous

    nL, k, force = 4096, K, (1e-6, 0.0)
    centres = inputs.disc_centres(nL, nL, bench.porous_discs(nL), 3, 13)
    solid = inputs.disc_mask(nL, nL, centres, 3)
    r = inputs.uniform(105, 2 * nL * nL)
    ux = (0.05 * (2 * r[:nL * nL] - 1)).reshape(nL, nL)
    uy = (0.05 * (2 * r[nL * nL:] - 1)).reshape(nL, nL)
    prob = inputs.Problem(nL, nL, 0.7, "periodic", "periodic", np.ones((nL, nL)), ux, uy, np.full((nL, nL), 0.5),
                          name="porous_4096", kind="field")
    dev = {key: torch.from_numpy(getattr(prob, key)).cuda() for key in ("n", "ux", "uy", "t")}
    lat = L.Lattice([prob], stat="mb", prec="f32", n_ref=1.0, t_ref=0.5)  # as bench.py
    lat.set_obstacles(solid)
    lat.set_force(*force)
    lat.init(fields_on_device=dev)
    L.lbm_autotune(lat.ctx, 2)
    lat.init(fields_on_device=dev)
    lat.step(k)
    cells = sample_cells(nL, nL, 24, seed=106)
    cells += [((cx + dx) % nL, (cy + dy) % nL) for cx, cy in centres[:12] for dx, dy in ((4, 0), (-3, 2), (0, -4))]
    got = gpu_cells(L, lat, 0, prob, cells)
    lat.close()
    del dev
    for (cx, cy), g in zip(cells, got):
        wx = np.arange(cx - k, cx + k + 1) % nL
        wy = np.arange(cy - k, cy + k + 1) % nL
        gx, gy = np.meshgrid(wx, wy)
        f = olbm.init_equilibrium(prob.n[gy, gx], ux[gy, gx], uy[gy, gx], prob.t[gy, gx], "mb")
        ref = porous.run(f, solid[gy, gx], prob.tau, "mb", force, k)[:, k, k]
        fmax = np.abs(ref).max()
        assert np.abs(g - ref).max() <= tol_for("f32", fmax, fmax), (cx, cy)
    # the near-disc cells do see a solid neighbour
    assert any(solid[(cy + dy) % nL, (cx + dx) % nL] for cx, cy in cells[24:] for dx in (-1, 0, 1) for dy in (-1, 0, 1))
