"""The allocation-free conservation sums (lbm_conservation_sums_static).

Callers that cannot allocate device memory (their memory belongs to another
allocator, or they run where allocation is not allowed) use this call instead
of lbm_moments' diagnostics.  It must give the same totals as the regular
entry point, on two calls in a row that share its static scratch array.  This
file is collected last so that a run stopping at the first failure has run
every other test before it.
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


def _totals(d):
    return np.array([d["sum_n"], d["sum_jx"], d["sum_jy"], d["sum_E"], d["clamped"], d["nonfinite"]], dtype=np.float64)


def test_static_sums_match_lbm_moments_twice(L):
    import torch

    p = inputs.random_field(300, 7, 51, tau=0.7, bc_x="bounceback", u_max=0.05)
    lat = L.Lattice([p], stat="fd", prec="f64")
    lat.init()
    f = torch.empty((9, p.ny, p.nx), dtype=torch.float64, device="cuda")
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        lat.step(3 + call)
        ref = _totals(L.lbm_moments(lat.ctx, 0, diag=True))
        L.lbm_get_populations(lat.ctx, 0, f, on_device=True)
        torch.cuda.synchronize()
        assert L.lbm_conservation_sums_static(f, p.nx, p.ny, out, stat="fd") == L.LBM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:4], ref[:4], rtol=1e-12, atol=1e-12 * abs(ref[0]))
        assert got[4] == ref[4] and got[5] == ref[5]
        out.fill_(float("nan"))
    lat.close()


def test_static_sums_leave_obstacle_cells_out(L):
    """With the obstacle mask of an lbm_set_obstacles context, the totals
    equal lbm_moments' diagnostics (which leave solid cells out), on two calls
    in a row.  Solid cells are never updated, so they keep their initial
    populations in one of the two buffers: there the totals without the mask
    exceed those with it by exactly the solid cells' mass, so the mask is
    what makes them agree."""
    import torch

    p = inputs.random_field(48, 20, 5, tau=0.8, t_lo=0.3, t_hi=0.6, u_max=0.05)
    solid = inputs.disc_mask(48, 20, [(12, 6), (33, 14)], 3)
    lat = L.Lattice([p], stat="mb", prec="f64")
    lat.set_obstacles(solid)
    lat.set_force(2e-5, -1e-5)
    lat.init()
    f = torch.empty((9, p.ny, p.nx), dtype=torch.float64, device="cuda")
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    mask = torch.from_numpy(solid.astype(np.uint8)).cuda()
    for call in range(2):
        lat.step(2 + call)
        ref = _totals(L.lbm_moments(lat.ctx, 0, diag=True))
        L.lbm_get_populations(lat.ctx, 0, f, on_device=True)
        torch.cuda.synchronize()
        assert L.lbm_conservation_sums_static(f, p.nx, p.ny, out, stat="mb", solid=mask) == L.LBM_OK
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:4], ref[:4], rtol=1e-12, atol=1e-12 * abs(ref[0]))
        assert got[4] == ref[4] and got[5] == ref[5]
        out.fill_(float("nan"))
    lat.step(1)  # 6 steps: the buffer that still holds the solid cells' initial populations
    L.lbm_get_populations(lat.ctx, 0, f, on_device=True)
    assert L.lbm_conservation_sums_static(f, p.nx, p.ny, out, stat="mb", solid=mask) == L.LBM_OK
    torch.cuda.synchronize()
    masked = out.cpu().numpy().copy()
    assert L.lbm_conservation_sums_static(f, p.nx, p.ny, out, stat="mb") == L.LBM_OK
    torch.cuda.synchronize()
    unmasked = out.cpu().numpy()
    solid_mass = float(f.cpu().numpy()[:, solid].sum())
    lat.close()
    assert solid_mass > 0.5 * solid.sum() * p.n.min()
    assert abs((unmasked[0] - masked[0]) - solid_mass) <= 1e-12 * unmasked[0]


def test_static_sums_reject_size_above_limit(L):
    import torch

    f = torch.zeros((9, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros((6,), dtype=torch.float64, device="cuda")
    assert L.lbm_conservation_sums_static(f, 4097, 4096, out) == L.LBM_EINVAL
    assert "exceeds the limit" in L.lbm_last_error(None)
    assert L.lbm_conservation_sums_static(f, 0, 4, out) == L.LBM_EINVAL
    assert "nx and ny" in L.lbm_last_error(None)
