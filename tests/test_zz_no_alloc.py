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


def test_static_sums_reject_size_above_limit(L):
    import torch

    f = torch.zeros((9, 1), dtype=torch.float64, device="cuda")
    out = torch.zeros((6,), dtype=torch.float64, device="cuda")
    assert L.lbm_conservation_sums_static(f, 4097, 4096, out) == L.LBM_EINVAL
    assert L.lbm_conservation_sums_static(f, 0, 4, out) == L.LBM_EINVAL
