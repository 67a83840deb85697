"""FP32 field exchange (lbm_init_fields_f32, lbm_moments_f32) against the
double calls on the same values: the initial populations are bitwise those
of FIELD given the float values as doubles, and every float moment is the
double moment rounded once.  Host arrays are exercised page-locked (read and
written in place by the kernels) and pageable (staged), and as device
tensors."""
import numpy as np
import pytest

from paper_1510_07328_gb300 import inputs

pytestmark = pytest.mark.gpu

NAMES = ("n", "ux", "uy", "T", "mu", "t")


@pytest.fixture(scope="module")
def L():
    import torch

    assert torch.cuda.is_available()
    from paper_1510_07328_gb300 import build

    build.build()
    from paper_1510_07328_gb300 import lbm

    return lbm


def fields32(p):
    return {k: getattr(p, k).astype(np.float32) for k in ("n", "ux", "uy", "t")}


def host32(a, where):
    import torch

    if where == "pageable":
        return np.ascontiguousarray(a, dtype=np.float32)
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    return t.pin_memory() if where == "pinned" else t.cuda()


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("where", ["pageable", "pinned", "device"])
def test_init_f32_equals_double_field(L, prec, where):
    import torch

    p = inputs.random_field(300, 7, 91, tau=0.7, bc_x="bounceback", t_lo=0.02, t_hi=0.3)
    f32 = fields32(p)
    a = L.Lattice([p], prec=prec, n_ref=0.95, t_ref=0.1)
    b = L.Lattice([p], prec=prec, n_ref=0.95, t_ref=0.1)
    L.lbm_init_riemann(a.ctx, 0, "field", fields={k: v.astype(np.float64) for k, v in f32.items()})
    args = [host32(f32[k], where) for k in ("n", "ux", "uy", "t")]
    L.lbm_init_fields_f32(b.ctx, 0, *args, on_device=where == "device")
    torch.cuda.synchronize()
    fa, fb = a.populations(0), b.populations(0)
    a.close()
    b.close()
    assert np.array_equal(fa, fb)


@pytest.mark.parametrize("prec", ["f32", "bf16"])
@pytest.mark.parametrize("where", ["pageable", "pinned", "device"])
def test_moments_f32_is_the_double_rounded_once(L, prec, where):
    import torch

    p = inputs.random_field(257, 9, 92, tau=0.8, t_lo=0.02, t_hi=0.3)
    lat = L.Lattice([p], prec=prec, n_ref=0.95, t_ref=0.1)
    lat.init()
    lat.step(3)
    ref = {k: np.empty((p.ny, p.nx)) for k in NAMES}
    dref = L.lbm_moments(lat.ctx, 0, diag=True, **ref)
    out = {k: host32(np.zeros((p.ny, p.nx), np.float32), where) for k in NAMES}
    d32 = L.lbm_moments_f32(lat.ctx, 0, on_device=where == "device", diag=True, **out)
    torch.cuda.synchronize()
    lat.close()
    for k in NAMES:
        got = out[k].cpu().numpy() if hasattr(out[k], "cpu") else out[k]
        assert np.array_equal(got, ref[k].astype(np.float32)), k
    assert d32 == dref


def test_f32_exchange_rejects_fp64_storage_and_d1v3(L):
    p = inputs.random_field(64, 4, 93)
    f32 = fields32(p)
    lat = L.Lattice([p], prec="f64")
    for call in (lambda: L.lbm_init_fields_f32(lat.ctx, 0, f32["n"], f32["ux"], f32["uy"], f32["t"]),
                 lambda: L.lbm_moments_f32(lat.ctx, 0, n=np.zeros((p.ny, p.nx), np.float32))):
        with pytest.raises(L.LbmError) as e:
            call()
        assert e.value.status == L.LBM_EUNSUPPORTED
    lat.close()
    q = inputs.random_field(256, 1, 94, t_lo=0.05, t_hi=0.05)  # a d1v3 lattice (ny = 1)
    lat = L.Lattice([q], stat="t0", prec="f32", n_ref=0.95, t_ref=0.05, dim=1)
    with pytest.raises(L.LbmError) as e:
        L.lbm_moments_f32(lat.ctx, 0, n=np.zeros((q.ny, q.nx), np.float32))
    assert e.value.status == L.LBM_EUNSUPPORTED
    lat.close()
    lat = L.Lattice([p], prec="f32", n_ref=0.95, t_ref=0.1)
    with pytest.raises(L.LbmError) as e:
        L.lbm_init_fields_f32(lat.ctx, 0, None, f32["ux"], f32["uy"], f32["t"])
    assert e.value.status == L.LBM_EINVAL
    lat.close()
