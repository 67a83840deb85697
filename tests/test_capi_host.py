"""The C-ABI library without a GPU: it builds, loads, exports every symbol that
include/lbm.h declares, and rejects invalid arguments on the host before any
CUDA call."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1510_07328_gb300 import build

    build.build()
    from paper_1510_07328_gb300 import lbm

    return lbm


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lbm_create", "lbm_init_riemann", "lbm_step", "lbm_moments", "lbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (lbm_[a-z_]+)$", out, flags=re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib.LIB, n)


@pytest.mark.parametrize("bad,msg", [
    (dict(tau=0.5), "tau"),
    (dict(nx=0), "nx"),
    (dict(ny=-1), "nx"),
])
def test_create_rejects_bad_problem(lib, bad, msg):
    p = dict(nx=8, ny=4, tau=0.8, bc_x="periodic", bc_y="periodic", n_ref=1.0, t_ref=0.05)
    p.update(bad)
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create([p])
    assert e.value.status == lib.LBM_EINVAL
    assert msg in str(e.value)


@pytest.mark.parametrize("shape,msg", [
    ((1 << 21, 1 << 20), "problem too large"),      # 2^41 cells in one problem
    ((65536, 32769), "more than 2^31 cells"),       # 2^31 + 65536 cells: 32-bit plane offsets
])
def test_create_rejects_oversize(lib, shape, msg):
    """Maximum sizes: one problem above 2^40 cells, or a context whose planes
    exceed the 32-bit offsets of the step kernels, is refused before any
    allocation."""
    p = dict(nx=shape[0], ny=shape[1], tau=0.8, bc_x="periodic", bc_y="periodic", n_ref=1.0, t_ref=0.05)
    for prec in ("f32", "f64"):
        with pytest.raises(lib.LbmError) as e:
            lib.lbm_create([p], prec=prec)
        assert e.value.status == lib.LBM_EINVAL
        assert msg in str(e.value)


def test_create_rejects_too_many_cells_over_problems(lib):
    """The 2^31-cell limit counts the padded planes of all problems together."""
    p = dict(nx=32768, ny=32768, tau=0.8, bc_x="periodic", bc_y="periodic", n_ref=1.0, t_ref=0.05)
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create([p, p, dict(p, nx=8, ny=8)], prec="f32")
    assert e.value.status == lib.LBM_EINVAL
    assert "more than 2^31 cells" in str(e.value)


def test_create_rejects_reference_out_of_range(lib):
    p = dict(nx=8, ny=4, tau=0.8, n_ref=1.0, t_ref=20.0)
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create([p], prec="f32")
    assert e.value.status == lib.LBM_EINVAL and "t_ref" in str(e.value)
    p["t_ref"] = 0.05
    p["n_ref"] = -1.0
    with pytest.raises(lib.LbmError):
        lib.lbm_create([p], prec="bf16")


def test_create_rejects_unsupported_and_null(lib):
    import ctypes as C

    arr = (lib.lbm_problem * 1)(lib.lbm_problem(8, 4, 0.8, 0, 0, 1.0, 0.05))
    ctx = C.c_void_p()
    par = lib.lbm_params(3, 3, 0, 0, 0, 1, arr)
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EUNSUPPORTED
    par = lib.lbm_params(2, 4, 0, 0, 0, 1, arr)
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EUNSUPPORTED
    assert "order" in lib.lbm_last_error(None)
    assert lib.LIB.lbm_create(None, None, C.byref(ctx)) == lib.LBM_EINVAL
    par = lib.lbm_params(2, 3, 7, 0, 0, 1, arr)
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EINVAL
    # calls on a NULL context fail cleanly
    assert lib.LIB.lbm_step(None, 1) == lib.LBM_EINVAL
    assert lib.LIB.lbm_destroy(None) == lib.LBM_OK
    assert lib.LIB.lbm_launch_count(None) == 0


def test_create_rejects_d1v3_misuse(lib):
    """d1v3 has no finite-temperature closure and its problems are one row."""
    import ctypes as C

    ctx = C.c_void_p()
    arr = (lib.lbm_problem * 1)(lib.lbm_problem(64, 1, 0.8, 0, 0, 1.0, 0.05))
    par = lib.lbm_params(1, 3, lib.STAT["fd"], 0, 0, 1, arr)
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EUNSUPPORTED
    assert "d1v3" in lib.lbm_last_error(None)
    par = lib.lbm_params(1, 3, lib.STAT["t0"], 1, 1, 1, arr)  # learned inversion
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EUNSUPPORTED
    arr2 = (lib.lbm_problem * 1)(lib.lbm_problem(64, 2, 0.8, 0, 0, 1.0, 0.05))
    par = lib.lbm_params(1, 3, lib.STAT["t0"], 0, 0, 1, arr2)
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EINVAL
    assert "ny = 1" in lib.lbm_last_error(None)
    par = lib.lbm_params(0, 3, lib.STAT["t0"], 0, 0, 1, arr)
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EUNSUPPORTED


def test_create_rejects_fixed_theta_misuse(lib):
    """The fixed-theta closure (LBM_STAT_FT) needs d2v9, the exact inversion,
    and theta = n_ref t_ref/(2 pi) from a positive n_ref and t_ref in
    [1e-3, 10] at every precision; every check happens before any CUDA call."""
    import ctypes as C

    ft = lib.STAT["ft"]
    ctx = C.c_void_p()
    arr = (lib.lbm_problem * 1)(lib.lbm_problem(64, 1, 0.8, 0, 0, 1.0, 0.05))
    par = lib.lbm_params(1, 3, ft, 0, 0, 1, arr)  # d1v3
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EUNSUPPORTED
    arr = (lib.lbm_problem * 1)(lib.lbm_problem(64, 4, 0.8, 0, 0, 1.0, 0.05))
    par = lib.lbm_params(2, 3, ft, 1, 1, 1, arr)  # learned inversion
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EUNSUPPORTED
    for n_ref, t_ref in ((0.0, 0.05), (1.0, 0.0), (1.0, 20.0)):
        arr = (lib.lbm_problem * 1)(lib.lbm_problem(64, 4, 0.8, 0, 0, n_ref, t_ref))
        par = lib.lbm_params(2, 3, ft, 0, 0, 1, arr)  # FP64 storage: still required
        assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EINVAL
    par = lib.lbm_params(2, 3, 4, 0, 0, 1, arr)  # no closure 4
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EINVAL


@pytest.mark.parametrize("kw,msg", [
    (dict(stat="FD"), "closure"),
    (dict(prec="fp32"), "storage"),
    (dict(inv="Exact"), "inversion"),   # must not fall through to the learned inversion
])
def test_binding_rejects_unknown_names(lib, kw, msg):
    p = dict(nx=8, ny=4, tau=0.8, bc_x="periodic", bc_y="periodic", n_ref=1.0, t_ref=0.05)
    with pytest.raises(ValueError, match=msg):
        lib.lbm_create([p], **kw)
    with pytest.raises(ValueError, match="boundary"):
        lib.lbm_create([dict(p, bc_x="wall")])
    with pytest.raises(ValueError, match="engine"):
        lib.lbm_surrogate_engine(None, "tcgen05")


def test_create_rejects_fp64_inversion_misuse(lib):
    """LBM_INV_EXACT_F64 exists for the FD closure on d2v9 only; an unknown
    inversion is invalid.  Every check happens before any CUDA call."""
    import ctypes as C

    ctx = C.c_void_p()
    arr = (lib.lbm_problem * 1)(lib.lbm_problem(64, 4, 0.8, 0, 0, 1.0, 0.05))
    for stat in ("t0", "mb", "ft"):
        par = lib.lbm_params(2, 3, lib.STAT[stat], 1, lib.LBM_INV_EXACT_F64, 1, arr)
        assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EUNSUPPORTED
        assert "FP64 inversion" in lib.lbm_last_error(None)
    arr1 = (lib.lbm_problem * 1)(lib.lbm_problem(64, 1, 0.8, 0, 0, 1.0, 0.05))
    par = lib.lbm_params(1, 3, lib.STAT["t0"], 1, lib.LBM_INV_EXACT_F64, 1, arr1)
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EUNSUPPORTED
    par = lib.lbm_params(2, 3, lib.STAT["fd"], 1, 3, 1, arr)
    assert lib.LIB.lbm_create(C.byref(par), None, C.byref(ctx)) == lib.LBM_EINVAL


def test_lattice_rejects_theta_count_mismatch(lib):
    """A per-problem theta list must hold one value per problem; the check
    runs in the binding, before any context exists."""
    from paper_1510_07328_gb300 import inputs

    probs = [inputs.riemann_1d(), inputs.riemann_1d(nx=64)]
    with pytest.raises(ValueError, match="theta"):
        lib.Lattice(probs, stat="ft", prec="f64", theta=[0.01])
