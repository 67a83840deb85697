"""Thin ctypes binding of the C ABI in include/lbm.h.

Every function here only marshals arguments and calls the library of the same
name; all arithmetic of the method runs in the CUDA kernels of
``liblbm_gb300.so``.  Importing this module loads the library and fails loudly
if it has not been built (``python -m paper_1510_07328_gb300.build``); there is
no CPU fallback.

Device buffers and streams come from PyTorch (``torch.cuda`` tensors and
``torch.cuda.current_stream().cuda_stream``); host buffers are NumPy arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ETIMEOUT, LBM_EUNSUPPORTED = range(6)
LBM_STAT_FD, LBM_STAT_FD_T0, LBM_STAT_MB, LBM_STAT_FT = range(4)
LBM_F64, LBM_F32_DEV, LBM_BF16_DEV = range(3)
LBM_INV_EXACT, LBM_INV_SURROGATE, LBM_INV_EXACT_F64 = range(3)
LBM_BC_PERIODIC, LBM_BC_BOUNCEBACK = range(2)
LBM_INIT_HALF, LBM_INIT_QUADRANT, LBM_INIT_FIELD = range(3)

STAT = {"fd": LBM_STAT_FD, "t0": LBM_STAT_FD_T0, "mb": LBM_STAT_MB, "ft": LBM_STAT_FT}
PREC = {"f64": LBM_F64, "f32": LBM_F32_DEV, "bf16": LBM_BF16_DEV}
BC = {"periodic": LBM_BC_PERIODIC, "bounceback": LBM_BC_BOUNCEBACK}


class lbm_problem(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("tau", C.c_double), ("bc_x", C.c_int32),
                ("bc_y", C.c_int32), ("n_ref", C.c_double), ("t_ref", C.c_double)]


class lbm_params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("order", C.c_int32), ("stat", C.c_int32), ("prec", C.c_int32),
                ("inv", C.c_int32), ("nproblems", C.c_int32), ("problems", C.POINTER(lbm_problem))]


class lbm_state(C.Structure):
    _fields_ = [("n", C.c_double), ("ux", C.c_double), ("uy", C.c_double), ("t", C.c_double)]


class lbm_riemann_desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("x0", C.c_int32), ("y0", C.c_int32), ("s", lbm_state * 4),
                ("n", C.c_void_p), ("ux", C.c_void_p), ("uy", C.c_void_p), ("t", C.c_void_p),
                ("field_on_device", C.c_int32)]


class lbm_tiling(C.Structure):
    _fields_ = [("rows_per_tile", C.c_int32), ("ctas", C.c_int32), ("ms_per_step", C.c_double)]


class lbm_train_cfg(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("lr_final", C.c_float)]


class lbm_train_report(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("loss_first", C.c_double), ("loss_last", C.c_double),
                ("val_rmse_lnT", C.c_double), ("val_rmse_mu", C.c_double), ("val_max_rel_x", C.c_double),
                ("seconds", C.c_double)]


class lbm_diag(C.Structure):
    _fields_ = [("sum_n", C.c_double), ("sum_jx", C.c_double), ("sum_jy", C.c_double), ("sum_E", C.c_double),
                ("clamped", C.c_int64), ("nonfinite", C.c_int64)]


def _load():
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1510_07328_gb300.build` "
                          "(the library has no CPU fallback)")
    lib = C.CDLL(path)
    V = C.c_void_p
    sig = {
        "lbm_create": (C.c_int, [C.POINTER(lbm_params), V, C.POINTER(V)]),
        "lbm_init_riemann": (C.c_int, [V, C.c_int32, C.POINTER(lbm_riemann_desc)]),
        "lbm_step": (C.c_int, [V, C.c_int32]),
        "lbm_moments": (C.c_int, [V, C.c_int32, V, V, V, V, V, V, C.c_int32, C.POINTER(lbm_diag)]),
        "lbm_init_fields_f32": (C.c_int, [V, C.c_int32, V, V, V, V, C.c_int32]),
        "lbm_moments_f32": (C.c_int, [V, C.c_int32, V, V, V, V, V, V, C.c_int32, C.POINTER(lbm_diag)]),
        "lbm_get_populations": (C.c_int, [V, C.c_int32, V, C.c_int32]),
        "lbm_set_populations": (C.c_int, [V, C.c_int32, V, C.c_int32]),
        "lbm_destroy": (C.c_int, [V]),
        "lbm_last_error": (C.c_char_p, [V]),
        "lbm_launch_count": (C.c_int64, [V]),
        "lbm_conservation_sums_static": (C.c_int, [V, C.c_int32, C.c_int32, V, C.c_int32, V, V]),
        "lbm_set_tiling": (C.c_int, [V, C.c_int32, C.c_int32]),
        "lbm_get_tiling": (C.c_int, [V, C.POINTER(lbm_tiling)]),
        "lbm_autotune": (C.c_int, [V, C.c_int32, C.POINTER(lbm_tiling)]),
        "lbm_surrogate_targets": (C.c_int, [V, V, C.c_int64, C.c_int32, V, V, V]),
        "lbm_surrogate_loss_grad": (C.c_int, [V, V, V, C.c_int64, V, C.POINTER(C.c_double), V]),
        "lbm_surrogate_train": (C.c_int, [V, V, C.c_int64, V, V, C.c_int64, C.c_int32, C.POINTER(lbm_train_cfg),
                                          V, C.POINTER(lbm_train_report), V]),
        "lbm_surrogate_eval": (C.c_int, [V, V, V, C.c_int64, V, V, C.c_int32, V]),
        "lbm_surrogate_load": (C.c_int, [V, V]),
        "lbm_surrogate_stats": (C.c_int, [V, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "lbm_surrogate_engine": (C.c_int, [V, C.c_int32]),
        "lbm_surrogate_wait_limit": (C.c_int, [V, C.c_int32]),
        "lbm_set_obstacles": (C.c_int, [V, C.c_int32, V, C.c_int32]),
        "lbm_set_force": (C.c_int, [V, C.c_int32, C.c_double, C.c_double]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


LIB = _load()
EXPORTS = ("lbm_create", "lbm_init_riemann", "lbm_step", "lbm_moments", "lbm_get_populations",
           "lbm_set_populations", "lbm_destroy", "lbm_last_error", "lbm_launch_count",
           "lbm_conservation_sums_static", "lbm_set_tiling", "lbm_get_tiling", "lbm_autotune",
           "lbm_surrogate_targets", "lbm_surrogate_loss_grad", "lbm_surrogate_train", "lbm_surrogate_eval",
           "lbm_surrogate_load", "lbm_surrogate_stats", "lbm_surrogate_engine", "lbm_surrogate_wait_limit",
           "lbm_set_obstacles", "lbm_set_force", "lbm_init_fields_f32", "lbm_moments_f32")
LBM_SURROGATE_FP32_PIPE, LBM_SURROGATE_TENSOR_CORES, LBM_SURROGATE_WARP_MMA = 0, 1, 2
NPARAM = 4482


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def _check(status: int, ctx) -> None:
    if status != LBM_OK:
        raise LbmError(status, LIB.lbm_last_error(ctx).decode())


def _ptr(a, dtype: str = "float64") -> int | None:
    """Address of a NumPy array or torch tensor of the given element type
    (None stays NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"] or a.dtype != np.dtype(dtype):
            raise ValueError(f"host arrays must be C-contiguous {dtype}")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous() or str(a.dtype) != f"torch.{dtype}":
            raise ValueError(f"tensors must be contiguous {dtype}")
        return a.data_ptr()
    raise TypeError("expected a numpy array or a torch tensor")


# ---------------------------------------------------------------- C-ABI calls, same names


def _choice(kind: str, value, table: dict):
    if value not in table:
        raise ValueError(f"unknown {kind} {value!r}; expected one of {sorted(table)}")
    return table[value]


def lbm_create(problems, stat="fd", prec="f64", inv="exact", stream=None, dim=2):
    """problems: list of dicts with nx, ny, tau, bc_x, bc_y, n_ref, t_ref;
    dim 2: d2v9, dim 1: d1v3 (ny = 1)."""
    stat_c = _choice("closure", stat, STAT)
    prec_c = _choice("storage", prec, PREC)
    inv_c = _choice("inversion", inv, {"exact": LBM_INV_EXACT, "surrogate": LBM_INV_SURROGATE,
                                         "exact_f64": LBM_INV_EXACT_F64})
    for p in problems:
        for k in ("bc_x", "bc_y"):
            _choice("boundary", p.get(k, "periodic"), BC)
    arr = (lbm_problem * len(problems))()
    for i, p in enumerate(problems):
        arr[i] = lbm_problem(int(p["nx"]), int(p["ny"]), float(p["tau"]), BC[p.get("bc_x", "periodic")],
                             BC[p.get("bc_y", "periodic")], float(p.get("n_ref", 1.0)), float(p.get("t_ref", 0.05)))
    par = lbm_params(int(dim), 3, stat_c, prec_c, inv_c, len(problems), arr)
    ctx = C.c_void_p()
    _check(LIB.lbm_create(C.byref(par), C.c_void_p(stream or 0), C.byref(ctx)), None)
    return ctx


def lbm_init_riemann(ctx, problem: int, kind: str, states=(), split=(0, 0), fields=None, on_device=False):
    d = lbm_riemann_desc()
    d.kind = {"half": LBM_INIT_HALF, "quadrant": LBM_INIT_QUADRANT, "field": LBM_INIT_FIELD}[kind]
    d.x0, d.y0 = int(split[0]), int(split[1])
    for r, s in enumerate(states):
        d.s[r] = lbm_state(*[float(v) for v in s])
    keep = []
    if fields is not None:
        for name in ("n", "ux", "uy", "t"):
            a = fields[name]
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            setattr(d, name, _ptr(a))
        d.field_on_device = 1 if on_device else 0
    _check(LIB.lbm_init_riemann(ctx, int(problem), C.byref(d)), ctx)


def lbm_init_fields_f32(ctx, problem: int, n, ux, uy, t, on_device=False):
    """FIELD initialisation from float32 arrays (FP32 / BF16 deviation storage)."""
    keep = [np.ascontiguousarray(a, dtype=np.float32) if isinstance(a, np.ndarray) else a for a in (n, ux, uy, t)]
    _check(LIB.lbm_init_fields_f32(ctx, int(problem), *[_ptr(a, "float32") for a in keep], 1 if on_device else 0),
           ctx)


def lbm_step(ctx, nsteps: int):
    _check(LIB.lbm_step(ctx, int(nsteps)), ctx)


def lbm_moments(ctx, problem: int, n=None, ux=None, uy=None, T=None, mu=None, t=None, on_device=False,
                diag=False):
    dg = lbm_diag() if diag else None
    _check(LIB.lbm_moments(ctx, int(problem), _ptr(n), _ptr(ux), _ptr(uy), _ptr(T), _ptr(mu), _ptr(t),
                           1 if on_device else 0, C.byref(dg) if dg is not None else None), ctx)
    if dg is not None:
        return {"sum_n": dg.sum_n, "sum_jx": dg.sum_jx, "sum_jy": dg.sum_jy, "sum_E": dg.sum_E,
                "clamped": dg.clamped, "nonfinite": dg.nonfinite}
    return None


def lbm_moments_f32(ctx, problem: int, n=None, ux=None, uy=None, T=None, mu=None, t=None, on_device=False,
                    diag=False):
    """lbm_moments into float32 arrays (FP32 / BF16 deviation storage)."""
    dg = lbm_diag() if diag else None
    _check(LIB.lbm_moments_f32(ctx, int(problem), *[_ptr(a, "float32") for a in (n, ux, uy, T, mu, t)],
                               1 if on_device else 0, C.byref(dg) if dg is not None else None), ctx)
    if dg is not None:
        return {"sum_n": dg.sum_n, "sum_jx": dg.sum_jx, "sum_jy": dg.sum_jy, "sum_E": dg.sum_E,
                "clamped": dg.clamped, "nonfinite": dg.nonfinite}
    return None


def lbm_get_populations(ctx, problem: int, f, on_device=False):
    _check(LIB.lbm_get_populations(ctx, int(problem), _ptr(f), 1 if on_device else 0), ctx)


def lbm_set_populations(ctx, problem: int, f, on_device=False):
    _check(LIB.lbm_set_populations(ctx, int(problem), _ptr(f), 1 if on_device else 0), ctx)


def lbm_set_obstacles(ctx, problem: int, solid=None, on_device=False):
    """solid: (ny, nx) mask (NumPy bool / uint8, or a contiguous uint8 / bool
    device tensor with on_device=True); None removes the obstacles."""
    keep = None
    if solid is None:
        ptr = None
    elif isinstance(solid, np.ndarray):
        keep = np.ascontiguousarray(solid, dtype=np.uint8)
        ptr = keep.ctypes.data
    else:
        if not solid.is_contiguous() or solid.element_size() != 1:
            raise ValueError("device masks must be contiguous 1-byte tensors")
        ptr = solid.data_ptr()
    _check(LIB.lbm_set_obstacles(ctx, int(problem), ptr, 1 if on_device else 0), ctx)
    del keep


def lbm_set_force(ctx, problem: int, fx: float, fy: float = 0.0):
    _check(LIB.lbm_set_force(ctx, int(problem), float(fx), float(fy)), ctx)


def lbm_destroy(ctx):
    _check(LIB.lbm_destroy(ctx), None)


def lbm_last_error(ctx=None) -> str:
    return LIB.lbm_last_error(ctx).decode()


def lbm_launch_count(ctx) -> int:
    return int(LIB.lbm_launch_count(ctx))


def lbm_set_tiling(ctx, rows_per_tile: int, ctas: int = 0):
    _check(LIB.lbm_set_tiling(ctx, int(rows_per_tile), int(ctas)), ctx)


def lbm_get_tiling(ctx) -> dict:
    t = lbm_tiling()
    _check(LIB.lbm_get_tiling(ctx, C.byref(t)), ctx)
    return {"rows_per_tile": t.rows_per_tile, "ctas": t.ctas}


def lbm_autotune(ctx, steps_per_candidate: int = 4) -> dict:
    t = lbm_tiling()
    _check(LIB.lbm_autotune(ctx, int(steps_per_candidate), C.byref(t)), ctx)
    return {"rows_per_tile": t.rows_per_tile, "ctas": t.ctas, "ms_per_step": t.ms_per_step}


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data


def _status(st, what):
    if st != LBM_OK:
        raise LbmError(st, what)


def lbm_surrogate_targets(n, t):
    """(features, targets) of the exact forward map for host arrays n, t."""
    n, pn = _f64(n)
    t, pt = _f64(t)
    feat = np.empty((len(n), 2), dtype=np.float32)
    targ = np.empty((len(n), 2), dtype=np.float32)
    _status(LIB.lbm_surrogate_targets(pn, pt, len(n), 0, feat.ctypes.data, targ.ctypes.data, None),
            "lbm_surrogate_targets")
    return feat, targ


def lbm_surrogate_loss_grad(params, feat, targ):
    p, pp = _f32(params)
    f, pf = _f32(feat)
    g_, pg = _f32(targ)
    grad = np.empty(NPARAM, dtype=np.float32)
    loss = C.c_double()
    _status(LIB.lbm_surrogate_loss_grad(pp, pf, pg, f.shape[0], grad.ctypes.data, C.byref(loss), None),
            "lbm_surrogate_loss_grad")
    return loss.value, grad


def lbm_surrogate_train(params, n, t, n_val=None, t_val=None, epochs=32, batch=1024, lr=5e-3, lr_final=1e-6,
                        stream=None):
    """Train from initial params (not modified); returns (params, report)."""
    p = np.array(params, dtype=np.float32, copy=True)
    n, pn = _f64(n)
    t, pt = _f64(t)
    if n_val is not None:
        nv, pnv = _f64(n_val)
        tv, ptv = _f64(t_val)
        cv = len(nv)
    else:
        pnv = ptv = None
        cv = 0
    cfg = lbm_train_cfg(int(epochs), int(batch), float(lr), float(lr_final))
    rep = lbm_train_report()
    _status(LIB.lbm_surrogate_train(pn, pt, len(n), pnv, ptv, cv, 0, C.byref(cfg), p.ctypes.data, C.byref(rep),
                                    C.c_void_p(stream or 0)), "lbm_surrogate_train")
    return p, {k: getattr(rep, k) for k, _ in lbm_train_report._fields_}


def lbm_surrogate_eval(params, n, e):
    p, pp = _f32(params)
    n, pn = _f64(n)
    e, pe = _f64(e)
    T = np.empty(len(n))
    mu = np.empty(len(n))
    _status(LIB.lbm_surrogate_eval(pp, pn, pe, len(n), T.ctypes.data, mu.ctypes.data, 0, None), "lbm_surrogate_eval")
    return T, mu


def lbm_surrogate_load(ctx, params):
    p, pp = _f32(params)
    _check(LIB.lbm_surrogate_load(ctx, pp), ctx)


SURROGATE_ENGINES = {"fp32": LBM_SURROGATE_FP32_PIPE, "tensor": LBM_SURROGATE_TENSOR_CORES,
                     "mma": LBM_SURROGATE_WARP_MMA}


def lbm_surrogate_engine(ctx, engine: str = "tensor"):
    """'tensor' (tcgen05 MMAs over 128-cell tile rows, default), 'mma'
    (warp-level MMAs, activations in registers) or 'fp32' (FP32 pipe)."""
    if engine not in SURROGATE_ENGINES:
        raise ValueError(f"unknown surrogate engine {engine!r}")
    _check(LIB.lbm_surrogate_engine(ctx, SURROGATE_ENGINES[engine]), ctx)


def lbm_surrogate_wait_limit(ctx, polls: int):
    """Poll limit of the tensor-core engine's waits between layers (polls < 0:
    the default; 0: every such wait gives up at once)."""
    _check(LIB.lbm_surrogate_wait_limit(ctx, int(polls)), ctx)


def lbm_surrogate_stats(ctx, allow_timeout: bool = False) -> dict:
    """Counts since the context was created.  A timed-out tensor-core wait
    raises LbmError(LBM_ETIMEOUT) unless allow_timeout, in which case the
    counts come back with "status" and "message" set."""
    fb = C.c_int64()
    ev = C.c_int64()
    st = LIB.lbm_surrogate_stats(ctx, C.byref(fb), C.byref(ev))
    if st != LBM_OK and not (allow_timeout and st == LBM_ETIMEOUT):
        _check(st, ctx)
    out = {"fallbacks": fb.value, "evaluations": ev.value, "status": st}
    if st != LBM_OK:
        out["message"] = LIB.lbm_last_error(ctx).decode()
    return out


def lbm_conservation_sums_static(f, nx: int, ny: int, out, stat="fd", solid=None, stream=None):
    """Conservation totals of device FP64 populations f[9][ny][nx] into the
    device array out (6 doubles), without any allocation: for callers that
    may not call cudaMalloc.  solid: optional device mask (one byte per cell,
    nonzero = obstacle), left out of the totals.  Returns the status code
    (0 = LBM_OK; the message of a failure is lbm_last_error(None))."""
    sp = None
    if solid is not None:
        if not solid.is_contiguous() or solid.element_size() != 1:
            raise ValueError("the solid mask must be a contiguous 1-byte device tensor")
        sp = solid.data_ptr()
    return int(LIB.lbm_conservation_sums_static(C.c_void_p(_ptr(f)), int(nx), int(ny), C.c_void_p(sp), STAT[stat],
                                                C.c_void_p(_ptr(out)), C.c_void_p(stream or 0)))


# ---------------------------------------------------------------- convenience


class Lattice:
    """One context over a list of problems (``inputs.Problem`` objects)."""

    def __init__(self, problems, stat="fd", prec="f64", stream=None, t_ref=None, n_ref=None, inv="exact",
                 surrogate=None, dim=2, engine=None, theta=None):
        """theta: the fixed temperature of stat "ft" (sets t_ref = 2 pi theta/n_ref),
        one value for every problem or a sequence with one per problem."""
        self.problems = list(problems)
        self.q = 9 if dim == 2 else 3
        if theta is not None and np.ndim(theta) and len(theta) != len(self.problems):
            raise ValueError(f"theta: {len(theta)} values for {len(self.problems)} problems")
        descs = []
        for i, p in enumerate(self.problems):
            tr = t_ref if t_ref is not None else float(np.median(p.t)) if stat in ("fd", "ft") else 0.05
            nr = n_ref if n_ref is not None else float(np.mean(p.n))
            if theta is not None:
                th = float(theta[i]) if np.ndim(theta) else float(theta)
                tr = 2.0 * np.pi * th / nr
            descs.append(dict(nx=p.nx, ny=p.ny, tau=p.tau, bc_x=p.bc_x, bc_y=p.bc_y, n_ref=nr,
                              t_ref=min(max(tr, 1e-3), 10.0)))
        self.ctx = lbm_create(descs, stat, prec, inv=inv, stream=stream, dim=dim)
        self.stat = stat
        if surrogate is not None:
            lbm_surrogate_load(self.ctx, surrogate)
        if engine is not None:
            lbm_surrogate_engine(self.ctx, engine)

    def init(self, index=None, fields_on_device=None):
        for i, p in enumerate(self.problems):
            if index is not None and i != index:
                continue
            if p.kind in ("half", "quadrant"):
                lbm_init_riemann(self.ctx, i, p.kind, p.states, p.split)
            else:
                f = fields_on_device if fields_on_device is not None else dict(n=p.n, ux=p.ux, uy=p.uy, t=p.t)
                lbm_init_riemann(self.ctx, i, "field", fields=f, on_device=fields_on_device is not None)

    def step(self, n: int):
        lbm_step(self.ctx, n)

    def populations(self, i: int = 0) -> np.ndarray:
        p = self.problems[i]
        f = np.empty((self.q, p.ny, p.nx))
        lbm_get_populations(self.ctx, i, f)
        return f

    def set_obstacles(self, solid, i: int = 0):
        lbm_set_obstacles(self.ctx, i, solid)

    def set_force(self, fx: float, fy: float = 0.0, i: int = 0):
        lbm_set_force(self.ctx, i, fx, fy)

    def set_populations(self, f: np.ndarray, i: int = 0):
        lbm_set_populations(self.ctx, i, np.ascontiguousarray(f, dtype=np.float64))

    def fields(self, i: int = 0, diag: bool = False) -> dict:
        p = self.problems[i]
        out = {k: np.empty((p.ny, p.nx)) for k in ("n", "ux", "uy", "T", "mu", "t")}
        d = lbm_moments(self.ctx, i, diag=diag, **out)
        if diag:
            out["diag"] = d
        return out

    def close(self):
        if self.ctx:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
