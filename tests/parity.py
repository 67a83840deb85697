"""Comparison helpers shared by the parity tests (no GPU needed to import).

Every comparison of a CUDA result with the oracle goes through ``rel_err`` or
``max_abs_err``: a NaN or infinity in either array fails the comparison
unless both arrays hold it at the same places (a state outside the domain of
the expansion, 0 < J_2 < 2, is NaN on both sides by design).  Python's
``max(x, nan)`` returns ``x`` and a mask of finite entries hides a mismatch,
so neither appears in a parity test.
"""
from __future__ import annotations

import numpy as np


def finite_pair(got, ref) -> np.ndarray:
    """Mask of the finite entries; fails unless got and ref have their NaN and
    infinite entries at the same places, and at least one entry is finite."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.shape != ref.shape:
        raise AssertionError(f"shapes differ: {got.shape} against {ref.shape}")
    if not np.array_equal(np.isnan(got), np.isnan(ref)):
        raise AssertionError(f"NaN entries differ: {int(np.isnan(got).sum())} in the result, "
                             f"{int(np.isnan(ref).sum())} in the reference")
    gi, ri = np.isinf(got), np.isinf(ref)
    if not (np.array_equal(gi, ri) and np.array_equal(got[gi], ref[ri])):
        raise AssertionError("infinite entries differ")
    fin = np.isfinite(ref)
    if not fin.any():
        raise AssertionError("no finite entry to compare")
    return fin


def max_abs_err(got, ref) -> float:
    """max |got - ref| over the finite entries (NaN masks must agree)."""
    fin = finite_pair(got, ref)
    return float(np.abs(np.asarray(got)[fin] - np.asarray(ref)[fin]).max())


def rel_err(got, ref) -> float:
    """max |got - ref| / max |ref| over the finite entries (NaN masks must
    agree)."""
    fin = finite_pair(got, ref)
    ref = np.asarray(ref)
    return float(np.abs(np.asarray(got)[fin] - ref[fin]).max() / np.abs(ref[fin]).max())


def require_finite(a, what: str = "oracle state") -> None:
    """Fails if a holds a NaN or an infinity."""
    a = np.asarray(a)
    if not np.isfinite(a).all():
        raise AssertionError(f"{what} holds {int((~np.isfinite(a)).sum())} non-finite entries")
