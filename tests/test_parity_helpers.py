"""The comparison helpers of the parity tests (tests/parity.py), on the CPU.

A NaN planted in an oracle state on the host must turn a comparison red,
whichever side holds it; NaN at the same places on both sides (the cells
outside the expansion's domain) compares equal there and leaves the rest to
the tolerance.
"""
import numpy as np
import pytest

from oracle import lbm as olbm
from paper_1510_07328_gb300 import inputs
from parity import finite_pair, max_abs_err, rel_err, require_finite


def _state():
    p = inputs.random_field(40, 3, 5, tau=0.8)
    return olbm.init_equilibrium(p.n, p.ux, p.uy, p.t)


def test_nan_planted_in_the_oracle_state_fails():
    ref = _state()
    got = ref * (1.0 + 1e-14)
    assert rel_err(got, ref) < 1e-13
    bad = ref.copy()
    bad[3, 1, 7] = np.nan
    with pytest.raises(AssertionError):
        rel_err(got, bad)
    with pytest.raises(AssertionError):
        require_finite(bad)
    # the pattern the helpers replace: Python's max() drops the NaN silently
    worst = max(0.0, float(np.abs(got - bad).max() / np.abs(bad).max()))
    assert worst == 0.0


def test_nan_on_the_cuda_side_fails():
    ref = _state()
    got = ref.copy()
    got[0, 0, 0] = np.nan
    with pytest.raises(AssertionError):
        max_abs_err(got, ref)
    got[0, 0, 0] = np.inf
    with pytest.raises(AssertionError):
        max_abs_err(got, ref)


def test_shared_nan_cells_compare_equal_and_rest_is_checked():
    ref = _state()
    ref[:, 1, 4] = np.nan  # one cell outside the domain, all nine populations
    got = ref.copy()
    assert rel_err(got, ref) == 0.0
    got[2, 0, 0] *= 1.0 + 1e-6
    assert rel_err(got, ref) > 1e-7
    assert finite_pair(got, ref).sum() == ref.size - 9


def test_all_nan_has_nothing_to_compare():
    a = np.full((9, 2, 2), np.nan)
    with pytest.raises(AssertionError):
        rel_err(a, a.copy())
