"""The FP32 inversion's fits (csrc/fd_device_f32.cuh) against their
generator (paper_1510_07328_gb300/fit_x_of_j2.py, mpmath only): the header's
coefficients are the generator's; the Newton start stays within its stated
4.0e-5 of x, and the degenerate-range fit within 1e-8 relative, on points the
fits did not use; the branch thresholds are 3/2 - J_2(7) and 3/2 - J_2(17)."""
import os
import re
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_1510_07328_gb300"))
mp = pytest.importorskip("mpmath")
import fit_x_of_j2 as gen  # noqa: E402

HEADER = os.path.join(ROOT, "paper_1510_07328_gb300", "csrc", "fd_device_f32.cuh")


def header_constants():
    src = open(HEADER).read()
    body = re.search(r"x_start_general\(float J2\) \{\s*constexpr float c\[9\] = \{([^}]*)\}", src).group(1)
    coeffs = [float(v.strip().rstrip("f")) for v in body.split(",")]
    delta7 = float(re.search(r"kDelta7 = ([0-9.e+-]+)f", src).group(1))
    return np.array(coeffs), delta7


def header_degenerate():
    src = open(HEADER).read()
    body = re.search(r"x_degenerate_fit\(float delta\) \{\s*constexpr float c\[9\] = \{([^}]*)\}", src).group(1)
    coeffs = np.array([float(v.strip().rstrip("f")) for v in body.split(",")])
    m, ih = (float(v) for v in re.search(r"\(__logf\(delta\) \+ ([0-9.]+)f\) \* ([0-9.]+)f", src).groups())
    delta17 = float(re.search(r"kDelta17 = ([0-9.e+-]+)f", src).group(1))
    return coeffs, -m, ih, delta17


def test_header_matches_generator():
    c_hdr, _ = header_constants()
    c_gen, err = gen.fit()
    np.testing.assert_allclose(c_hdr, c_gen, rtol=1e-8, atol=1e-14)
    assert err < 4.1e-5


def test_fit_accuracy_off_the_fit_points_and_threshold():
    c_hdr, delta7 = header_constants()
    mp.mp.dps = 30
    x_lo = float(mp.log(mp.e ** mp.mpf("0.1") - 1))
    xs = x_lo + (7.3 - x_lo) * (np.arange(37) + 0.37) / 37  # points between the fit's samples
    J = np.array([float(gen.j2(x)) for x in xs])
    v = np.log((J - 1.0) / (1.5 - J))
    assert np.abs(np.polyval(c_hdr, v) - xs).max() < 4.5e-5
    assert abs(delta7 - float(1.5 - gen.j2(7))) < 1e-8


def test_degenerate_fit_matches_generator_and_holds():
    c_hdr, m_hdr, ih_hdr, d17_hdr = header_degenerate()
    c_gen, m, h, err, d7, d17 = gen.fit_degenerate()
    np.testing.assert_allclose(c_hdr, c_gen, rtol=1e-8, atol=1e-13)
    assert abs(m_hdr - m) < 1e-8 and abs(ih_hdr - 1.0 / h) < 1e-8
    assert abs(d17_hdr - d17) < 1e-8 and err < 1e-8
    mp.mp.dps = 30
    xs = 7.0 + 10.0 * (np.arange(29) + 0.41) / 29  # points between the fit's samples
    d = np.array([float(1.5 - gen.j2(x)) for x in xs])
    u = (np.log(d) - m) / h
    assert (np.abs(np.polyval(c_hdr, u) - xs) / xs).max() < 1e-8
