"""The FP32 inversion's fits (csrc/fd_device_f32.cuh) against their
generator (paper_1510_07328_gb300/fit_x_of_j2.py, mpmath only): the header's
coefficients are the generator's; the Newton start stays within its stated
4.0e-5 of x, and the degenerate-range fit within 1e-8 relative, on points the
fits did not use; the branch thresholds are 3/2 - J_2(7) and 3/2 - J_2(17).
The three polynomials that give J_4 straight from delta = 3/2 - J_2 (x >= 17,
7 < x < 17 and x_lo < x <= 7) are the generator's and hold against the
polylogarithm's J_4, in exact arithmetic and in the header's FP32
evaluation."""
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


def header_j4_polys():
    src = open(HEADER).read()
    deg = re.search(r"j4_degenerate_poly\(float delta\) \{\s*constexpr float c\[5\] = \{([^}]*)\}", src).group(1)
    mid = re.search(r"j4_mid_poly\(float delta\) \{\s*constexpr float c\[8\] = \{([^}]*)\}", src).group(1)
    ih, m_ih, ih2 = re.search(r"fmaf\(delta, ([0-9.e+-]+)f, -([0-9.e+-]+)f \* ([0-9.e+-]+)f\)", src).groups()
    assert ih == ih2
    cd = np.array([float(v.strip().rstrip("f")) for v in deg.split(",")])
    cm = np.array([float(v.strip().rstrip("f")) for v in mid.split(",")])
    return cd, cm, float(m_ih), float(ih)


def header_j4_low():
    src = open(HEADER).read()
    body = re.search(r"j4_low_poly\(float delta\) \{\s*constexpr float c\[13\] = \{([^}]*)\}", src).group(1)
    ih, m_ih, ih2 = re.search(r"j4_low_poly.*?fmaf\(delta, ([0-9.e+-]+)f, -([0-9.e+-]+)f \* ([0-9.e+-]+)f\)", src,
                              re.S).groups()
    assert ih == ih2
    return np.array([float(v.strip().rstrip("f")) for v in body.split(",")]), float(m_ih), float(ih)


def horner_fp32(c, v):
    """The header's Horner evaluation in FP32, each step one rounding (fmaf)."""
    c32 = np.asarray(c, dtype=np.float32).astype(np.float64)
    v = np.asarray(v, dtype=np.float32).astype(np.float64)
    y = np.full_like(v, c32[0])
    for k in range(1, len(c32)):
        y = (y * v + c32[k]).astype(np.float32).astype(np.float64)
    return y


def test_j4_polynomials_match_generator():
    cd, cm, m_hdr, ih_hdr = header_j4_polys()
    c_gen, err, _ = gen.fit_j4_degenerate()
    np.testing.assert_allclose(cd, c_gen, rtol=1e-8, atol=1e-12)
    assert err < 2e-10
    c_gen, m, h, err = gen.fit_j4_mid()
    np.testing.assert_allclose(cm, c_gen, rtol=1e-8, atol=1e-14)
    assert abs(m_hdr - m) < 1e-10 and abs(ih_hdr - 1.0 / h) < 1e-6 and err < 2e-9


def test_j4_polynomials_against_polylog_off_the_fit_points():
    """J_4 from delta against J_4 = f_3^2/(f_2 f_4) of mpmath's polylogarithm
    at points the fits did not use: x in [17, 300] for the degenerate
    polynomial (its dropped tails are below 3.4e-9 there) and x in (7, 17)
    for the middle one; exact arithmetic within 4e-9 and 2e-9, and the
    header's FP32 evaluation within 2 FP32 ulps of J_4."""
    cd, cm, m_ih, ih = header_j4_polys()
    mp.mp.dps = 30
    ulp = 2.0 ** -23
    xs = np.concatenate([17.0 + 13.0 * (np.arange(23) + 0.37) / 23, 30.0 + 270.0 * (np.arange(11) + 0.5) / 11])
    d = np.array([float(1.5 - gen.j2(x)) for x in xs])
    J = np.array([float(gen.j4(x)) for x in xs])
    assert (np.abs(np.polyval(cd, d) - J) / J).max() < 4e-9
    assert (np.abs(horner_fp32(cd, d) - J) / J).max() < 2 * ulp
    xs = 7.0 + 10.0 * (np.arange(31) + 0.43) / 31
    d = np.array([float(1.5 - gen.j2(x)) for x in xs])
    J = np.array([float(gen.j4(x)) for x in xs])
    v = d * ih - m_ih * ih
    assert (np.abs(np.polyval(cm, v) - J) / J).max() < 2e-9
    v32 = (np.float32(d) * np.float32(ih)).astype(np.float64) - np.float32(np.float32(m_ih) * np.float32(ih))
    assert (np.abs(horner_fp32(cm, v32) - J) / J).max() < 2 * ulp


def test_j4_closed_form_is_the_degenerate_limit():
    """The degenerate polynomial's target: 4/3 at delta = 0, and equal to the
    polylogarithm's J_4 to the size of the dropped tails at x = 17 and 40."""
    mp.mp.dps = 30
    assert abs(float(gen.j4_closed_form(0.0)) - 4.0 / 3.0) < 1e-15
    for x, tol in ((17.0, 4e-9), (40.0, 1e-15)):
        d = 1.5 - gen.j2(x)
        assert abs(float(gen.j4_closed_form(d) / gen.j4(x)) - 1.0) < tol


def test_j4_low_polynomial_matches_generator_and_holds():
    """The polynomial that replaces the Newton iteration's J_4 for
    x_lo < x <= 7 (x_lo = x(t = 10)): the generator's coefficients, and
    within 1e-9 of the polylogarithm's J_4 off the fit points in exact
    arithmetic, within 2 FP32 ulps in the header's FP32 evaluation."""
    c_hdr, m_ih, ih = header_j4_low()
    c_gen, m, h, err = gen.fit_j4_low()
    np.testing.assert_allclose(c_hdr, c_gen, rtol=1e-8, atol=1e-15)
    assert abs(m_ih - m) < 1e-10 and abs(ih - 1.0 / h) < 1e-6 and err < 1e-9
    mp.mp.dps = 30
    x_lo = float(mp.log(mp.e ** mp.mpf("0.1") - 1))
    xs = x_lo + (7.0 - x_lo) * (np.arange(41) + 0.47) / 41
    d = np.array([float(1.5 - gen.j2(x)) for x in xs])
    J = np.array([float(gen.j4(x)) for x in xs])
    v = d * ih - m_ih * ih
    assert (np.abs(np.polyval(c_hdr, v) - J) / J).max() < 1e-9
    v32 = (np.float32(d) * np.float32(ih)).astype(np.float64) - np.float32(np.float32(m_ih) * np.float32(ih))
    assert (np.abs(horner_fp32(c_hdr, v32) - J) / J).max() < 2 * 2.0 ** -23
