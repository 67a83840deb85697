"""The FMA-pipe SiLU of the tensor-core learned step: the packed FP16
constants in csrc/tc_sm100.cuh are the ones paper_1510_07328_gb300/
fit_silu_poly.py derives (Lawson's minimax fit of q(s) = s tanh s - s), and
the FP16 evaluation stays within 4e-3 of max(1, |silu|) (three times the
MUFU path's 1.1e-3; the polish absorbs it)."""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "paper_1510_07328_gb300"))
import fit_silu_poly as F  # noqa: E402


def header_constants():
    txt = open(os.path.join(ROOT, "paper_1510_07328_gb300", "csrc", "tc_sm100.cuh")).read()
    return {k: int(v, 16) for k, v in re.findall(r"(kSilu\w+) = 0x([0-9A-F]{8})u", txt)}


def half_bits(v: float) -> int:
    b = int(np.array([v], dtype=np.float16).view(np.uint16)[0])
    return (b << 16) | b


def test_header_constants_are_the_fit():
    h = header_constants()
    coef, _ = F.lawson(F.C_CLAMP, F.DEGREE)
    for k, c in zip(range(F.DEGREE, -1, -1), coef):
        assert h[f"kSiluC{k}"] == half_bits(c), k
    assert h["kSiluClamp"] == half_bits(F.C_CLAMP)
    assert h["kSiluScale"] == half_bits(2.0 / F.C_CLAMP)
    assert h["kSiluMinus1"] == half_bits(-1.0) and h["kSiluTwo"] == half_bits(2.0)


def test_fp16_evaluation_error():
    coef, e64 = F.lawson(F.C_CLAMP, F.DEGREE)
    e16, emufu = F.report(coef, F.C_CLAMP)
    assert e64 < 3e-3 and e16 < 4e-3 and emufu < 1.2e-3
    # the identity the kernel relies on: silu(z) = relu(z) + q(|z|/2)
    z = np.linspace(-30, 30, 1201)
    np.testing.assert_allclose(np.maximum(z, 0) + F.q(np.abs(z) / 2), z / (1 + np.exp(-z)), atol=1e-12)
