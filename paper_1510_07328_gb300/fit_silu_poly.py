"""Generator of the FMA-pipe SiLU of the tensor-core learned step
(csrc/tc_sm100.cuh, silu2_poly).

With h = z/2 (the hidden layers hold z/2 in FP16),
    silu(z) = z / (1 + e^{-z}) = relu(z) + q(|h|),   q(s) = s tanh(s) - s,
because h tanh(h) is even in h and h + |h| = relu(z).  q is a bump:
q(0) = 0, minimum -0.28 near s = 0.64, and |q(s)| < 2 s e^{-2 s}, so that
q(4.5) = -1.1e-3.  The kernel evaluates
    silu(z) ~ 2 max(h, 0) + P(t),   t = min(|h|, c) (2/c) - 1,
with P of degree d in t, by Horner's rule in packed FP16 (FMA pipe only: one
FP16 multiply-add per degree), so that part of a layer's activations bypass
the MUFU unit.

P is the minimax approximation of q(c (t + 1)/2) on t in [-1, 1] found by
Lawson's algorithm (iteratively reweighted least squares, C. L. Lawson, 1961)
on Chebyshev nodes.  The clamp at c adds the tail |q(c)| to the error.
The script reports the largest error of the FP64 fit and of the FP16
evaluation (every operation rounded to FP16), measured as
|approximation - silu(z)| / max(1, |silu(z)|) over z in [-24, 24], beside the
same measure for the MUFU path (tanh rounded to FP16, one FP16 multiply-add).

Run: python paper_1510_07328_gb300/fit_silu_poly.py  (prints the
coefficients, highest degree first).
"""
import numpy as np

C_CLAMP = 4.5
DEGREE = 6


def q(s):
    return s * np.tanh(s) - s


def lawson(c: float, d: int, nodes: int = 4000, iters: int = 200):
    """Minimax polynomial of degree d for q(c (t + 1)/2), t in [-1, 1]."""
    t = np.cos(np.linspace(0.0, np.pi, nodes))
    f = q(c * (t + 1.0) / 2.0)
    V = np.vander(t, d + 1)
    w = np.full(nodes, 1.0 / nodes)
    coef = None
    for _ in range(iters):
        sw = np.sqrt(w)
        coef, *_ = np.linalg.lstsq(V * sw[:, None], f * sw, rcond=None)
        e = np.abs(V @ coef - f)
        w = w * e
        w /= w.sum()
    return coef, float(np.abs(V @ coef - f).max())


def fp16_eval(coef, c: float, h: np.ndarray) -> np.ndarray:
    """The kernel's evaluation with every operation rounded to FP16."""
    h16 = h.astype(np.float16)
    s = np.minimum(np.abs(h16), np.float16(c))
    t = (s * np.float16(2.0 / c) + np.float16(-1.0)).astype(np.float16)
    p = np.float16(coef[0])
    for a in coef[1:]:
        p = (p * t + np.float16(a)).astype(np.float16)
    return (np.maximum(h16, np.float16(0.0)) * np.float16(2.0) + p).astype(np.float16)


def report(coef, c: float):
    h = np.linspace(-12.0, 12.0, 480001).astype(np.float16).astype(np.float64)
    z = 2.0 * h
    ref = z / (1.0 + np.exp(-z))
    scale = np.maximum(1.0, np.abs(ref))
    poly = fp16_eval(coef, c, h).astype(np.float64)
    t16 = np.tanh(h).astype(np.float16).astype(np.float64)
    mufu = (h + h * t16).astype(np.float16).astype(np.float64)
    return float((np.abs(poly - ref) / scale).max()), float((np.abs(mufu - ref) / scale).max())


if __name__ == "__main__":
    coef, e64 = lawson(C_CLAMP, DEGREE)
    e16, em = report(coef, C_CLAMP)
    print(f"clamp c = {C_CLAMP}, degree {DEGREE}: minimax error {e64:.3e} (plus tail {abs(q(C_CLAMP)):.1e})")
    print(f"FP16 evaluation: {e16:.3e} of max(1, |silu|); MUFU path: {em:.3e}")
    print("coefficients, highest degree first:")
    print(", ".join(f"{v:.9e}f" for v in coef))
