"""Plain FP64 reference of the learned Fermi-Dirac inversion (surrogate).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The surrogate replaces the per-cell inversion J_2 -> x of the method (the FD
form of I_2N, Sect. "Generalized polynomials in D dimensions") by a small
network that maps the cell's density and internal energy (n, e) to its
temperature and chemical potential (T, mu).  The paper has no network; this
module restates the network and its training loss plainly so that the CUDA
training kernels can be checked:

* inputs    (n, e) with e = sum f |e_a - u_0|^2 = D n J_2 / 3 (D = 2), the
  internal energy in lattice units; the fixed input embedding is
  n_hat = (n - 1.25)/0.75 and l_hat = (ln delta + 5.3)/3.7 with
  delta = 3/2 - 3 e/(2 n) = 3/2 - J_2 (the temperature enters the FD
  moments through this difference, ln T ~ ln delta / 2 near degeneracy)
* layers    z1 = W1 x + b1 (64), h1 = silu(z1), z2 = W2 h1 + b2 (64),
            h2 = silu(z2), y = W3 h2 + b3 (2); silu(z) = z / (1 + e^{-z})
* outputs   y_0 = (ln T - LNT_MID)/LNT_HALF, y_1 = (mu - MU_MID)/MU_HALF
            (LNT_HALF = 0.5 weights the temperature, which sets x = mu/T)
* loss      mean over the batch of sum_o (y_o - target_o)^2
* targets   from the exact forward map of the method: x = x(t),
            J_2 = J_2(x), e = 2 n J_2 / 3, T = n t/(2 pi), mu = T x

Parameter vector (4482 entries, this order): W1 [64][2], b1 [64],
W2 [64][64], b2 [64], W3 [2][64], b3 [2] (row-major, [out][in]).
"""
from __future__ import annotations

import math

import numpy as np

from . import fd as _fd

H = 64
NPARAM = H * 2 + H + H * H + H + 2 * H + 2
N_MID, N_HALF = 1.25, 0.75
LD_MID, LD_HALF = -5.3, 3.7
LNT_MID, LNT_HALF = -5.09, 0.5
MU_MID, MU_HALF = 0.1985, 0.12


def unpack(p: np.ndarray):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + 2 * H].reshape(H, 2); o += 2 * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + 2 * H].reshape(2, H); o += 2 * H
    b3 = p[o:o + 2]; o += 2
    assert o == NPARAM
    return W1, b1, W2, b2, W3, b3


def features(n, e):
    n = np.asarray(n, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    delta = 1.5 - 1.5 * e / n
    return np.stack([(n - N_MID) / N_HALF, (np.log(delta) - LD_MID) / LD_HALF], axis=-1)


def targets_from_state(n, t):
    """Exact forward map (n, t) -> features (n, e) and normalised (ln T, mu)."""
    n = np.asarray(n, dtype=np.float64)
    x = _fd.x_of_t(t)
    j2 = _fd.j2_of_x(x)
    e = 2.0 * n * j2 / 3.0
    T = n * np.asarray(t, dtype=np.float64) / (2.0 * math.pi)
    mu = T * x
    y = np.stack([(np.log(T) - LNT_MID) / LNT_HALF, (mu - MU_MID) / MU_HALF], axis=-1)
    return n, e, y, T, mu


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, X):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    z1 = X @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    y = h2 @ W3.T + b3
    return y, (z1, h1, z2, h2)


def loss_and_grad(p, X, Y):
    """Mean squared error over the batch and its gradient (backpropagation
    written out layer by layer)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    y, (z1, h1, z2, h2) = forward(p, X)
    B = X.shape[0]
    r = y - Y
    loss = float((r * r).sum() / B)
    dy = 2.0 * r / B
    gW3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dz2 = (dy @ W3) * dsilu(z2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * dsilu(z1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def predict(p, n, e):
    """(T, mu) from the network."""
    y, _ = forward(p, features(n, e))
    T = np.exp(y[:, 0] * LNT_HALF + LNT_MID)
    mu = y[:, 1] * MU_HALF + MU_MID
    return T, mu
