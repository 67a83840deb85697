"""Pins for oracle/mlp.py (the surrogate's reference network and loss).

The backpropagation is checked against central finite differences of the
loss, and the targets against the exact forward map of the method."""
import math

import numpy as np

from oracle import fd, mlp
from paper_1510_07328_gb300 import inputs


def init_params(seed):
    r = inputs.uniform(seed, mlp.NPARAM)
    return (2 * r - 1) * 0.3


def test_gradient_matches_finite_differences():
    p = init_params(3)
    n, t = inputs.surrogate_set(16, seed=5)
    _, e, Y, _, _ = mlp.targets_from_state(n, t)
    X = mlp.features(n, e)
    loss, g = mlp.loss_and_grad(p, X, Y)
    rng = np.random.default_rng(0)
    idx = np.concatenate([np.arange(0, 4), np.arange(128, 132), rng.integers(0, mlp.NPARAM, 40),
                          np.arange(mlp.NPARAM - 4, mlp.NPARAM)])
    h = 1e-6
    for i in idx:
        d = np.zeros_like(p)
        d[i] = h
        num = (mlp.loss_and_grad(p + d, X, Y)[0] - mlp.loss_and_grad(p - d, X, Y)[0]) / (2 * h)
        assert abs(num - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, num, g[i])


def test_targets_are_the_exact_forward_map():
    n = np.array([0.7, 1.3])
    t = np.array([0.02, 0.2])
    nn, e, Y, T, mu = mlp.targets_from_state(n, t)
    x = fd.x_of_t(t)
    np.testing.assert_allclose(e, 2 * n * fd.j2_of_x(x) / 3)
    np.testing.assert_allclose(T, n * t / (2 * math.pi))
    np.testing.assert_allclose(mu / T, x)
    # normalised features of the training range stay within [-1, 1], targets O(1)
    n, t = inputs.surrogate_set(20000, seed=4)
    _, e, Y, _, _ = mlp.targets_from_state(n, t)
    assert np.abs(Y[:, 0]).max() < 6.0 and np.abs(Y[:, 1]).max() < 1.5
    assert np.abs(mlp.features(n, e)).max() <= 1.0 + 1e-3
    # the embedding is ln(3/2 - J_2)
    np.testing.assert_allclose(mlp.features(n, e)[:, 1] * mlp.LD_HALF + mlp.LD_MID,
                               np.log(1.5 - fd.j2_of_x(fd.x_of_t(t))), rtol=1e-12)


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    np.testing.assert_allclose(mlp.dsilu(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_network_domain_constants_match_the_forward_map():
    """The kernels send a cell through the network only inside its training
    domain, n in [0.5, 2] and t in [0.005, 0.3], tested on delta = 3/2 - J_2.
    The delta limits written in the CUDA header are the exact forward map's
    values at the ends of the t range (FP32-rounded), and the n limits are
    the training range of inputs.surrogate_set."""
    import os
    import re

    from oracle import fd
    from paper_1510_07328_gb300 import inputs

    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            "paper_1510_07328_gb300", "csrc", "surrogate.cuh")).read()
    val = {k: float(v) for k, v in re.findall(r"(kSur(?:Delta|N)(?:Lo|Hi)) = ([0-9.e+-]+)f", hdr)}
    for t, key in ((0.005, "kSurDeltaLo"), (0.3, "kSurDeltaHi")):
        delta = 1.5 - float(fd.j2_of_x(fd.x_of_t(np.array([t])))[0])
        assert abs(val[key] - delta) <= 1e-7 * delta, (key, val[key], delta)
    n, t = inputs.surrogate_set(4096, seed=4)
    assert val["kSurNLo"] <= n.min() and n.max() <= val["kSurNHi"]
    assert abs(n.min() - val["kSurNLo"]) < 0.01 and abs(n.max() - val["kSurNHi"]) < 0.01
    assert 0.005 <= t.min() and t.max() <= 0.3
