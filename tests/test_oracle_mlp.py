"""Pins of the FP64 reference network used to check the surrogate's gradients. CPU only."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_matches_normal_cdf():
    st = pytest.importorskip("scipy.stats")
    z = np.linspace(-6, 6, 101)
    assert np.allclose(mlp.gelu(z), z * st.norm.cdf(z), atol=1e-14)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def test_encoding_ranges():
    x = np.array([[0.0, -30.0, 1e9], [90.0, 30.0, 12e9], [180.0, 0.0, math.sqrt(12) * 1e9]])
    e = mlp.encode(x)
    assert np.allclose(e[:, 0], [0, 1, 0], atol=1e-15) and np.allclose(e[:, 1], [1, 0, -1], atol=1e-15)
    assert np.allclose(e[:, 2], [-1, 1, 0]) and np.allclose(e[:, 3], [-1, 1, 0])


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    width, depth, nf = 6, 3, 8
    _, n = mlp.layout(width, depth, nf)
    p = rng.normal(0, 0.5, n)
    B = rng.normal(0, 1.0, (nf // 2, 4))
    x = np.stack([rng.uniform(0, 360, 5), rng.uniform(-30, 30, 5), np.exp(rng.uniform(np.log(1e9), np.log(12e9), 5))], 1)
    t = rng.normal(size=(5, 4))
    loss, g, _ = mlp.loss_and_grads(p, B, x, t, width, depth, nf)
    h = 1e-6
    for i in rng.choice(n, 40, replace=False):
        e = np.zeros(n)
        e[i] = h
        fd = (mlp.loss_and_grads(p + e, B, x, t, width, depth, nf)[0]
              - mlp.loss_and_grads(p - e, B, x, t, width, depth, nf)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])
