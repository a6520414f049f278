"""FP64 numpy reference of the surrogate network, for gradient checks.

TEST INFRASTRUCTURE ONLY (imported by tests/). Same architecture and parameter
layout as the surrogate of the library: inputs (az deg, el deg, f Hz) ->
(sin az, cos az, el / 30, 2 ln(f / 1 GHz) / ln 12 - 1) -> Fourier features
[sin 2 pi B x, cos 2 pi B x] -> `depth` layers z = h W^T + b, h = GELU(z) ->
y = h W_head^T + b_head (4 outputs); loss = mean of (y - t)^2 over all entries.
GELU(z) = z Phi(z) with Phi the standard normal CDF. Parameters are one flat
vector [W_0, b_0, W_1, b_1, ..., W_head, b_head], each W row-major [out][in].
"""
from __future__ import annotations

import math

import numpy as np


def _erf(x):
    return np.vectorize(math.erf, otypes=[np.float64])(x)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def encode(x):
    x = np.asarray(x, np.float64)
    az = np.radians(x[:, 0])
    return np.stack([np.sin(az), np.cos(az), x[:, 1] / 30.0, 2.0 * np.log(x[:, 2] / 1e9) / np.log(12.0) - 1.0], 1)


def layout(width, depth, n_fourier):
    """[(W offset, W shape, b offset, b size)] for the hidden layers and the head."""
    out, off = [], 0
    for l in range(depth + 1):
        k = n_fourier if l == 0 else width
        n = width if l < depth else 4
        out.append((off, (n, k), off + n * k, n))
        off += n * k + n
    return out, off


def unpack(p, width, depth, n_fourier):
    lay, _ = layout(width, depth, n_fourier)
    p = np.asarray(p, np.float64)
    return [(p[o:o + s[0] * s[1]].reshape(s), p[ob:ob + nb]) for o, s, ob, nb in lay]


def loss_and_grads(p, B, x, t, width, depth, n_fourier):
    """Mean squared error and its gradient with respect to the flat parameter vector."""
    Ws = unpack(p, width, depth, n_fourier)
    x4 = encode(x)
    arg = 2.0 * np.pi * (x4 @ np.asarray(B, np.float64).T)
    h = [np.concatenate([np.sin(arg), np.cos(arg)], 1)]
    zs = []
    for l in range(depth):
        W, b = Ws[l]
        z = h[-1] @ W.T + b
        zs.append(z)
        h.append(gelu(z))
    Wh, bh = Ws[depth]
    y = h[-1] @ Wh.T + bh
    t = np.asarray(t, np.float64)
    n = y.size
    loss = float(np.mean((y - t) ** 2))
    dy = 2.0 * (y - t) / n
    grads = [None] * (depth + 1)
    grads[depth] = (dy.T @ h[depth], dy.sum(0))
    dh = dy @ Wh
    for l in range(depth - 1, -1, -1):
        dz = dh * gelu_grad(zs[l])
        grads[l] = (dz.T @ h[l], dz.sum(0))
        dh = dz @ Ws[l][0]
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in grads])
    return loss, flat, y
