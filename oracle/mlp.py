"""CPU reference of the warm-start MLP -- TEST INFRASTRUCTURE ONLY.

Plain numpy float64 forward and backward passes of the network the library
trains on the GPU (three linear layers with SiLU between them), on the same
BF16-rounded weights and inputs, and the Adam update.  Used to check the
library's hand-written training kernels.  Pinned by central finite
differences (tests/test_mlp_oracle.py).
"""
from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """Round float32 values to bfloat16 (round to nearest even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, x):
    """params: dict W1 [H,I], b1 [H], W2 [H,H], b2 [H], W3 [O,H], b3 [O]; x: [B,I].
    Returns y [B,O] and the cache for backward."""
    z1 = x @ params["W1"].T + params["b1"]
    h1 = silu(z1)
    z2 = h1 @ params["W2"].T + params["b2"]
    h2 = silu(z2)
    y = h2 @ params["W3"].T + params["b3"]
    return y, (x, z1, h1, z2, h2)


def mse_loss(y, t):
    """Mean over the batch of the squared error summed over outputs."""
    d = y - t
    return float(np.sum(d * d) / y.shape[0]), 2.0 * d / y.shape[0]


def backward(params, cache, dy):
    x, z1, h1, z2, h2 = cache
    g = {}
    g["W3"] = dy.T @ h2
    g["b3"] = dy.sum(0)
    dh2 = dy @ params["W3"]
    dz2 = dh2 * dsilu(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dh1 = dz2 @ params["W2"]
    dz1 = dh1 * dsilu(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return g


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) on float64 copies; returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
