"""Pins of the CPU MLP reference: backward against central finite
differences of the loss, BF16 rounding against torch, Adam on a quadratic."""
import numpy as np
import pytest

from oracle import mlp


def _params(rng, I=7, H=5, O=3):
    return {"W1": rng.standard_normal((H, I)) * 0.5, "b1": rng.standard_normal(H) * 0.1,
            "W2": rng.standard_normal((H, H)) * 0.5, "b2": rng.standard_normal(H) * 0.1,
            "W3": rng.standard_normal((O, H)) * 0.5, "b3": rng.standard_normal(O) * 0.1}


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    P = _params(rng)
    x = rng.standard_normal((4, 7))
    t = rng.standard_normal((4, 3))
    y, cache = mlp.forward(P, x)
    L, dy = mlp.mse_loss(y, t)
    g = mlp.backward(P, cache, dy)
    h = 1e-6
    for name, arr in P.items():
        num = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            old = arr[idx]
            arr[idx] = old + h
            lp, _ = mlp.mse_loss(mlp.forward(P, x)[0], t)
            arr[idx] = old - h
            lm, _ = mlp.mse_loss(mlp.forward(P, x)[0], t)
            arr[idx] = old
            num[idx] = (lp - lm) / (2 * h)
        assert np.allclose(g[name], num, rtol=1e-6, atol=1e-8), name


def test_silu_derivative():
    z = np.linspace(-6, 6, 101)
    h = 1e-6
    assert np.allclose(mlp.dsilu(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), atol=1e-8)


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.random.default_rng(1).standard_normal(1000).astype(np.float32) * 10
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(a), ref)


def test_adam_converges_on_quadratic():
    p = np.array([3.0, -2.0])
    m = np.zeros(2)
    v = np.zeros(2)
    for s in range(1, 3001):
        p, m, v = mlp.adam(p, 2 * (p - np.array([1.0, 0.5])), m, v, s, 1e-2)
    assert np.allclose(p, [1.0, 0.5], atol=1e-3)
