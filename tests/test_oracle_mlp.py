"""Pins for the learned-projection oracle (oracle/mlp.py): closed forms of
gelu and the loss, central finite differences for every gradient, and the
first Adam step."""
import math

import numpy as np
import pytest

from oracle import mlp


def _net(rng, d=6, h=10, dy=5, scale=0.5):
    return (rng.normal(0, scale, (h, d)), rng.normal(0, 0.1, h),
            rng.normal(0, scale, (dy, h)), rng.normal(0, 0.1, dy))


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([10.0]))[0] == pytest.approx(10.0, abs=1e-12)
    assert abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-12
    # gelu(x) = x * Phi(x); Phi(1) = 0.841344746...
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-12)
    assert mlp.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-15)
    x = np.linspace(-4, 4, 41)
    fd = (mlp.gelu(x + 1e-6) - mlp.gelu(x - 1e-6)) / 2e-6
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-8)


def test_forward_shapes_and_bias_only():
    rng = np.random.default_rng(0)
    W1, b1, W2, b2 = _net(rng)
    X = rng.normal(size=(7, 6))
    Y, H, A = mlp.forward(X, W1, b1, np.zeros_like(W2), b2)
    assert Y.shape == (7, 5) and H.shape == (7, 10)
    assert np.allclose(Y, b2)                          # W2 = 0: y = b2
    assert np.allclose(H, X @ W1.T + b1)


def test_pair_loss_closed_forms():
    Y = np.array([[1.0, 0.0], [2.0, 0.0], [0.0, 3.0], [-1.0, 0.0]])
    ia, ib = np.array([0, 0, 0]), np.array([1, 2, 3])
    # cos = 1, 0, -1
    loss, _ = mlp.pair_loss(Y, ia, ib, np.array([1, 1, 0]), 0.9, 0.5)
    assert loss == pytest.approx((0.0 + 0.9 + 0.0) / 3)
    loss, _ = mlp.pair_loss(Y, ia, ib, np.array([0, 0, 1]), 0.9, 0.5)
    assert loss == pytest.approx((0.5 + 0.0 + 1.9) / 3)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradients_match_finite_differences(seed):
    rng = np.random.default_rng(seed)
    W1, b1, W2, b2 = _net(rng)
    X = rng.normal(size=(12, 6))
    ia = rng.integers(0, 12, 20)
    ib = (ia + 1 + rng.integers(0, 11, 20)) % 12
    label = rng.integers(0, 2, 20)
    mp, mn = 0.95, 0.2
    loss, grads = mlp.loss_and_grads(X, W1, b1, W2, b2, ia, ib, label, mp, mn)
    params = [W1, b1, W2, b2]
    for p, g in zip(params, grads):
        flat = p.reshape(-1)
        for idx in rng.choice(flat.size, min(8, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + 1e-6
            lp, _ = mlp.loss_and_grads(X, W1, b1, W2, b2, ia, ib, label, mp, mn)
            flat[idx] = old - 1e-6
            lm, _ = mlp.loss_and_grads(X, W1, b1, W2, b2, ia, ib, label, mp, mn)
            flat[idx] = old
            fd = (lp - lm) / 2e-6
            assert g.reshape(-1)[idx] == pytest.approx(fd, rel=1e-4, abs=1e-7)


def test_first_adam_step_is_signed_lr():
    w = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 0.0])
    w2, m, v = mlp.adam_step(w, g, np.zeros(3), np.zeros(3), 1, 0.01)
    # m_hat / sqrt(v_hat) = g / |g| on the first step
    assert np.allclose(w2, w - 0.01 * np.array([1.0, -1.0, 0.0]), atol=1e-6)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
