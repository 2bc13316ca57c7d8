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


def test_adam_three_steps_hand_worked():
    """Three Adam steps with carried moments, worked by hand (Kingma & Ba
    2015, Algorithm 1) with beta1 = 1/2, beta2 = 3/4, eps = 0, lr = 1 and
    gradients 1, -1, 2 from w = 0, m = v = 0:
      t = 1: m = 1/2,     v = 1/4;           m^ = 1,    v^ = 1     -> w = -1
      t = 2: m = 1/4 - 1/2 = -1/4,  v = 3/16 + 1/4 = 7/16;
             m^ = (-1/4) / (3/4) = -1/3, v^ = (7/16) / (7/16) = 1  -> w = -2/3
      t = 3: m = -1/8 + 1 = 7/8,  v = 21/64 + 1 = 85/64;
             m^ = (7/8) / (7/8) = 1, v^ = (85/64) / (37/64) = 85/37
                                                   -> w = -2/3 - sqrt(37/85)
    Steps 2 and 3 start from nonzero moments, so a dropped beta1 * m or
    beta2 * v term, or a missing bias correction, changes w."""
    w, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    want_w = [-1.0, -2.0 / 3.0, -2.0 / 3.0 - math.sqrt(37.0 / 85.0)]
    want_m = [0.5, -0.25, 0.875]
    want_v = [0.25, 7.0 / 16.0, 85.0 / 64.0]
    for t, g in enumerate([1.0, -1.0, 2.0], start=1):
        w, m, v = mlp.adam_step(w, np.array([g]), m, v, t, 1.0, beta1=0.5, beta2=0.75, eps=0.0)
        assert w[0] == pytest.approx(want_w[t - 1], rel=1e-14, abs=1e-15)
        assert m[0] == pytest.approx(want_m[t - 1], rel=1e-14)
        assert v[0] == pytest.approx(want_v[t - 1], rel=1e-14)


def test_adam_matches_torch_optimizer_float64():
    """Five steps against torch.optim.Adam (an independent implementation)
    in float64 with varying gradients; the oracle carries m and v between
    calls exactly as the optimizer's state does."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    w0 = rng.normal(size=17)
    grads = [rng.normal(size=17) * s for s in (1.0, 0.3, 2.0, 0.01, 5.0)]
    p = torch.nn.Parameter(torch.tensor(w0, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=0.05, betas=(0.8, 0.95), eps=1e-6)
    w, m, v = w0.copy(), np.zeros(17), np.zeros(17)
    for t, g in enumerate(grads, start=1):
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        w, m, v = mlp.adam_step(w, g, m, v, t, 0.05, beta1=0.8, beta2=0.95, eps=1e-6)
        assert np.allclose(w, p.detach().numpy(), rtol=1e-13, atol=1e-15)
