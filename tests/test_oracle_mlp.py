"""Pins of the FP64 selector-network oracle (oracle/mlp.py)."""
import numpy as np

from oracle import mlp

F, H, C = 7, 16, 5


def _data(seed=0, batch=11):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.4, mlp.n_params(F, H, C))
    X = rng.normal(0, 1, (batch, F))
    T = rng.normal(0, 1, (batch, C))
    mask = (rng.uniform(size=(batch, C)) > 0.3).astype(np.float64)
    mask[0, :] = 1
    return theta, X, T, mask


def test_gradient_matches_central_differences():
    theta, X, T, mask = _data()
    L, g = mlp.loss_grad(theta, X, T, mask, F, H, C)
    idx = list(range(0, len(theta), 7))
    fd = mlp.finite_difference_grad(theta, X, T, mask, F, H, C, idx)
    np.testing.assert_allclose(g[idx], fd, rtol=1e-5, atol=1e-8)


def test_loss_direct_evaluation_and_mask():
    theta, X, T, mask = _data(1)
    P = mlp.unpack(theta, F, H, C)
    h1 = np.maximum(X @ P["W1"].T + P["b1"], 0)
    h2 = np.maximum(h1 @ P["W2"].T + P["b2"], 0)
    y = h2 @ P["W3"].T + P["b3"]
    want = np.sum(mask * (y - T) ** 2) / mask.sum()
    assert abs(mlp.loss(theta, X, T, mask, F, H, C) - want) < 1e-12
    # masked entries do not contribute to the gradient of the output bias
    _, g = mlp.loss_grad(theta, X, T, np.zeros_like(mask) + np.eye(1, C, 0), F, H, C)
    gb3 = g[-C:]
    assert np.all(gb3[1:] == 0)


def test_adam_decreases_loss():
    theta, X, T, mask = _data(2, batch=64)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    L0 = mlp.loss(theta, X, T, mask, F, H, C)
    for t in range(1, 201):
        _, g = mlp.loss_grad(theta, X, T, mask, F, H, C)
        theta, m, v = mlp.adam(theta, g, m, v, t, 1e-2)
    assert mlp.loss(theta, X, T, mask, F, H, C) < 0.5 * L0
