"""FP64 reference of the selector network -- TEST INFRASTRUCTURE ONLY.

Parity: pinned (tests/test_oracle_mlp.py: analytic gradients against central
finite differences in FP64; the loss against a direct evaluation).

The network predicts one value per candidate mapping from a descriptor's
feature vector:  H1 = relu(X W1^T + b1),  H2 = relu(H1 W2^T + b2),
Y = H2 W3^T + b3, with W1: [h, f], W2: [h, h], W3: [c, h].  The loss is the
masked mean squared error  L = sum(mask * (Y - T)^2) / sum(mask).
Parameters are one flat vector in the order W1, b1, W2, b2, W3, b3 (row-major
weights), the layout the library's kernels use.
"""
from __future__ import annotations

from typing import Dict, Tuple

import numpy as np


def shapes(n_in: int, n_hidden: int, n_out: int):
    return [("W1", (n_hidden, n_in)), ("b1", (n_hidden,)), ("W2", (n_hidden, n_hidden)),
            ("b2", (n_hidden,)), ("W3", (n_out, n_hidden)), ("b3", (n_out,))]


def n_params(n_in, n_hidden, n_out) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(n_in, n_hidden, n_out))


def unpack(theta, n_in, n_hidden, n_out) -> Dict[str, np.ndarray]:
    out, k = {}, 0
    for name, s in shapes(n_in, n_hidden, n_out):
        n = int(np.prod(s))
        out[name] = np.asarray(theta[k:k + n], np.float64).reshape(s)
        k += n
    return out


def forward(theta, X, n_in, n_hidden, n_out):
    P = unpack(theta, n_in, n_hidden, n_out)
    X = np.asarray(X, np.float64)
    Z1 = X @ P["W1"].T + P["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ P["W2"].T + P["b2"]
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ P["W3"].T + P["b3"]
    return Y, (X, Z1, H1, Z2, H2)


def loss(theta, X, T, mask, n_in, n_hidden, n_out) -> float:
    Y, _ = forward(theta, X, n_in, n_hidden, n_out)
    m = np.asarray(mask, np.float64)
    return float(np.sum(m * (Y - np.asarray(T, np.float64)) ** 2) / np.sum(m))


def loss_grad(theta, X, T, mask, n_in, n_hidden, n_out) -> Tuple[float, np.ndarray]:
    """Loss and its gradient by backpropagation (chain rule layer by layer)."""
    P = unpack(theta, n_in, n_hidden, n_out)
    Y, (X, Z1, H1, Z2, H2) = forward(theta, X, n_in, n_hidden, n_out)
    m = np.asarray(mask, np.float64)
    cnt = np.sum(m)
    R = Y - np.asarray(T, np.float64)
    L = float(np.sum(m * R ** 2) / cnt)
    dY = 2.0 * m * R / cnt
    g = {}
    g["W3"] = dY.T @ H2
    g["b3"] = dY.sum(axis=0)
    dH2 = dY @ P["W3"]
    dZ2 = dH2 * (Z2 > 0)
    g["W2"] = dZ2.T @ H1
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ P["W2"]
    dZ1 = dH1 * (Z1 > 0)
    g["W1"] = dZ1.T @ X
    g["b1"] = dZ1.sum(axis=0)
    flat = np.concatenate([g[name].ravel() for name, _ in shapes(n_in, n_hidden, n_out)])
    return L, flat


def finite_difference_grad(theta, X, T, mask, n_in, n_hidden, n_out, idx, h=1e-6):
    """Central differences of the loss for the parameters listed in idx."""
    theta = np.asarray(theta, np.float64)
    out = []
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        out.append((loss(tp, X, T, mask, n_in, n_hidden, n_out) -
                    loss(tm, X, T, mask, n_in, n_hidden, n_out)) / (2 * h))
    return np.array(out)


def adam(theta, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba), bias-corrected; returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
