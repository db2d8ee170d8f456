"""ORACLE -- test infrastructure only.  Plain FP64 numpy reference of the
learned tuner's multilayer perceptron (in_dim -> hidden -> hidden -> 1, ReLU,
mean squared error, Adam), used to check the GPU training kernels.

Parameter layout (flat, row-major weights W[out][in]):
    W1[H][D] | b1[H] | W2[H][H] | b2[H] | W3[H] | b3

Parity status: forward pinned by a hand-computed example; gradients pinned by
central finite differences of the loss; Adam pinned by its first-step closed
form (update = lr * g / (|g| + eps) from zero moments).
"""
from __future__ import annotations

import numpy as np


def param_count(D: int, H: int) -> int:
    return H * D + H + H * H + H + H + 1


def unpack(p: np.ndarray, D: int, H: int):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    W1 = p[i:i + H * D].reshape(H, D); i += H * D
    b1 = p[i:i + H]; i += H
    W2 = p[i:i + H * H].reshape(H, H); i += H * H
    b2 = p[i:i + H]; i += H
    W3 = p[i:i + H]; i += H
    b3 = p[i]
    return W1, b1, W2, b2, W3, b3


def forward(p, X, D, H):
    """Y, H1, H2 for inputs X[N][D]."""
    W1, b1, W2, b2, W3, b3 = unpack(p, D, H)
    X = np.asarray(X, dtype=np.float64)
    H1 = np.maximum(X @ W1.T + b1, 0.0)
    H2 = np.maximum(H1 @ W2.T + b2, 0.0)
    Y = H2 @ W3 + b3
    return Y, H1, H2


def loss(p, X, T, D, H) -> float:
    Y, _, _ = forward(p, X, D, H)
    return float(np.mean((Y - np.asarray(T, dtype=np.float64)) ** 2))


def backward(p, X, T, D, H) -> np.ndarray:
    """Gradient of the mean squared error by the chain rule, written out."""
    W1, b1, W2, b2, W3, b3 = unpack(p, D, H)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    N = X.shape[0]
    Y, H1, H2 = forward(p, X, D, H)
    dY = 2.0 * (Y - T) / N                       # dL/dY
    dW3 = H2.T @ dY
    db3 = dY.sum()
    d2 = np.outer(dY, W3) * (H2 > 0)             # dL/d(pre-activation 2)
    dW2 = d2.T @ H1
    db2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (H1 > 0)                    # dL/d(pre-activation 1)
    dW1 = d1.T @ X
    db1 = d1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3, [db3]])


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step; returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
