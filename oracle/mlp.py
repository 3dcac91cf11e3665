"""Plain FP64 CPU reference of the (n, P) selector network: 6 -> H -> H -> 2 with ReLU,
mean squared error, packed parameters W1 (H x 6), b1, W2 (H x H), b2, W3 (2 x H), b3.

TEST INFRASTRUCTURE ONLY: the gradient of the device kernels is checked against this, and this
is checked against central finite differences.  The network is not part of the paper (the
paper chooses N_i with chebfun2); it stands in for that choice.
"""
from __future__ import annotations

import numpy as np


def unpack(theta: np.ndarray, H: int):
    o = 0
    W1 = theta[o:o + 6 * H].reshape(H, 6); o += 6 * H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + 2 * H].reshape(2, H); o += 2 * H
    b3 = theta[o:o + 2]; o += 2
    assert o == theta.size
    return W1, b1, W2, b2, W3, b3


def forward(theta, H, X):
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, np.float64), H)
    X = np.asarray(X, np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    return h2 @ W3.T + b3


def loss_and_grad(theta, H, X, T):
    """L = mean over samples and outputs of (y - t)^2 and dL/dtheta (packed like theta)."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, np.float64), H)
    X = np.asarray(X, np.float64)
    T = np.asarray(T, np.float64)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ W3.T + b3
    n = y.size
    L = float(np.sum((y - T) ** 2) / n)
    dy = 2.0 * (y - T) / n
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = (dy @ W3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g
