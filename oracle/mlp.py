"""Plain FP64 CPU multilayer perceptron: the oracle of the learned block preconditioner's network.

TEST INFRASTRUCTURE ONLY.  Three affine layers with ReLU between them,
    h1 = relu(x W1^T + b1),  h2 = relu(h1 W2^T + b2),  y = h2 W3^T + b3,
mean-squared-error loss L = sum((y - t)^2) / (2 n), and the exact backward pass (chain rule).
Weights are stored out x in (row-major), like the device kernels' float32 master copies.
"""
from __future__ import annotations

import numpy as np


def forward(params, x):
    W1, b1, W2, b2, W3, b3 = params
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3.T + b3
    return y, (x, z1, h1, z2, h2)


def loss(params, x, t):
    y, _ = forward(params, x)
    return float(np.sum((y - t) ** 2) / (2.0 * x.shape[0]))


def grad(params, x, t):
    """Gradients of loss() w.r.t. (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    y, (x, z1, h1, z2, h2) = forward(params, x)
    n = x.shape[0]
    dy = (y - t) / n
    dW3 = dy.T @ h2
    db3 = dy.sum(0)
    dh2 = dy @ W3
    dz2 = dh2 * (z2 > 0)
    dW2 = dz2.T @ h1
    db2 = dz2.sum(0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    dW1 = dz1.T @ x
    db1 = dz1.sum(0)
    return [dW1, db1, dW2, db2, dW3, db3]
