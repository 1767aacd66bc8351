"""Pins of the oracle MLP: its gradient against central finite differences of its loss, and the
reduction to a plain linear least-squares gradient when the ReLUs are all active."""
import numpy as np

from oracle import mlp
from paper_2009_00706_gb300 import inputs as I


def _params(nin, w, nout, seed):
    shapes = [(w, nin), (w,), (w, w), (w,), (nout, w), (nout,)]
    out, off = [], 0
    for k, s in enumerate(shapes):
        n = int(np.prod(s))
        out.append(0.3 * I.normal(seed + k, n).reshape(s))
    return out


def test_gradient_matches_central_differences():
    x = I.normal(1, 7 * 9).reshape(7, 9)
    t = I.normal(2, 7 * 5).reshape(7, 5)
    p = _params(9, 6, 5, 10)
    g = mlp.grad(p, x, t)
    rng = np.random.default_rng(0)
    for k in range(6):
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            eps = 1e-6
            pp = [q.copy() for q in p]
            pm = [q.copy() for q in p]
            pp[k][idx] += eps
            pm[k][idx] -= eps
            fd = (mlp.loss(pp, x, t) - mlp.loss(pm, x, t)) / (2 * eps)
            assert abs(fd - g[k][idx]) <= 1e-7 + 1e-6 * abs(fd), (k, idx, fd, g[k][idx])


def test_active_relus_reduce_to_linear_least_squares():
    # all pre-activations positive: y = x A^T + c with A = W3 W2 W1; dL/db3 = mean residual
    x = np.abs(I.normal(3, 4 * 3).reshape(4, 3)) + 1.0
    W1 = np.abs(I.normal(4, 2 * 3).reshape(2, 3)); b1 = np.ones(2)
    W2 = np.abs(I.normal(5, 2 * 2).reshape(2, 2)); b2 = np.ones(2)
    W3 = I.normal(6, 3 * 2).reshape(3, 2); b3 = I.normal(7, 3)
    t = I.normal(8, 4 * 3).reshape(4, 3)
    p = [W1, b1, W2, b2, W3, b3]
    y, _ = mlp.forward(p, x)
    A = W3 @ W2 @ W1
    c = W3 @ (W2 @ b1 + b2) + b3
    assert np.allclose(y, x @ A.T + c, atol=1e-12)
    g = mlp.grad(p, x, t)
    assert np.allclose(g[5], (y - t).mean(0), atol=1e-12)
