"""Pins of the FP64 numpy backprop of the proposal network (no GPU): its gradient
equals central finite differences of its loss, and its forward pass equals the
layer-by-layer definition evaluated by hand for one sample."""

import numpy as np

from oracle import mlp


def _problem(seed=0, n=37):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(mlp.N_PARAMS) * 0.3
    x = rng.standard_normal((n, 6))
    t = rng.standard_normal(n)
    return p, x, t


def test_gradient_matches_central_differences():
    p, x, t = _problem()
    _, g = mlp.loss_grad(p, x, t)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False), [0, 383, 384, 447, 448, 4543, 4544,
                                                                         4607, 4608, 4671, 4672]])
    eps = 1e-6
    for i in idx:
        dp = np.zeros_like(p)
        dp[i] = eps
        fd = (mlp.loss(p + dp, x, t) - mlp.loss(p - dp, x, t)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_by_hand():
    p, x, _ = _problem(n=1)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p)
    h1 = [0.0] * 64
    for j in range(64):
        z = b1[j] + sum(W1[j, i] * x[0, i] for i in range(6))
        h1[j] = z / (1 + np.exp(-z))
    y = b3
    for k in range(64):
        z = b2[k] + sum(W2[k, j] * h1[j] for j in range(64))
        y += w3[k] * z / (1 + np.exp(-z))
    assert abs(mlp.forward(p, x)[0] - y) <= 1e-12 * max(1.0, abs(y))
