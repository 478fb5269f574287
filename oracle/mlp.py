"""Plain FP64 numpy forward and backward pass of the jump-time proposal network.

TEST INFRASTRUCTURE ONLY: the checker of the library's MLP training kernels
(imported by the tests alone).  Network: 6 -> 64 -> 64 -> 1 with SiLU(z) =
z / (1 + exp(-z)); loss = mean over samples of (y - t)^2.  Parameter layout
(a flat vector): W1[64][6], b1[64], W2[64][64], b2[64], w3[64], b3.  The
backward pass is the chain rule written out layer by layer; its correctness is
pinned by central finite differences of the loss in the tests.
"""

import numpy as np

H, D = 64, 6
N_PARAMS = H * D + H + H * H + H + H + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * D].reshape(H, D); o += H * D
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, x):
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    return h2 @ w3 + b3


def loss(p, x, t):
    e = forward(p, x) - np.asarray(t, dtype=np.float64)
    return float(np.mean(e * e))


def loss_grad(p, x, t):
    """Returns (loss, gradient) in FP64."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = len(t)
    z1 = x @ W1.T + b1
    h1 = silu(z1)
    z2 = h1 @ W2.T + b2
    h2 = silu(z2)
    y = h2 @ w3 + b3
    e = y - t
    dy = 2.0 * e / n
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    d2 = np.outer(dy, w3) * silu_grad(z2)
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * silu_grad(z1)
    g_W1 = d1.T @ x
    g_b1 = d1.sum(axis=0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return float(np.mean(e * e)), g
