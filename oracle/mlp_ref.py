"""Plain float64 reference of the cost-model MLP (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests compare the library's CUDA forward and
backward kernels against these functions.  Network: x -> relu(W1 x + b1)
-> relu(W2 h1 + b2) -> w3 . h2 + b3; loss = mean over samples of
0.5 (y - t)^2.  Parameters are one flat vector in the order
W1 [H x n_in], b1 [H], W2 [H x H], b2 [H], w3 [H], b3 [1].

Pinned by central finite differences of loss() (tests/test_oracle_mlp.py);
gradient() is written out by the chain rule, independently of those."""
from __future__ import annotations

import numpy as np


def n_params(n_in: int, H: int) -> int:
    return H * n_in + H + H * H + H + H + 1


def unpack(p, n_in, H):
    p = np.asarray(p, np.float64)
    o = 0
    W1 = p[o:o + H * n_in].reshape(H, n_in); o += H * n_in
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, x, n_in, H):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, H)
    x = np.asarray(x, np.float64)
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    return h2 @ w3 + b3, (z1, h1, z2, h2)


def loss(p, x, t, n_in, H):
    y, _ = forward(p, x, n_in, H)
    return float(np.mean(0.5 * (y - np.asarray(t, np.float64)) ** 2))


def gradient(p, x, t, n_in, H):
    """Gradient of loss() by the chain rule."""
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, H)
    x = np.asarray(x, np.float64)
    y, (z1, h1, z2, h2) = forward(p, x, n_in, H)
    N = x.shape[0]
    dy = (y - np.asarray(t, np.float64)) / N          # d loss / d y
    gw3 = dy @ h2
    gb3 = dy.sum()
    d2 = np.outer(dy, w3) * (z2 > 0)                 # d loss / d z2
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (z1 > 0)                        # d loss / d z1
    gW1 = d1.T @ x
    gb1 = d1.sum(0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])


def init_params(n_in, H, seed):
    """He-normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((H, n_in)) * np.sqrt(2.0 / n_in)
    W2 = rng.standard_normal((H, H)) * np.sqrt(2.0 / H)
    w3 = rng.standard_normal(H) * np.sqrt(1.0 / H)
    return np.concatenate([W1.ravel(), np.zeros(H), W2.ravel(), np.zeros(H), w3, [0.0]])
