"""The learned preconditioner's network in FP64 (oracle; test infrastructure only).

Architecture 4 -> H (tanh) -> H (tanh) -> 1 with the parameter layout of the library:
W1[H][4], b1[H], W2[H][H], b2[H], w3[H], b3.  Loss of a batch (X, w, T):

    L = 1/(2B) sum_b (w_b y_b - T_b)^2,   y = MLP(X).

The gradient is backpropagation written out layer by layer (chain rule), independent
of the CUDA kernels; a pin compares it with central finite differences.
"""
from __future__ import annotations

import numpy as np


def n_params(H: int) -> int:
    return 4 * H + H + H * H + H + H + 1


def unpack(p, H):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + 4 * H].reshape(H, 4); o += 4 * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, H, X):
    W1, b1, W2, b2, w3, b3 = unpack(p, H)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3, (h1, h2)


def loss(p, H, X, w, T):
    y, _ = forward(p, H, X)
    e = w * y - T
    return 0.5 * np.mean(e * e)


def grad(p, H, X, w, T):
    W1, b1, W2, b2, w3, b3 = unpack(p, H)
    B = X.shape[0]
    y, (h1, h2) = forward(p, H, X)
    dy = (w * y - T) * w / B                  # dL/dy
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dz2 = np.outer(dy, w3) * (1.0 - h2 * h2)   # through tanh of layer 2
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)         # through W2 and tanh of layer 1
    g_W1 = dz1.T @ X
    g_b1 = dz1.sum(axis=0)
    return np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])


def features(D, theta, sD, x2, x3):
    """Inputs of one component (see the library header): d, 1/d (clamped), sector terms."""
    d = (np.asarray(D, dtype=np.float64) - theta) / sD
    x0 = np.clip(d, -8.0, 8.0)
    with np.errstate(divide="ignore"):
        inv = np.where(d != 0.0, 1.0 / np.where(d != 0.0, d, 1.0), 16.0)
    x1 = np.clip(inv, -16.0, 16.0) / 16.0
    return np.stack([x0, x1, np.full_like(d, x2), np.full_like(d, x3)], axis=1)
