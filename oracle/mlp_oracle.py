"""Plain FP64 CPU reference of the tuner's cost-model MLP: forward pass, mean-squared loss,
back-propagation and one Adam update.

TEST INFRASTRUCTURE ONLY: the CUDA training and inference kernels of the cost model are
checked against this module (gradients, forward values, Adam steps).  It shares no code with
them.  Each function is the textbook definition written out with numpy, no fusion.

Network (the same layout the CUDA kernels use): input x (d features) ->
    h1 = tanh(W1 x + b1)      W1: (H, d)
    h2 = tanh(W2 h1 + b2)     W2: (H, H)
    y  = W3 h2 + b3           W3: (1, H)
Parameters are one flat vector: W1 (row-major), b1, W2, b2, W3, b3.
Loss over n samples: L = (1/n) sum_s (y_s - t_s)^2.
Adam (Kingma & Ba): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
    p -= lr * (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps), k = step number (from 1).
"""
from __future__ import annotations

import numpy as np


def param_count(d: int, hidden: int) -> int:
    return hidden * d + hidden + hidden * hidden + hidden + hidden + 1


def unpack(p: np.ndarray, d: int, hidden: int):
    H = hidden
    o = 0
    W1 = p[o:o + H * d].reshape(H, d); o += H * d
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H].reshape(1, H); o += H
    b3 = p[o:o + 1]; o += 1
    return W1, b1, W2, b2, W3, b3


def forward(p, X, d: int, hidden: int):
    """Returns (y, h1, h2) for inputs X of shape (n, d)."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(p, dtype=np.float64), d, hidden)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = (h2 @ W3.T + b3)[:, 0]
    return y, h1, h2


def loss(p, X, t, d: int, hidden: int) -> float:
    y, _, _ = forward(p, X, d, hidden)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradient(p, X, t, d: int, hidden: int) -> np.ndarray:
    """dL/dp by the chain rule, in the flat parameter layout."""
    p = np.asarray(p, dtype=np.float64)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    W1, b1, W2, b2, W3, b3 = unpack(p, d, hidden)
    y, h1, h2 = forward(p, X, d, hidden)
    dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / n          # (n,)
    gW3 = dy[None, :] @ h2                                         # (1, H)
    gb3 = np.array([dy.sum()])
    dh2 = dy[:, None] * W3                                         # (n, H)
    dz2 = dh2 * (1.0 - h2 ** 2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (1.0 - h1 ** 2)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def adam_step(p, g, m, v, k: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update; returns (p, m, v) new arrays."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** k)
    vhat = v / (1.0 - beta2 ** k)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
