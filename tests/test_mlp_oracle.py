"""Pins of the FP64 MLP oracle: back-propagation against central finite differences of the
loss, the forward pass against a hand-expanded tiny network, and Adam's first step (whose
magnitude is lr in every coordinate with a non-zero gradient)."""
import math

import numpy as np

from oracle import mlp_oracle as M


def _case(seed, d=7, H=5, n=11):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.5, M.param_count(d, H))
    X = rng.normal(0, 1, (n, d))
    t = rng.normal(0, 1, n)
    return p, X, t, d, H


def test_gradient_matches_finite_differences():
    for seed in range(3):
        p, X, t, d, H = _case(seed)
        g = M.gradient(p, X, t, d, H)
        fd = np.empty_like(p)
        h = 1e-6
        for i in range(p.size):
            e = np.zeros_like(p)
            e[i] = h
            fd[i] = (M.loss(p + e, X, t, d, H) - M.loss(p - e, X, t, d, H)) / (2 * h)
        assert np.max(np.abs(g - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd)))


def test_forward_hand_expanded_tiny_network():
    d, H = 2, 2
    W1 = np.array([[0.5, -1.0], [0.25, 2.0]])
    b1 = np.array([0.1, -0.2])
    W2 = np.array([[1.0, 0.5], [-0.5, 1.5]])
    b2 = np.array([0.0, 0.3])
    W3 = np.array([[2.0, -1.0]])
    b3 = np.array([0.7])
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    x = np.array([0.3, -0.4])
    a1 = math.tanh(0.5 * 0.3 - 1.0 * -0.4 + 0.1)
    a2 = math.tanh(0.25 * 0.3 + 2.0 * -0.4 - 0.2)
    c1 = math.tanh(1.0 * a1 + 0.5 * a2 + 0.0)
    c2 = math.tanh(-0.5 * a1 + 1.5 * a2 + 0.3)
    want = 2.0 * c1 - 1.0 * c2 + 0.7
    y, _, _ = M.forward(p, x[None, :], d, H)
    assert abs(y[0] - want) < 1e-14


def test_adam_first_step_has_magnitude_lr():
    p, X, t, d, H = _case(5)
    g = M.gradient(p, X, t, d, H)
    p2, m, v = M.adam_step(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr=1e-2, eps=0.0)
    step = np.abs(p2 - p)
    assert np.allclose(step[g != 0], 1e-2, rtol=1e-12)


def test_training_reduces_loss():
    p, X, t, d, H = _case(6, n=40)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = M.loss(p, X, t, d, H)
    for k in range(1, 301):
        p, m, v = M.adam_step(p, M.gradient(p, X, t, d, H), m, v, k, lr=1e-2)
    assert M.loss(p, X, t, d, H) < 0.2 * L0


def test_adam_steps_with_a_constant_gradient_have_magnitude_lr():
    """With the same gradient every step the bias-corrected moments are exactly g and g^2, so
    every step (not only the first) moves each coordinate by lr (eps = 0)."""
    p, X, t, d, H = _case(7)
    g = M.gradient(p, X, t, d, H)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for k in range(1, 4):
        p2, m, v = M.adam_step(p, g, m, v, k, lr=1e-2, eps=0.0)
        assert np.allclose(np.abs(p2 - p)[g != 0], 1e-2, rtol=1e-10), k
        p = p2
