"""Plant plausible mistakes in a copy of the MLP oracle's source and check that its pins
(central finite differences of the loss, the hand-expanded forward pass, Adam's step magnitude
with a constant gradient) catch every one of them.  Each mutated copy runs as a module of its
own; the oracle under test is never modified."""
import math
import os
import types

import numpy as np
import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "mlp_oracle.py")

MUTANTS = [
    ("tanh_derivative", "dz2 = dh2 * (1.0 - h2 ** 2)", "dz2 = dh2 * (1.0 - h2)"),
    ("loss_factor_two", "dy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / n",
     "dy = (y - np.asarray(t, dtype=np.float64)) / n"),
    ("bias_gradient_before_activation", "gb2 = dz2.sum(axis=0)", "gb2 = dh2.sum(axis=0)"),
    ("transposed_weight", "dh1 = dz2 @ W2", "dh1 = dz2 @ W2.T"),
    ("adam_v_bias_correction", "vhat = v / (1.0 - beta2 ** k)", "vhat = v / (1.0 - beta2)"),
    ("forward_bias_dropped", "h1 = np.tanh(X @ W1.T + b1)", "h1 = np.tanh(X @ W1.T)"),
    ("output_weight_gradient_layer", "gW3 = dy[None, :] @ h2", "gW3 = dy[None, :] @ h1"),
]


def _module(src: str):
    m = types.ModuleType("mlp_oracle_mutant")
    exec(compile(src, "mlp_oracle_mutant", "exec"), m.__dict__)
    return m


def _pins(M) -> list:
    fails = []
    rng = np.random.default_rng(3)
    d, H, n = 4, 3, 6
    p = rng.normal(0, 0.5, M.param_count(d, H))
    X = rng.normal(0, 1, (n, d))
    t = rng.normal(0, 1, n)
    g = M.gradient(p, X, t, d, H)
    fd = np.empty_like(p)
    for i in range(p.size):
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd[i] = (M.loss(p + e, X, t, d, H) - M.loss(p - e, X, t, d, H)) / 2e-6
    if not np.max(np.abs(g - fd)) <= 1e-7 * max(1.0, np.max(np.abs(fd))):
        fails.append("finite_differences")
    # forward pass of a tiny network evaluated by hand
    W1 = np.array([[0.5, -1.0], [0.25, 2.0]])
    b1 = np.array([0.1, -0.2])
    W2 = np.array([[1.0, 0.5], [-0.5, 1.5]])
    b2 = np.array([0.0, 0.3])
    W3 = np.array([[2.0, -1.0]])
    b3 = np.array([0.7])
    q = np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])
    a1 = math.tanh(0.5 * 0.3 - 1.0 * -0.4 + 0.1)
    a2 = math.tanh(0.25 * 0.3 + 2.0 * -0.4 - 0.2)
    c1 = math.tanh(1.0 * a1 + 0.5 * a2 + 0.0)
    c2 = math.tanh(-0.5 * a1 + 1.5 * a2 + 0.3)
    y, _, _ = M.forward(q, np.array([[0.3, -0.4]]), 2, 2)
    if not abs(y[0] - (2.0 * c1 - 1.0 * c2 + 0.7)) < 1e-14:
        fails.append("forward")
    # Adam: every step with a constant gradient moves each coordinate by lr
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for k in range(1, 4):
        p2, m, v = M.adam_step(p, g, m, v, k, lr=1e-2, eps=0.0)
        if not np.allclose(np.abs(p2 - p)[g != 0], 1e-2, rtol=1e-10):
            fails.append(f"adam_{k}")
            break
        p = p2
    return fails


def test_unmutated_mlp_oracle_passes_the_battery():
    assert _pins(_module(open(SRC).read())) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    assert _pins(_module(src.replace(old, new))), f"mutant {name} survived every pin"
