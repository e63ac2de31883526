"""The cost model's CUDA kernels against the FP64 CPU MLP oracle: forward values, the
back-propagated gradient, Adam steps, and training that lowers the loss."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _model(d, H, seed):
    from paper_1204_4779_gb300 import costmodel
    net = costmodel.MLP(d, H, seed=seed)
    rng = np.random.default_rng(seed + 100)
    p = rng.normal(0, 0.4, net.n_params).astype(np.float32)
    net.set_params(p)
    return net, p.astype(np.float64)


@pytest.mark.parametrize("d,H,n", [(7, 5, 11), (31, 64, 2000), (3, 64, 1)])
def test_forward_and_gradient_match_oracle(d, H, n):
    net, p = _model(d, H, d)
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (n, d)).astype(np.float32)
    t = rng.normal(0, 1, n).astype(np.float32)
    y = net.predict(X)
    yo, _, _ = M.forward(p, X.astype(np.float64), d, H)
    assert np.max(np.abs(y - yo)) <= 1e-5 * max(1.0, np.max(np.abs(yo)))
    g, loss = net.gradient(X, t)
    go = M.gradient(p, X.astype(np.float64), t.astype(np.float64), d, H)
    lo = M.loss(p, X.astype(np.float64), t.astype(np.float64), d, H)
    assert abs(loss - lo) <= 1e-5 * max(1.0, lo)
    assert np.max(np.abs(g - go)) <= 1e-4 * max(1e-3, np.max(np.abs(go)))


def test_adam_matches_oracle():
    d, H = 9, 16
    net, p = _model(d, H, 3)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (50, d)).astype(np.float32)
    t = rng.normal(0, 1, 50).astype(np.float32)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for k in range(1, 6):
        g = M.gradient(p, X.astype(np.float64), t.astype(np.float64), d, H)
        p, m, v = M.adam_step(p, g, m, v, k, lr=1e-2)
        gg, _ = net.gradient(X, t)
        net.adam(gg, lr=1e-2)
    assert np.max(np.abs(net.get_params() - p)) <= 1e-4


def test_training_reduces_loss_deterministically():
    d, H = 12, 64
    rng = np.random.default_rng(4)
    X = rng.normal(0, 1, (500, d)).astype(np.float32)
    t = (np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2]).astype(np.float32)
    a, _ = _model(d, H, 5)
    b, _ = _model(d, H, 5)
    la = a.train(X, t, 300, lr=3e-3)
    lb = b.train(X, t, 300, lr=3e-3)
    assert la[-1] < 0.2 * la[0]
    assert np.array_equal(la, lb) and np.array_equal(a.get_params(), b.get_params())


def test_training_equals_gradient_and_adam_steps():
    """hydro_mlp_train (epochs replayed from a captured graph, the step number kept on the
    device) computes the same updates as the same number of gradient + Adam calls, and its loss
    history is the loss before each step."""
    d, H = 10, 64
    rng = np.random.default_rng(6)
    X = rng.normal(0, 1, (300, d)).astype(np.float32)
    t = rng.normal(0, 1, 300).astype(np.float32)
    a, _ = _model(d, H, 7)
    b, _ = _model(d, H, 7)
    epochs = 37  # two replays of 16 captured epochs and five direct ones
    hist = a.train(X, t, epochs, lr=3e-3)
    losses = []
    for _ in range(epochs):
        g, loss = b.gradient(X, t)
        losses.append(loss)
        b.adam(g, lr=3e-3)
    pa, pb = a.get_params(), b.get_params()
    assert np.max(np.abs(pa - pb)) <= 1e-5 * max(1.0, np.max(np.abs(pb)))
    assert np.allclose(hist, losses, rtol=1e-5, atol=1e-7)
