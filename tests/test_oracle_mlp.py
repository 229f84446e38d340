"""Pins of the FP64 reference network used to check the GPU training kernels:
the analytic gradient against central differences of the loss (a dropped
tanh' factor, a transposed weight or a wrong bias gradient would fail), the
forward pass against a direct evaluation, and Adam against its textbook
first step (|update| = lr for every coordinate with a nonzero gradient)."""
import numpy as np

from oracle import mlp


def test_gradient_central_differences():
    rng = np.random.default_rng(3)
    F = 7
    th = mlp.init(F, seed=1)
    X = rng.normal(size=(13, F))
    t = rng.normal(size=13)
    L, g = mlp.loss_and_grad(th, X, t)
    idx = rng.choice(len(th), size=60, replace=False)
    for i in idx:
        h = 1e-6
        e = np.zeros_like(th)
        e[i] = h
        Lp, _ = mlp.loss_and_grad(th + e, X, t)
        Lm, _ = mlp.loss_and_grad(th - e, X, t)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(fd)), (i, fd, g[i])


def test_forward_direct():
    rng = np.random.default_rng(4)
    F = 5
    th = mlp.init(F, seed=2)
    x = rng.normal(size=F)
    W1, b1, W2, b2, W3, b3, w4, b4 = mlp.unpack(th, F)
    h = np.tanh(W1 @ x + b1)
    h = np.tanh(W2 @ h + b2)
    h = np.tanh(W3 @ h + b3)
    y = float(w4 @ h + b4[0])
    assert abs(mlp.forward(th, x[None, :])[0][0] - y) < 1e-14
    assert len(th) == mlp.n_params(F)


def test_adam_first_step():
    th = np.zeros(6)
    g = np.array([1.0, -2.0, 0.5, 0.0, 3.0, -1e-3])
    m = np.zeros(6)
    v = np.zeros(6)
    mlp.adam_step(th, g, m, v, 1, lr=0.01, eps=1e-30)
    nz = g != 0
    assert np.allclose(np.abs(th[nz]), 0.01)
    assert np.all(np.sign(th[nz]) == -np.sign(g[nz]))
    assert th[3] == 0.0
