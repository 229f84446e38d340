"""Pins of the FP64 reference network used to check the GPU training kernels:
the analytic gradient against central differences of the loss (a dropped
tanh' factor, a transposed weight or a wrong bias gradient would fail), the
forward pass against a direct evaluation, the expectile weighting against
the defining equation of a sample expectile (a swapped tau / 1 - tau fails),
and Adam against its textbook first step (|update| = lr for every coordinate
with a nonzero gradient)."""
import numpy as np
import pytest

from oracle import mlp


@pytest.mark.parametrize("tau", [0.5, 0.9])
def test_gradient_central_differences(tau):
    rng = np.random.default_rng(3)
    F = 7
    th = mlp.init(F, seed=1)
    X = rng.normal(size=(13, F))
    t = rng.normal(size=13)
    L, g = mlp.loss_and_grad(th, X, t, tau)
    idx = rng.choice(len(th), size=60, replace=False)
    for i in idx:
        h = 1e-6
        e = np.zeros_like(th)
        e[i] = h
        Lp, _ = mlp.loss_and_grad(th + e, X, t, tau)
        Lm, _ = mlp.loss_and_grad(th - e, X, t, tau)
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


def test_expectile_weighting():
    """A network that outputs a constant b4 (every weight zero) minimises the
    expectile loss at the sample's tau-expectile: the b4 gradient vanishes
    there and has the right sign on either side.  tau = 1/2 gives the mean;
    tau near 1 approaches the maximum."""
    rng = np.random.default_rng(5)
    F = 3
    t = rng.normal(size=41) ** 3
    X = rng.normal(size=(41, F))
    nb = mlp.n_params(F)
    assert abs(mlp.expectile(t, 0.5) - t.mean()) < 1e-12
    e99 = mlp.expectile(t, 0.99)
    assert t.mean() < e99 < t.max()
    for tau in (0.5, 0.8, 0.99):
        e = mlp.expectile(t, tau)
        for db, sign in ((0.0, 0), (0.05, 1), (-0.05, -1)):
            th = np.zeros(nb)
            th[-1] = e + db
            L, g = mlp.loss_and_grad(th, X, t, tau)
            if sign == 0:
                assert abs(g[-1]) < 1e-10
            else:
                assert np.sign(g[-1]) == sign
            # direct evaluation of the loss at the constant prediction
            r = th[-1] - t
            w = np.where(r < 0, 2 * tau, 2 * (1 - tau))
            assert abs(L - np.mean(w * r * r)) < 1e-12
