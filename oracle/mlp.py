"""Plain FP64 reference of the learned-screening network (test infrastructure).

TEST INFRASTRUCTURE ONLY (tests, smoke check, bench CPU leg).  The network is
the project's own addition to the method (the paper screens with the
Supplementary Material's estimates only): a multilayer perceptron with three
hidden layers of 64 tanh units,

    h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3),
    y  = w4 . h3 + b4,

fitted to log10 of SR work-item magnitudes with the expectile loss
L = (1/n) sum_s w_s (y_s - t_s)^2, w_s = 2 tau where y_s < t_s and 2 (1 - tau)
elsewhere (asymmetric least squares, Newey & Powell 1987; tau = 1/2 is the
mean squared error, tau near 1 fits an upper envelope of the targets).  Parameters are packed in one vector in the
order W1 [64 x F] (row-major), b1 [64], W2 [64 x 64], b2, W3 [64 x 64], b3,
w4 [64], b4 [1] -- the same packing the CUDA kernels use.  The backward pass
is the chain rule written out; tests pin it against central differences.
"""
from __future__ import annotations

import numpy as np

H = 64


def n_params(F: int) -> int:
    return H * F + H + 2 * (H * H + H) + H + 1


def unpack(theta: np.ndarray, F: int):
    o = 0
    out = []
    for shape in ((H, F), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)):
        n = int(np.prod(shape))
        out.append(theta[o:o + n].reshape(shape))
        o += n
    return out


def forward(theta, X):
    F = X.shape[1]
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(np.asarray(theta, np.float64), F)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    h3 = np.tanh(h2 @ W3.T + b3)
    y = h3 @ w4 + b4[0]
    return y, (h1, h2, h3)


def loss_and_grad(theta, X, t, tau=0.5):
    """Expectile loss and its gradient with respect to the packed parameters."""
    X = np.asarray(X, np.float64)
    t = np.asarray(t, np.float64)
    n, F = X.shape
    W1, b1, W2, b2, W3, b3, w4, b4 = unpack(np.asarray(theta, np.float64), F)
    y, (h1, h2, h3) = forward(theta, X)
    r = y - t
    w = np.where(r < 0.0, 2.0 * tau, 2.0 * (1.0 - tau))
    L = float(np.mean(w * r * r))
    dy = 2.0 * w * r / n                  # dL/dy
    gw4 = h3.T @ dy
    gb4 = np.array([dy.sum()])
    d3 = np.outer(dy, w4) * (1.0 - h3 * h3)
    gW3 = d3.T @ h2
    gb3 = d3.sum(0)
    d2 = (d3 @ W3) * (1.0 - h2 * h2)
    gW2 = d2.T @ h1
    gb2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    gW1 = d1.T @ X
    gb1 = d1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3, gw4, gb4])
    return L, g


def expectile(t, tau):
    """The tau-expectile of a sample: the e solving
    tau sum_{t > e} (t - e) = (1 - tau) sum_{t < e} (e - t), by bisection."""
    t = np.asarray(t, np.float64)
    lo, hi = float(t.min()), float(t.max())
    for _ in range(200):
        e = 0.5 * (lo + hi)
        if tau * np.sum(np.maximum(t - e, 0.0)) > (1.0 - tau) * np.sum(np.maximum(e - t, 0.0)):
            lo = e
        else:
            hi = e
    return 0.5 * (lo + hi)


def init(F: int, seed: int = 0) -> np.ndarray:
    """Uniform +-sqrt(1/fan_in) initialisation (the CUDA side receives it from the host)."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, shape in ((F, (H, F)), (F, (H,)), (H, (H, H)), (H, (H,)), (H, (H, H)), (H, (H,)), (H, (H,)), (H, (1,))):
        s = np.sqrt(1.0 / fan_in)
        parts.append(rng.uniform(-s, s, size=shape).ravel())
    return np.concatenate(parts)


def adam_step(theta, g, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), in place on theta, m, v."""
    m *= b1
    m += (1 - b1) * g
    v *= b2
    v += (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    theta -= lr * mh / (np.sqrt(vh) + eps)
    return theta
