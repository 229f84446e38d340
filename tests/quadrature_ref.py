"""Brute-force quadrature for Cartesian Gaussian integrals (test helper).

Independent of the oracle's McMurchie-Davidson code: the kernels are written
through the integral representations
    1/r          = (2/sqrt(pi)) int_0^inf   e^{-t^2 r^2} dt
    erf(w r)/r   = (2/sqrt(pi)) int_0^w     e^{-t^2 r^2} dt
    erfc(w r)/r  = (2/sqrt(pi)) int_w^inf   e^{-t^2 r^2} dt
so that, for fixed t, the six-dimensional integral splits into x, y and z
factors.  In each factor the aux-side coordinate is integrated in closed form
(a Gaussian moment after completing the square) and the AO-side coordinate by
the trapezoid rule on a fine uniform grid (spectrally accurate for Gaussians);
t is integrated by Gauss-Legendre.  Unnormalised primitives, the same
Cartesian component order as the libraries (lexicographic, x^l first).
"""
import math

import numpy as np


def cart(l):
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def _moment(k, s):
    # int y^k e^{-s y^2} dy
    if k % 2:
        return np.zeros_like(s)
    return math.gamma((k + 1) / 2.0) / s ** ((k + 1) / 2.0)


def _factor(t, g, C, a, A, b, B, lc, la, lb, h=0.02):
    """F[nt, c, i, j] = int int (x1-C)^c e^{-g(x1-C)^2} e^{-t^2 (x1-x2)^2}
    (x2-A)^i (x2-B)^j e^{-a(x2-A)^2 - b(x2-B)^2} dx1 dx2"""
    p = a + b
    P = (a * A + b * B) / p
    width = math.sqrt(50.0 / p)
    x = np.arange(P - width - 1.0, P + width + 1.0 + h, h)
    t2 = (t * t)[:, None]
    s = g + t2
    kap = g * t2 / s
    delta = (g * C + t2 * x[None, :]) / s - C          # m - C
    gaussx = np.exp(-kap * (C - x[None, :]) ** 2)
    inner = []
    for c in range(lc + 1):
        acc = np.zeros((len(t), len(x)))
        for k in range(c + 1):
            acc = acc + math.comb(c, k) * delta ** (c - k) * _moment(k, s)
        inner.append(acc * gaussx)
    w = np.exp(-a * (x - A) ** 2 - b * (x - B) ** 2)
    F = np.zeros((len(t), lc + 1, la + 1, lb + 1))
    for c in range(lc + 1):
        for i in range(la + 1):
            for j in range(lb + 1):
                F[:, c, i, j] = h * np.sum(inner[c] * ((x - A) ** i * (x - B) ** j * w)[None, :], axis=1)
    return F


def _t_nodes(kernel, omega, n=160):
    xg, wg = np.polynomial.legendre.leggauss(n)
    def interval(lo, hi):
        return 0.5 * (hi - lo) * xg + 0.5 * (hi + lo), 0.5 * (hi - lo) * wg
    def tail(t0):
        # t = t0/u, u in (0, 1]
        u, wu = interval(0.0, 1.0)
        return t0 / u, wu * t0 / u ** 2
    if kernel == 1:
        return interval(0.0, omega)
    if kernel == 2:
        t1, w1 = interval(omega, omega + 2.0)
        t2, w2 = tail(omega + 2.0)
        return np.concatenate([t1, t2]), np.concatenate([w1, w2])
    t1, w1 = interval(0.0, 2.0)
    t2, w2 = tail(2.0)
    return np.concatenate([t1, t2]), np.concatenate([w1, w2])


def int3c(kernel, omega, lc, g, C, la, a, A, lb, b, B):
    C, A, B = (np.asarray(v, dtype=float) for v in (C, A, B))
    t, wt = _t_nodes(kernel, omega)
    F = [_factor(t, g, C[d], a, A[d], b, B[d], lc, la, lb) for d in range(3)]
    cc, ca, cb = cart(lc), cart(la), cart(lb)
    out = np.zeros((len(cc), len(ca), len(cb)))
    for ic, c in enumerate(cc):
        for ia, ai in enumerate(ca):
            for ib, bj in enumerate(cb):
                prod = F[0][:, c[0], ai[0], bj[0]] * F[1][:, c[1], ai[1], bj[1]] * F[2][:, c[2], ai[2], bj[2]]
                out[ic, ia, ib] = 2.0 / math.sqrt(math.pi) * np.sum(wt * prod)
    return out


def ovlp(la, a, A, lb, b, B, h=0.01):
    A, B = np.asarray(A, float), np.asarray(B, float)
    out = np.zeros((len(cart(la)), len(cart(lb))))
    p = a + b
    for ia, ai in enumerate(cart(la)):
        for ib, bj in enumerate(cart(lb)):
            v = 1.0
            for d in range(3):
                P = (a * A[d] + b * B[d]) / p
                wd = math.sqrt(60.0 / p)
                x = np.arange(P - wd, P + wd + h, h)
                v *= h * np.sum((x - A[d]) ** ai[d] * (x - B[d]) ** bj[d] * np.exp(-a * (x - A[d]) ** 2 - b * (x - B[d]) ** 2))
            out[ia, ib] = v
    return out


def ft(la, a, A, lb, b, B, q, h=0.005):
    A, B, q = np.asarray(A, float), np.asarray(B, float), np.asarray(q, float)
    out = np.zeros((len(cart(la)), len(cart(lb))), dtype=complex)
    p = a + b
    for ia, ai in enumerate(cart(la)):
        for ib, bj in enumerate(cart(lb)):
            v = 1.0 + 0j
            for d in range(3):
                P = (a * A[d] + b * B[d]) / p
                wd = math.sqrt(60.0 / p)
                x = np.arange(P - wd, P + wd + h, h)
                f = (x - A[d]) ** ai[d] * (x - B[d]) ** bj[d] * np.exp(-a * (x - A[d]) ** 2 - b * (x - B[d]) ** 2)
                v *= h * np.sum(f * np.exp(-1j * q[d] * x))
            out[ia, ib] = v
    return out
