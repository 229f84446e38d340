"""The downward recursion of the erfc auxiliary integrals used by the SR kernel
(CPU only, against arbitrary precision).

With H_n = F_n(T) - s^{n+1/2} F_n(sT), the integral of t^{2n} e^{-T t^2} over
[sqrt s, 1], integration by parts gives (2n+1) H_n = 2T H_{n+1} + e^{-T} -
s^{n+1/2} e^{-sT}; for G_n = (-2 alpha)^n H_n and R^2 = T/alpha:

    G_n = (-R^2 G_{n+1} + fw_n e^{-T} - fw_n sw_n e^{-sT}) / (2n+1),
    fw_n = (-2 alpha)^n, sw_n = s^{n+1/2}.

The kernel seeds G_L from F_L(T) and F_L(sT) (table or, above T = 100, the power
law with e^{-T} = 0) and recurs down in FP64.  Claimed: the rounding error of
every G_n stays at the scale eps |fw_n| (F_n(T) + s^{n+1/2} F_n(sT)), because F's
own recursion bounds the factor 2T/(2n+1) by F_n/F_{n+1}.  The reference here is
F_n(x) = gamma(n + 1/2, x) / (2 x^{n+1/2}) at 40 digits."""
import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40
EPS = 2.0 ** -52


def boys_mp(n, x):
    x = mpmath.mpf(x)
    if x == 0:
        return mpmath.mpf(1) / (2 * n + 1)
    return mpmath.gammainc(n + mpmath.mpf(1) / 2, 0, x) / (2 * x ** (n + mpmath.mpf(1) / 2))


def merged_recursion(L, T, s, alpha, sign=-1.0):
    """G_n, n = 0..L, in FP64 from correctly rounded seeds, in the kernel's order."""
    R2 = T / alpha
    sT = s * T
    if T < 100.0:
        FL, eT = float(boys_mp(L, T)), float(mpmath.e ** (-mpmath.mpf(T)))
    else:
        FL, eT = float(boys_mp(L, T)), 0.0
    FsL, esT = float(boys_mp(L, sT)), float(mpmath.e ** (-mpmath.mpf(sT)))
    sw, fw = np.sqrt(s), 1.0
    pa, pb = [], []
    for n in range(L + 1):
        if n < L:
            pa.append(fw * (1.0 / (2 * n + 1)))
            pb.append(-(fw * sw) * (1.0 / (2 * n + 1)))
        else:
            fwL, swL = fw, sw
        sw *= s
        fw *= -2.0 * alpha
    G = [0.0] * (L + 1)
    G[L] = fwL * (FL - swL * FsL)
    for n in range(L - 1, -1, -1):
        b = pa[n] * eT + pb[n] * esT
        G[n] = (sign * R2 * (1.0 / (2 * n + 1))) * G[n + 1] + b
    return G


def reference(L, T, s, alpha):
    out = []
    for n in range(L + 1):
        fw = (-2 * mpmath.mpf(alpha)) ** n
        sw = mpmath.mpf(s) ** (n + mpmath.mpf(1) / 2)
        Fn, Fsn = boys_mp(n, T), boys_mp(n, s * T)
        out.append((fw * (Fn - sw * Fsn), abs(fw) * (Fn + sw * Fsn)))
    return out


def _grid():
    rng = np.random.default_rng(12)
    for L in range(2, 10):
        for T in (1e-3, 0.05, 0.7, 3.0, 11.0, 27.0, 45.0, 80.0, 99.0, 130.0, 300.0):
            s = float(rng.uniform(0.01, 0.99))
            if s * T >= 70.0:      # the kernel skips these terms (they vanish below 1e-30)
                s = 0.5 * 70.0 / T
            yield L, T, s, float(rng.uniform(0.05, 20.0))


def test_merged_recursion_error_at_the_claimed_scale():
    worst = 0.0
    for L, T, s, alpha in _grid():
        G = merged_recursion(L, T, s, alpha)
        for n, (g_ref, scale) in enumerate(reference(L, T, s, alpha)):
            err = abs(G[n] - float(g_ref))
            ratio = err / (EPS * float(scale))
            worst = max(worst, ratio)
            assert ratio < 64.0, (L, T, s, alpha, n, G[n], float(g_ref), ratio)
    assert worst > 0.0


def test_wrong_sign_of_the_recursion_fails():
    # a plausible slip (+R^2 instead of -R^2) is caught by the same reference
    bad = 0
    for L, T, s, alpha in _grid():
        G = merged_recursion(L, T, s, alpha, sign=+1.0)
        for n, (g_ref, scale) in enumerate(reference(L, T, s, alpha)):
            if abs(G[n] - float(g_ref)) > 64.0 * EPS * float(scale):
                bad += 1
    assert bad > 0
