"""Pins of the oracle's Boys function F_m(T) = int_0^1 t^{2m} e^{-T t^2} dt
against closed forms and library routines that share nothing with it."""
import math

import numpy as np
import pytest
from scipy import special


def boys_scipy(m, T):
    # F_m(T) = Gamma(m+1/2) P(m+1/2, T) / (2 T^{m+1/2})   (regularised lower incomplete gamma)
    if T == 0.0:
        return 1.0 / (2 * m + 1)
    return special.gamma(m + 0.5) * special.gammainc(m + 0.5, T) / (2.0 * T ** (m + 0.5))


@pytest.mark.parametrize("T", [0.0, 1e-12, 1e-6, 0.1, 0.7, 1.3, 5.0, 11.9, 22.0, 29.999, 30.0, 30.001, 45.0, 120.0, 900.0])
def test_boys_vs_incomplete_gamma(orc, T):
    F = orc.boys(16, T)
    for m in range(17):
        ref = boys_scipy(m, T)
        assert abs(F[m] - ref) <= 1e-14 * max(1.0, abs(ref)) + 1e-300, (m, T, F[m], ref)


def test_boys_f0_erf_closed_form(orc):
    for T in np.linspace(0.01, 60, 97):
        ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        assert abs(orc.boys(0, T)[0] - ref) < 1e-15


def test_boys_mpmath_high_precision(orc):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    for T in (0.37, 3.3, 17.5, 33.0):
        F = orc.boys(12, T)
        for m in (0, 3, 7, 12):
            ref = mpmath.quad(lambda t: t ** (2 * m) * mpmath.exp(-T * t * t), [0, 1])
            assert abs(F[m] - float(ref)) < 1e-15 * max(1.0, float(ref))


def test_boys_downward_recursion_identity(orc):
    # F_m = (2T F_{m+1} + e^{-T}) / (2m+1) holds for every T
    for T in (0.2, 4.0, 29.0, 31.0, 80.0):
        F = orc.boys(14, T)
        for m in range(14):
            assert abs(F[m] - (2 * T * F[m + 1] + math.exp(-T)) / (2 * m + 1)) < 1e-15 * max(1, F[m])
