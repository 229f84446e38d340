"""Pins of the oracle's higher angular momentum blocks (three-center, two-center,
overlap and Fourier transform) against brute-force quadrature that shares no
code or formula with the McMurchie-Davidson recursions (tests/quadrature_ref.py).
A dropped term, a wrong sign, a swapped index or a transposed component order in
the oracle would fail these."""
import numpy as np
import pytest

from quadrature_ref import int3c, ovlp, ft

RNG = np.random.default_rng(2024)


def _case(maxl=3):
    lc, la, lb = (int(x) for x in RNG.integers(0, maxl + 1, 3))
    g, a, b = (float(x) for x in np.exp(RNG.uniform(np.log(0.4), np.log(4.0), 3)))
    C, A, B = RNG.uniform(-1.2, 1.2, (3, 3))
    return lc, g, C, la, a, A, lb, b, B


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("rep", range(4))
def test_3c_vs_quadrature(orc, kernel, rep):
    lc, g, C, la, a, A, lb, b, B = _case()
    omega = float(RNG.uniform(0.3, 1.5))
    v = orc.prim3c(kernel, omega, lc, g, C, la, a, A, lb, b, B)
    r = int3c(kernel, omega, lc, g, C, la, a, A, lb, b, B)
    scale = max(1e-3, np.max(np.abs(r)))
    assert np.max(np.abs(v - r)) < 2e-10 * scale, (kernel, lc, la, lb, np.max(np.abs(v - r)), scale)


def test_fixed_high_l_case(orc):
    # (f | d f) with all centres distinct, erfc kernel
    C, A, B = np.array([0.1, -0.4, 0.3]), np.array([-0.5, 0.2, 0.9]), np.array([0.7, 0.6, -0.3])
    v = orc.prim3c(2, 0.6, 3, 1.1, C, 2, 0.8, A, 3, 1.7, B)
    r = int3c(2, 0.6, 3, 1.1, C, 2, 0.8, A, 3, 1.7, B)
    assert np.max(np.abs(v - r)) < 2e-10 * np.max(np.abs(r))


@pytest.mark.parametrize("kernel", [0, 2])
def test_2c_vs_quadrature(orc, kernel):
    for _ in range(3):
        lc, g, C, ld, e, D, _, _, _ = _case()
        v = orc.prim2c(kernel, 0.8, lc, g, C, ld, e, D)
        r = int3c(kernel, 0.8, lc, g, C, ld, e, D, 0, 0.0, D)[:, :, 0]
        assert np.max(np.abs(v - r)) < 2e-10 * max(1e-3, np.max(np.abs(r)))


def test_overlap_vs_quadrature(orc):
    for _ in range(6):
        _, _, _, la, a, A, lb, b, B = _case()
        v = orc.prim_ovlp(la, a, A, lb, b, B)
        r = ovlp(la, a, A, lb, b, B)
        assert np.max(np.abs(v - r)) < 1e-11 * max(1e-3, np.max(np.abs(r)))


def test_ft_vs_quadrature(orc):
    for _ in range(6):
        _, _, _, la, a, A, lb, b, B = _case()
        q = RNG.uniform(-2.5, 2.5, 3)
        v = orc.prim_ft(la, a, A, lb, b, B, q)
        r = ft(la, a, A, lb, b, B, q)
        assert np.max(np.abs(v - r)) < 1e-10 * max(1e-3, np.max(np.abs(r)))
