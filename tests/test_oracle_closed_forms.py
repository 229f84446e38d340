"""Pins of the oracle's primitive integrals against textbook closed forms.

s-type Gaussians: e^{-a r_A^2} e^{-b r_B^2} = K e^{-p r_P^2} with p = a+b,
K = exp(-ab/p |A-B|^2).  Two Gaussian charge clouds of exponents g, p at
distance R interact through 1/r as (pi/g)^{3/2} (pi/p)^{3/2} erf(eta R)/R with
eta^2 = g p/(g+p); through erf(omega r)/r eta is replaced by eta_w with
1/eta_w^2 = 1/eta^2 + 1/omega^2, and erfc = 1/r - erf.  This is the s-type
result that the Supplementary Material's screening section starts from (its
functions h(R12) and f(Rc) with eta1, eta2)."""
import math

import numpy as np
import pytest

RNG = np.random.default_rng(11)


def s3c_closed(kernel, omega, g, C, a, A, b, B):
    A, B, C = map(np.asarray, (A, B, C))
    p = a + b
    K = math.exp(-a * b / p * np.sum((A - B) ** 2))
    P = (a * A + b * B) / p
    R = float(np.linalg.norm(P - C))
    eta = math.sqrt(g * p / (g + p))
    etw = 1.0 / math.sqrt(1.0 / eta ** 2 + 1.0 / omega ** 2)

    def ferf(e):
        return 2 * e / math.sqrt(math.pi) if R < 1e-12 else math.erf(e * R) / R

    pref = (math.pi / g) ** 1.5 * (math.pi / p) ** 1.5 * K
    if kernel == 0:
        return pref * ferf(eta)
    if kernel == 1:
        return pref * ferf(etw)
    return pref * (ferf(eta) - ferf(etw))


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_s3c_closed_form(orc, kernel):
    for _ in range(40):
        g, a, b = np.exp(RNG.uniform(np.log(0.05), np.log(50.0), 3))
        C, A, B = RNG.uniform(-3, 3, (3, 3))
        omega = float(RNG.uniform(0.2, 2.0))
        v = orc.prim3c(kernel, omega, 0, g, C, 0, a, A, 0, b, B)[0, 0, 0]
        ref = s3c_closed(kernel, omega, g, C, a, A, b, B)
        assert abs(v - ref) <= 1e-13 * max(1.0, abs(ref)), (kernel, v, ref)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_s3c_coincident_centres_limit(orc, kernel):
    # R -> 0 limit 2 eta / sqrt(pi) of erf(eta R)/R
    C = A = B = np.array([0.3, -0.2, 1.1])
    v = orc.prim3c(kernel, 0.7, 0, 1.3, C, 0, 0.9, A, 0, 2.1, B)[0, 0, 0]
    ref = s3c_closed(kernel, 0.7, 1.3, C, 0.9, A, 2.1, B)
    assert abs(v - ref) < 1e-13 * abs(ref)


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_s2c_closed_form(orc, kernel):
    for _ in range(30):
        g, e = np.exp(RNG.uniform(np.log(0.05), np.log(50.0), 2))
        C, D = RNG.uniform(-3, 3, (2, 3))
        omega = float(RNG.uniform(0.2, 2.0))
        v = orc.prim2c(kernel, omega, 0, g, C, 0, e, D)[0, 0]
        # a Gaussian pair with b = 0 is the Gaussian itself
        ref = s3c_closed(kernel, omega, g, C, e, D, 1e-300, D)
        assert abs(v - ref) <= 1e-13 * max(1.0, abs(ref))


def test_erf_plus_erfc_is_coulomb(orc):
    for _ in range(20):
        lc, la, lb = RNG.integers(0, 4, 3)
        g, a, b = np.exp(RNG.uniform(np.log(0.1), np.log(10.0), 3))
        C, A, B = RNG.uniform(-2, 2, (3, 3))
        w = float(RNG.uniform(0.1, 3.0))
        full = orc.prim3c(0, w, lc, g, C, la, a, A, lb, b, B)
        lr = orc.prim3c(1, w, lc, g, C, la, a, A, lb, b, B)
        sr = orc.prim3c(2, w, lc, g, C, la, a, A, lb, b, B)
        assert np.max(np.abs(lr + sr - full)) < 1e-12 * max(1.0, np.max(np.abs(full)))


def test_s_overlap_and_charge(orc):
    for _ in range(20):
        a, b = np.exp(RNG.uniform(np.log(0.05), np.log(50.0), 2))
        A, B = RNG.uniform(-2, 2, (2, 3))
        p = a + b
        ref = (math.pi / p) ** 1.5 * math.exp(-a * b / p * np.sum((A - B) ** 2))
        assert abs(orc.prim_ovlp(0, a, A, 0, b, B)[0, 0] - ref) < 1e-14 * max(1, ref)


def test_s_fourier_transform(orc):
    # int e^{-a (r-A)^2} e^{-i q.r} dr = (pi/a)^{3/2} e^{-q^2/4a} e^{-i q.A}
    for _ in range(20):
        a = float(np.exp(RNG.uniform(np.log(0.05), np.log(50.0))))
        A, q = RNG.uniform(-2, 2, (2, 3))
        ref = (math.pi / a) ** 1.5 * math.exp(-q @ q / (4 * a)) * np.exp(-1j * q @ A)
        v = orc.prim_ft(0, a, A, 0, 0.0, A, q)[0, 0]
        assert abs(v - ref) < 1e-14 * max(1, abs(ref))


def test_ft_at_zero_is_overlap(orc):
    for _ in range(10):
        la, lb = RNG.integers(0, 4, 2)
        a, b = np.exp(RNG.uniform(np.log(0.2), np.log(5.0), 2))
        A, B = RNG.uniform(-1, 1, (2, 3))
        ft = orc.prim_ft(la, a, A, lb, b, B, np.zeros(3))
        ov = orc.prim_ovlp(la, a, A, lb, b, B)
        assert np.max(np.abs(ft - ov)) < 1e-14 * max(1, np.max(np.abs(ov)))


def test_normalisation_unit_xl_norm(orc):
    """Every contracted shell's x^l component has unit norm: check with the
    overlap of two copies at the same centre (only the (x^l, x^l) entry)."""
    from paper_2102_02989_gb300 import inputs
    p = inputs.config2()
    cn = orc.norm_coeffs(p.ao)
    for s in range(p.ao.nshell):
        l = int(p.ao.l[s]); o = int(p.ao.prim_off[s]); n = int(p.ao.nprim[s])
        A = p.ao.center[s]
        tot = 0.0
        for i in range(n):
            for j in range(n):
                tot += cn[o + i] * cn[o + j] * orc.prim_ovlp(l, p.ao.exps[o + i], A, l, p.ao.exps[o + j], A)[0, 0]
        assert abs(tot - 1.0) < 1e-13
