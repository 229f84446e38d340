"""Pins of the SR screening (Supplementary Material, "Conditions for
prescreening the double lattice summation").

* For s functions the oracle's R_c cutoff must solve the boxed Eq. bound_Rc,
  restated here independently (scipy root finder, brute-force S_h).
* The near-field cell count N_cell^NF of a cubic lattice within 3 a is the
  number of integer points with |n| <= 3 (123).
* Screened results at eps stay within 10 eps per integral of converged ones
  (eps = 1e-14) -- the paper's estimates are asymptotic, not rigorous.
"""
import math

import numpy as np
from scipy.optimize import brentq

from paper_2102_02989_gb300 import inputs


def test_nf_cell_count_cubic(orc):
    assert orc.count_nf_cells(4.0 * np.eye(3)) == 123
    # independent brute count for an FCC cell
    a = inputs.fcc_cell(6.74)
    vol = abs(np.linalg.det(a))
    rad = 3 * vol ** (1 / 3)
    n = 0
    for i in range(-12, 13):
        for j in range(-12, 13):
            for k in range(-12, 13):
                if np.linalg.norm(np.array([i, j, k]) @ a) <= rad:
                    n += 1
    assert orc.count_nf_cells(a) == n


def test_rc_bound_s_functions(orc):
    a = 5.0 * np.eye(3)
    vol = 125.0
    omega, eps = 0.6, 1e-9
    aP, am, an = 0.7, 1.3, 0.45
    A_, B_ = np.zeros(3), np.array([1.1, 0.4, -0.3])
    aux = inputs.make_basis([(0, np.zeros(3), [aP], [1.0])])
    ao = inputs.make_basis([(0, A_, [am], [1.0]), (0, B_, [an], [1.0])])
    rc, r12 = orc.sr_bounds(a, omega, eps, aux, 0, ao, 0, 1)
    n1s = lambda x: (2 * x / math.pi) ** 0.75
    p = am + an
    beta = am * an / p
    A = math.pi ** 3 * n1s(aP) * n1s(am) * n1s(an) / (aP * p) ** 1.5
    sh, hmax = 0.0, 0.0
    for i in range(-6, 7):
        for j in range(-6, 7):
            for k in range(-6, 7):
                R = np.linalg.norm(B_ + np.array([i, j, k]) @ a - A_)
                h = math.exp(-beta * R * R)
                hmax = max(hmax, h)
                if h >= 1e-4:
                    sh += h
    sh = max(sh, hmax)
    e1 = 1 / math.sqrt(1 / aP + 1 / p)
    e2 = 1 / math.sqrt(1 / e1 ** 2 + 1 / omega ** 2)
    g = lambda R: A * sh * 4 * math.pi / vol / math.sqrt(math.pi) / (2 * e2 ** 3) / R * math.exp(-(e2 * R) ** 2) - eps
    ref = brentq(g, 1e-3, 200.0, xtol=1e-13)
    assert abs(rc - ref) < 1e-8 * ref
    # the R12 windows are no shorter than the eps'-radius floor and cover [0, Rc_cut]
    assert len(r12) == int(rc // 1.0) + 1
    assert np.all(np.diff(r12[len(r12) // 2:]) <= 1e-12)   # decreasing in the far windows


def test_screened_within_10_eps_config1(orc):
    p = inputs.config1()
    eps = 1e-8
    V = orc.j3c(p.a, p.kmesh, p.ao, p.aux, p.omega, [(0, 0)], eps_sr=eps, lr=False, g0=False)
    Vc = orc.j3c(p.a, p.kmesh, p.ao, p.aux, p.omega, [(0, 0)], eps_sr=1e-14, lr=False, g0=False)
    err = np.max(np.abs(V - Vc))
    assert err < 10 * eps, err
    # and the screen is not vacuous: a 100x looser eps gives a visibly larger error
    V2 = orc.j3c(p.a, p.kmesh, p.ao, p.aux, p.omega, [(0, 0)], eps_sr=1e-6, lr=False, g0=False)
    assert np.max(np.abs(V2 - Vc)) > 3 * err


def test_screened_within_10_eps_config2_subset(orc):
    from rules_ref import omega_for
    p = inputs.config2()
    w = omega_for(p.a, p.gmesh, p.eps_lr, p.kmesh)
    kp = [(0, 0), (1, 6), (3, 2)]
    sh = (12, 16)    # the d and f aux shells of the first atom
    V = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp, eps_sr=1e-8, lr=False, g0=False, shells=sh)
    Vc = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp, eps_sr=1e-13, lr=False, g0=False, shells=sh)
    assert np.max(np.abs(V - Vc)) < 10 * 1e-8
