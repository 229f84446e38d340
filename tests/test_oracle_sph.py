"""Pins of the Cartesian -> real solid harmonic oracle (oracle/sph.py): the
textbook forms for l <= 2, harmonicity (the Laplacian of every coefficient row
vanishes, computed exactly from the monomials), unit norm and orthogonality
within a shell through the oracle's own Cartesian overlap integrals (no shared
formula with the coefficient fit), and the tensor transforms against explicit
loops."""
import itertools
import math

import numpy as np
import pytest

from oracle import sph


def test_textbook_forms_up_to_d():
    assert np.allclose(sph.coefficients(0), [[1.0]], atol=1e-13)
    # p: m = -1, 0, 1 -> y, z, x (components x, y, z)
    assert np.allclose(sph.coefficients(1), [[0, 1, 0], [0, 0, 1], [1, 0, 0]], atol=1e-13)
    r3 = math.sqrt(3.0)
    # d components xx, xy, xz, yy, yz, zz
    want = [[0, r3, 0, 0, 0, 0],                 # m = -2: sqrt3 xy
            [0, 0, 0, 0, r3, 0],                 # m = -1: sqrt3 yz
            [-0.5, 0, 0, -0.5, 0, 1.0],          # m =  0: z^2 - (x^2 + y^2)/2
            [0, 0, r3, 0, 0, 0],                 # m =  1: sqrt3 xz
            [r3 / 2, 0, 0, -r3 / 2, 0, 0]]       # m =  2: sqrt3/2 (x^2 - y^2)
    assert np.allclose(sph.coefficients(2), want, atol=1e-12)


@pytest.mark.parametrize("l", [1, 2, 3, 4])
def test_rows_are_harmonic_of_degree_l(l):
    comps = sph.cart_components(l)
    idx = {c: i for i, c in enumerate(comps)}
    s = sph.coefficients(l)
    for row in s:
        lap = {}
        for coef, (a, b, c) in zip(row, comps):
            for d, (p, q, r) in enumerate([(a, b, c)] * 3):
                e = [p, q, r]
                if e[d] >= 2:
                    f = list(e)
                    f[d] -= 2
                    lap[tuple(f)] = lap.get(tuple(f), 0.0) + coef * e[d] * (e[d] - 1)
        assert max(abs(v) for v in lap.values()) < 1e-10 if lap else True
    assert np.linalg.matrix_rank(s) == 2 * l + 1
    assert len(idx) == (l + 1) * (l + 2) // 2


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_unit_norm_and_orthogonal_through_oracle_overlaps(orc, l):
    a = 0.7
    S = orc.prim_ovlp(l, a, np.zeros(3), l, a, np.zeros(3))
    Sn = S / S[0, 0]                     # Cartesian functions with the x^l component normalised
    s = sph.coefficients(l)
    assert np.max(np.abs(s @ Sn @ s.T - np.eye(2 * l + 1))) < 1e-10


def test_tensor_transforms_against_loops():
    rng = np.random.default_rng(3)
    ao_l, aux_l = [1, 0, 2], [2, 1]
    nca = sum((l + 1) * (l + 2) // 2 for l in ao_l)
    ncx = sum((l + 1) * (l + 2) // 2 for l in aux_l)
    V = rng.normal(size=(2, ncx, nca, nca)) + 1j * rng.normal(size=(2, ncx, nca, nca))
    J = rng.normal(size=(3, ncx, ncx)) + 1j * rng.normal(size=(3, ncx, ncx))
    Sa, Sx = sph.basis_matrix(ao_l), sph.basis_matrix(aux_l)
    out = sph.j3c(V, ao_l, aux_l)
    for i, P, M, N in itertools.product(range(2), range(Sx.shape[0]), range(Sa.shape[0]), range(Sa.shape[0])):
        v = 0.0
        for p, m, n in itertools.product(range(ncx), range(nca), range(nca)):
            v += Sx[P, p] * Sa[M, m] * Sa[N, n] * V[i, p, m, n]
        assert abs(out[i, P, M, N] - v) < 1e-12
    oj = sph.j2c(J, aux_l)
    for k, P, Q in itertools.product(range(3), range(Sx.shape[0]), range(Sx.shape[0])):
        v = sum(Sx[P, p] * Sx[Q, q] * J[k, p, q] for p in range(ncx) for q in range(ncx))
        assert abs(oj[k, P, Q] - v) < 1e-12
