"""Pins of the oracle's Cholesky factorisation (textbook, column by column)
against LAPACK through numpy, and of its non-positive-pivot report on a
metric made singular by a duplicated aux shell (the linear-dependence case the
paper meets for LiF)."""
import numpy as np

from paper_2102_02989_gb300 import inputs
from rules_ref import gmesh_for


def test_cholesky_matches_lapack(orc):
    rng = np.random.default_rng(5)
    for n in (1, 2, 7, 40):
        X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        A = X @ X.conj().T + n * np.eye(n)
        L, piv = orc.cholesky(A)
        assert piv == -1
        assert np.max(np.abs(L - np.linalg.cholesky(A))) < 1e-12 * n
        assert np.max(np.abs(np.triu(L, 1))) == 0.0


def test_cholesky_reports_first_bad_pivot(orc):
    rng = np.random.default_rng(6)
    X = rng.normal(size=(6, 3))
    A = (X @ X.T).astype(complex)          # rank 3
    L, piv = orc.cholesky(A)
    assert piv == 3


def test_duplicated_aux_shell_makes_j2c_singular(orc):
    p = inputs.tiny(lmax_aux=1)
    aux = inputs.make_basis([(int(p.aux.l[0]), p.aux.center[0], [p.aux.exps[0]], [1.0]),
                             (int(p.aux.l[0]), p.aux.center[0], [p.aux.exps[0]], [1.0])])
    J = orc.j2c(p.a, (1, 1, 1), aux, 0.9, [0], eps_sr=1e-12, eps_lr=1e-14,
                gmesh=gmesh_for(p.a, 0.9, 1e-14, (1, 1, 1)))
    # the two rows agree up to the summation order of the threaded oracle: the
    # second pivot is zero or a rounding-level positive, never a real one
    L, piv = orc.cholesky(J[0])
    assert piv == 1 or (piv == -1 and abs(L[1, 1]) ** 2 <= 1e-12 * J[0][0, 0].real)
    from oracle import dfjk
    assert dfjk.cholesky_rel(J[0], rel=1e-12)[1] == 1
