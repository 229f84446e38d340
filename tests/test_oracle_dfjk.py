"""Pins of the density-fitting oracle (oracle/dfjk.py) against things other
than itself: the metric inverse from LAPACK's LU inverse, LAPACK's Cholesky,
the pivot a linearly dependent aux set must fail at, the k12 index from
fractional k vectors, and energies of the fitted ERIs (Eq. ERI_aux) written
out by brute force with an explicit metric inverse."""
import itertools

import numpy as np
import pytest

from oracle import dfjk
from paper_2102_02989_gb300 import inputs


def test_k12_index_from_fractional_vectors():
    for kmesh in [(2, 1, 1), (2, 3, 2), (3, 3, 3)]:
        ks = list(itertools.product(*[range(n) for n in kmesh]))
        frac = {k: np.array(k, float) / np.array(kmesh) for k in ks}
        for i1, a in enumerate(ks):
            for i2, b in enumerate(ks):
                f = np.mod(frac[b] - frac[a], 1.0)
                want = [i for i, c in enumerate(ks) if np.allclose(frac[c], f)]
                assert dfjk.k12_index(i1, i2, kmesh) == want[0]


def test_cholesky_matches_lapack():
    rng = np.random.default_rng(11)
    for n in (1, 3, 17):
        X = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
        A = X @ X.conj().T + 0.1 * np.eye(n)
        L, piv = dfjk.cholesky_rel(A)
        assert piv == -1
        assert np.max(np.abs(L - np.linalg.cholesky(A))) < 1e-12 * np.max(np.abs(A))


@pytest.mark.parametrize("kmesh", [(1, 1, 1), (3, 1, 1)])
def test_transforms_invert_the_metric(kmesh):
    J, _, _ = inputs.df_synthetic(kmesh, naux=20, nao=2, cond=1e-5, seed=1)
    for method in ("cholesky", "eigen", "auto"):
        T, route, kept, piv = dfjk.metric_transforms(J, method, rel=0.0)
        for k in range(len(J)):
            inv = np.linalg.inv(J[k])
            assert kept[k] == 20
            err = np.max(np.abs(T[k].conj().T @ T[k] - inv)) / np.max(np.abs(inv))
            assert err < 1e-9, (method, k, err)
            assert np.max(np.abs(T[k] @ J[k] @ T[k].conj().T - np.eye(20))) < 1e-9
        if method != "eigen":
            assert route == ["cholesky"] * len(J)
            assert all(np.max(np.abs(np.triu(T[k], 1))) == 0 for k in range(len(J)))


def test_linearly_dependent_metric_fails_cholesky_and_falls_back():
    naux, rank = 16, 13
    J, _, _ = inputs.df_synthetic((2, 1, 1), naux=naux, nao=2, rank=rank, seed=2)
    T, route, kept, piv = dfjk.metric_transforms(J, "cholesky", rel=1e-10)
    assert piv == [rank, rank] and kept == [0, 0] and np.all(T == 0)
    T, route, kept, piv = dfjk.metric_transforms(J, "auto", rel=1e-10)
    assert route == ["eigen", "eigen"] and kept == [rank, rank]
    for k in range(2):
        # T^H T is the pseudo-inverse; T J T^H the identity on the kept rows
        pinv = np.linalg.pinv(J[k], rcond=1e-10, hermitian=False)
        assert np.max(np.abs(T[k].conj().T @ T[k] - pinv)) < 1e-9 * np.max(np.abs(pinv))
        P = T[k] @ J[k] @ T[k].conj().T
        assert np.max(np.abs(P - np.diag([1.0] * rank + [0.0] * (naux - rank)))) < 1e-9
    # an exactly duplicated function fails at the copy's pivot
    A = inputs.df_synthetic((1, 1, 1), naux=8, nao=2, cond=1e-2, seed=3)[0][0]
    idx = [0, 1, 2, 3, 2, 4, 5, 6, 7]
    Ad = A[np.ix_(idx, idx)]
    _, pv = dfjk.cholesky_rel(Ad, rel=1e-12)
    assert pv == 4


def _brute_energies(V, kpairs, kmesh, D, Jinv):
    nk = int(np.prod(kmesh))
    npair, naux, nao, _ = V.shape
    v = np.zeros(naux, dtype=complex)
    for p, (k1, k2) in enumerate(kpairs):
        if k1 != k2:
            continue
        for Q in range(naux):
            for mu in range(nao):
                for nu in range(nao):
                    v[Q] += V[p, Q, mu, nu] * D[k1][nu, mu]
    ej = 0.0
    for Q in range(naux):
        for R in range(naux):
            ej += np.conj(v[Q]) * Jinv[0][Q, R] * v[R]
    ek = 0.0
    for p, (k1, k2) in enumerate(kpairs):
        q = [i for i in range(nk) if np.allclose(
            np.mod(np.array(np.unravel_index(k2, kmesh)) - np.array(np.unravel_index(k1, kmesh)), kmesh),
            np.unravel_index(i, kmesh))][0]
        for Q in range(naux):
            for R in range(naux):
                s = 0.0
                for nu, mu, la, si in itertools.product(range(nao), repeat=4):
                    s += D[k1][nu, mu] * V[p, Q, mu, la] * D[k2][la, si] * np.conj(V[p, R, nu, si])
                ek += Jinv[q][R, Q] * s
    return float(np.real(ej)) / (2 * nk * nk), -float(np.real(ek)) / (4 * nk * nk)


@pytest.mark.parametrize("method,rank", [("cholesky", None), ("eigen", None), ("auto", 4)])
def test_energies_equal_fitted_eri_brute_force(method, rank):
    kmesh = (2, 1, 1)
    J, V, D = inputs.df_synthetic(kmesh, naux=6, nao=3, nocc=1, cond=1e-3, rank=rank, seed=4)
    kp = inputs.kpairs_all(2)
    T, route, kept, _ = dfjk.metric_transforms(J, method, rel=1e-10)
    B = dfjk.fit(T, V, kp, kmesh)
    Jm, Km, _ = dfjk.jk(B, kp, kmesh, D)
    ej, ek = dfjk.energies(Jm, Km, D)
    Jinv = [np.linalg.pinv(J[k], rcond=1e-10) if rank else np.linalg.inv(J[k]) for k in range(2)]
    bj, bk = _brute_energies(V, kp, kmesh, D, Jinv)
    assert abs(ej - bj) < 1e-10 * abs(bj) and abs(ek - bk) < 1e-10 * abs(bk), (ej, bj, ek, bk)
    for k in range(2):
        assert np.max(np.abs(Km[k] - Km[k].conj().T)) < 1e-12 * np.max(np.abs(Km[k]))


def test_energies_independent_of_the_route():
    kmesh = (3, 1, 1)
    J, V, D = inputs.df_synthetic(kmesh, naux=12, nao=4, nocc=2, cond=1e-4, seed=5)
    kp = inputs.kpairs_all(3)
    out = []
    for method in ("cholesky", "eigen"):
        T, _, _, _ = dfjk.metric_transforms(J, method, rel=0.0)
        Jm, Km, _ = dfjk.jk(dfjk.fit(T, V, kp, kmesh), kp, kmesh, D)
        out.append((Jm, Km))
    for a, b in zip(out[0], out[1]):
        assert np.max(np.abs(a - b)) < 1e-9 * np.max(np.abs(a))
