"""Plain FP64 reference of the density-fitting consumers of j3c (test infrastructure).

TEST INFRASTRUCTURE ONLY (tests, smoke check, bench CPU leg).  Written from the
definitions, with numpy only:

Fitting transform of the aux metric (Eq. DF_eqn, whose normal equations
J^{k12} d = V are solved here through a factor of J).  For each k a matrix
T_k with T_k^H T_k = (J^k)^{-1} on the part of J^k that is kept:
  * Cholesky route: J^k = L L^H (L lower, positive real diagonal), T_k = L^{-1}.
    Pivot j fails when its Schur-complement diagonal d_j <= rel * max_i J_ii
    (rel = 0: the plain positivity test).
  * eigen route (canonical orthogonalisation, the fallback for a singular or
    nearly singular metric such as a linearly dependent aux set): the
    Hermitian part of J^k is U diag(lam) U^H with lam descending; row r of
    T_k is lam_r^{-1/2} (column r of U)^H for lam_r > rel * lam_0, zero for the
    rows beyond the kept count.
  * auto: Cholesky where it succeeds, eigen elsewhere.

Fitted three-index factors: B^{k1k2} = T_{k12} V^{k1k2} (k12 = k2 - k1 on the
mesh), so that sum_P B_P (x) conj(B_P) = sum_{QR} V_Q (x) conj(V_R) (J^{-1})_{RQ},
the fitted ERIs of Eq. ERI_aux.

Coulomb and exchange matrices of a density D^k (closed shell, D = 2 C C^H):
  rho_P  = sum_{(k,k) in pairs} sum_{mu nu} B^{kk}_{P mu nu} D^k_{nu mu}
  J^k    = (1/N_k) sum_P B^{kk}_P conj(rho_P)             (k with a pair (k, k))
  K^{k1} = (1/N_k) sum_{(k1,k2) in pairs} sum_P B^{k1k2}_P D^{k2} (B^{k1k2}_P)^H
and the energies per cell E_J = (1/2N_k) sum_k Tr[D^k J^k],
E_K = -(1/4N_k) sum_k Tr[D^k K^k].

Pins: tests/test_oracle_dfjk.py (inverse through other library routines,
LAPACK Cholesky, the pivot of a duplicated function, route independence, and
brute-force fitted-ERI energies built with an explicit metric inverse).
"""
from __future__ import annotations

import numpy as np


def k12_index(k1: int, k2: int, kmesh) -> int:
    """mesh index of k2 - k1 (last direction fastest)"""
    n1, n2 = kmesh[1], kmesh[2]
    a = (k1 // (n1 * n2), (k1 // n2) % n1, k1 % n2)
    b = (k2 // (n1 * n2), (k2 // n2) % n1, k2 % n2)
    d = [(b[i] - a[i]) % kmesh[i] for i in range(3)]
    return (d[0] * n1 + d[1]) * n2 + d[2]


def cholesky_rel(A, rel: float = 0.0):
    """Column-by-column Cholesky of the lower triangle of A; returns (L, pivot)
    with pivot = -1 on success, else the first j whose d_j <= rel * max diag
    (L then partial)."""
    A = np.array(A, dtype=np.complex128)
    n = A.shape[0]
    L = np.tril(A)
    cut = rel * float(np.max(np.real(np.diag(A))))
    for j in range(n):
        d = float(np.real(L[j, j]))
        if not d > cut or not d > 0.0:
            return L, j
        L[j, j] = np.sqrt(d)
        L[j + 1:, j] /= L[j, j]
        # Schur complement of the trailing lower triangle
        col = L[j + 1:, j]
        L[j + 1:, j + 1:] -= np.tril(np.outer(col, np.conj(col)))
    return L, -1


def transform_cholesky(Jk, rel: float = 0.0):
    """(T, pivot): T = L^{-1} (lower), or None and the failing pivot."""
    L, piv = cholesky_rel(Jk, rel)
    if piv >= 0:
        return None, piv
    n = L.shape[0]
    T = np.zeros_like(L)
    # forward substitution L T = I, column by column
    for j in range(n):
        x = np.zeros(n, dtype=np.complex128)
        x[j] = 1.0 / L[j, j]
        for i in range(j + 1, n):
            x[i] = -np.dot(L[i, j:i], x[j:i]) / L[i, i]
        T[:, j] = x
    return T, -1


def transform_eigen(Jk, rel: float = 1e-6):
    """(T, lam descending, nkept) by canonical orthogonalisation."""
    H = 0.5 * (np.asarray(Jk) + np.asarray(Jk).conj().T)
    lam, U = np.linalg.eigh(H)
    lam, U = lam[::-1], U[:, ::-1]
    keep = lam > max(rel * lam[0], 0.0)
    T = np.zeros_like(H)
    nk = int(np.count_nonzero(keep))
    T[:nk] = (U[:, :nk] / np.sqrt(lam[:nk])).conj().T
    return T, lam, nk


def metric_transforms(J, method: str = "auto", rel: float = 1e-6):
    """Per k: T [nk][n][n], route ('cholesky' | 'eigen'), kept rows, failing
    pivot (-1 if none).  method 'cholesky' leaves T zero where it fails."""
    J = np.asarray(J)
    nk, n, _ = J.shape
    T = np.zeros((nk, n, n), dtype=np.complex128)
    route, kept, pivot = [], [], []
    for k in range(nk):
        Tk, piv = (None, -1)
        if method in ("cholesky", "auto"):
            Tk, piv = transform_cholesky(J[k], rel)
        if Tk is not None:
            T[k], r, c = Tk, "cholesky", n
        elif method == "cholesky":
            r, c = "cholesky", 0
        else:
            T[k], _, c = transform_eigen(J[k], rel)
            r = "eigen"
        route.append(r)
        kept.append(c)
        pivot.append(piv)
    return T, route, kept, pivot


def fit(T, V, kpairs, kmesh):
    """B[pair] = T[k12] V[pair]; V, B complex [npair][naux][nao][nao]"""
    V = np.asarray(V)
    npair, naux, nao, _ = V.shape
    B = np.zeros_like(V, dtype=np.complex128)
    for p, (k1, k2) in enumerate(np.asarray(kpairs)):
        q = k12_index(int(k1), int(k2), kmesh)
        B[p] = (T[q] @ V[p].reshape(naux, nao * nao)).reshape(naux, nao, nao)
    return B


def jk(B, kpairs, kmesh, D, rho=None):
    """(J, K, rho): J, K complex [Nk][nao][nao] as defined in the header; rho
    given (the fitted density over more pairs than these) replaces the one
    summed from the listed diagonal pairs in J."""
    B = np.asarray(B)
    D = np.asarray(D)
    nk = int(np.prod(kmesh))
    npair, naux, nao, _ = B.shape
    if rho is None:
        rho = np.zeros(naux, dtype=np.complex128)
        for p, (k1, k2) in enumerate(np.asarray(kpairs)):
            if k1 == k2:
                rho += np.einsum("pmn,nm->p", B[p], D[k1])
    Jm = np.zeros((nk, nao, nao), dtype=np.complex128)
    Km = np.zeros((nk, nao, nao), dtype=np.complex128)
    for p, (k1, k2) in enumerate(np.asarray(kpairs)):
        k1, k2 = int(k1), int(k2)
        if k1 == k2:
            Jm[k1] = np.einsum("pmn,p->mn", B[p], np.conj(rho)) / nk
        for P in range(naux):
            Km[k1] += B[p, P] @ D[k2] @ B[p, P].conj().T / nk
    return Jm, Km, rho


def energies(Jm, Km, D):
    """(E_J, E_K) per cell from the Coulomb and exchange matrices."""
    nk = len(D)
    ej = sum(np.trace(D[k] @ Jm[k]) for k in range(nk)) / (2 * nk)
    ek = -sum(np.trace(D[k] @ Km[k]) for k in range(nk)) / (4 * nk)
    return float(np.real(ej)), float(np.real(ek))
