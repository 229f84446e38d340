"""First-order Hartree-Fock energy error of a j3c tensor (host, FP64 numpy).

An accuracy metric for reporting, not part of the integral path.  The aux
metric J^k (j2c) is inverted on its well-conditioned part: with
J^k = U diag(lam) U^H, the fitting transform is W_k = diag(lam)^{-1/2} U^H
restricted to lam > rel * max(lam) (canonical orthogonalisation; Cartesian
even-tempered aux sets are nearly linearly dependent, and a Cholesky inverse
would amplify any integral error along those directions).  The fitted
three-index factors are B^{k1k2} = W_{k12} V^{k1k2}, and for a fixed
closed-shell density D^k the fitted Coulomb and exchange energies per cell are

    E_J = 1/(2 N_k^2) sum_P | sum_k sum_{mu nu} B^{kk}_{P mu nu} D^k_{nu mu} |^2
    E_K = -1/(4 N_k^2) sum_{k1 k2} sum_P Tr[ D^{k1} B^{k1k2}_P D^{k2} (B^{k1k2}_P)^H ].

With the density held fixed, an integral error changes the converged HF energy
only at first order, so |dE_J| + |dE_K| between two j3c tensors measures
their HF-energy discrepancy.  The density is synthetic: per k a seeded
random complex C^k (n_ao x n_occ) with orthonormal columns (Euclidean
metric), C^{-k} = conj(C^k), D^k = 2 C^k C^k^H.
"""
from __future__ import annotations

import numpy as np


def _unravel(k, kmesh):
    return (k // (kmesh[1] * kmesh[2]), (k // kmesh[2]) % kmesh[1], k % kmesh[2])


def _ravel(n, kmesh):
    return (n[0] % kmesh[0]) * kmesh[1] * kmesh[2] + (n[1] % kmesh[1]) * kmesh[2] + n[2] % kmesh[2]


def kneg(k, kmesh):
    n = _unravel(k, kmesh)
    return _ravel((-n[0], -n[1], -n[2]), kmesh)


def k12(k1, k2, kmesh):
    a, b = _unravel(k1, kmesh), _unravel(k2, kmesh)
    return _ravel((b[0] - a[0], b[1] - a[1], b[2] - a[2]), kmesh)


def densities(kmesh, nao, nocc, seed=0):
    """D[k] (complex [nk][nao][nao]) with D^{-k} = conj(D^k), trace 2 nocc."""
    nk = int(np.prod(kmesh))
    rng = np.random.default_rng(seed)
    C = [None] * nk
    for k in range(nk):
        if C[k] is not None:
            continue
        A = rng.normal(size=(nao, nocc)) + 1j * rng.normal(size=(nao, nocc))
        Q, _ = np.linalg.qr(A)
        if kneg(k, kmesh) == k:
            Q = Q.real.astype(np.complex128)
            Q, _ = np.linalg.qr(Q)
        C[k] = Q
        C[kneg(k, kmesh)] = np.conj(Q)
    return np.array([2.0 * c @ c.conj().T for c in C])


def fit_transforms(J, rel=1e-6):
    """W[k] (kept x naux) with W J^k W^H = identity on the eigenvalues of J^k
    above rel * max; rel = 0 keeps every positive eigenvalue."""
    out = []
    for Jk in np.asarray(J):
        Jk = 0.5 * (Jk + Jk.conj().T)
        lam, U = np.linalg.eigh(Jk)
        keep = lam > max(rel * lam[-1], 0.0)
        out.append((U[:, keep] / np.sqrt(lam[keep])).conj().T)
    return out


def fitted_factors(V, kpairs, kmesh, W):
    """B[pair] = W_{k12} V[pair] (list: the kept rank may differ per k12)."""
    npair, naux, nao, _ = V.shape
    return [(W[k12(int(k1), int(k2), kmesh)] @ V[p].reshape(naux, nao * nao)).reshape(-1, nao, nao)
            for p, (k1, k2) in enumerate(kpairs)]


def energies(V, kpairs, kmesh, W, D):
    """(E_J, E_K) per cell over the given pairs (E_J from its diagonal pairs)."""
    nk = int(np.prod(kmesh))
    B = fitted_factors(np.asarray(V), np.asarray(kpairs), kmesh, W)
    rho = 0.0
    EK = 0.0
    for p, (k1, k2) in enumerate(kpairs):
        k1, k2 = int(k1), int(k2)
        if k1 == k2:
            rho = rho + np.einsum("pmn,nm->p", B[p], D[k1])
        # sum_P Tr[D1 B_P D2 B_P^H] = sum_P sum_{ml} (D1 B_P D2)_{ml} conj(B_P)_{ml}
        M = D[k1] @ B[p] @ D[k2]
        EK += float(np.sum(M * np.conj(B[p])).real)
    EJ = 0.5 * float(np.sum(np.abs(rho) ** 2)) / nk ** 2
    return EJ, -0.25 * EK / nk ** 2


def energy_error(V, Vref, kpairs, kmesh, J, rel=1e-6, nocc=None, seed=0):
    """|dE_J| + |dE_K| (Hartree per cell) between two j3c tensors fitted with
    the same metric J (j2c, [nk][naux][naux]), with the reference's energies
    for scale."""
    nao = V.shape[-1]
    W = fit_transforms(J, rel)
    D = densities(kmesh, nao, nocc if nocc else max(1, nao // 4), seed)
    ej, ek = energies(V, kpairs, kmesh, W, D)
    rj, rk = energies(Vref, kpairs, kmesh, W, D)
    return {"dE_J": abs(ej - rj), "dE_K": abs(ek - rk), "dE": abs(ej - rj) + abs(ek - rk), "E_J": rj, "E_K": rk}
