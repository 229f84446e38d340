"""Seeded synthetic inputs: cells, AO and auxiliary shells, k-meshes.

This module holds no arithmetic of the method (no normalisation, no integrals,
no screening, no parameter rules); it only draws the geometry and the shell
data that both the CUDA library and the CPU oracle consume.  The paper's own
workloads (diamond/cc-pVDZ with cc-pVDZ-jkfit; MgO and LiF with GTH-DZVP and an
even-tempered auxiliary basis of progression 2.0) are not available here; the
shapes below stand in for them: an FCC two-atom cell at diamond's lattice
constant, 3s2p1d AO shells per atom, and an even-tempered auxiliary basis of
about three times the AO count.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 2102_02989


@dataclass
class Basis:
    """Contracted Cartesian shells.  ``coeffs`` are raw contraction coefficients
    of the primitives; the libraries apply the normalisation themselves."""
    l: np.ndarray          # [nshell] int32
    nprim: np.ndarray      # [nshell] int32
    prim_off: np.ndarray   # [nshell] int32
    center: np.ndarray     # [nshell, 3] float64, Bohr
    exps: np.ndarray       # [nprim_total] float64
    coeffs: np.ndarray     # [nprim_total] float64

    @property
    def nshell(self) -> int:
        return int(len(self.l))

    @property
    def nfunc(self) -> int:
        return int(sum((int(l) + 1) * (int(l) + 2) // 2 for l in self.l))

    def subset(self, shells) -> "Basis":
        shells = list(shells)
        l, npr, off, cen, ex, co = [], [], [], [], [], []
        o = 0
        for s in shells:
            n = int(self.nprim[s])
            p0 = int(self.prim_off[s])
            l.append(int(self.l[s])); npr.append(n); off.append(o); cen.append(self.center[s])
            ex.extend(self.exps[p0:p0 + n]); co.extend(self.coeffs[p0:p0 + n])
            o += n
        return Basis(np.array(l, np.int32), np.array(npr, np.int32), np.array(off, np.int32),
                     np.array(cen, np.float64).reshape(-1, 3), np.array(ex, np.float64),
                     np.array(co, np.float64))


def make_basis(shells) -> Basis:
    """shells: iterable of (l, centre[3], exps[], coeffs[])."""
    l, npr, off, cen, ex, co = [], [], [], [], [], []
    o = 0
    for (ll, c, e, cf) in shells:
        e = list(map(float, e)); cf = list(map(float, cf))
        assert len(e) == len(cf) and len(e) > 0
        l.append(int(ll)); npr.append(len(e)); off.append(o); cen.append(list(map(float, c)))
        ex.extend(e); co.extend(cf); o += len(e)
    return Basis(np.array(l, np.int32), np.array(npr, np.int32), np.array(off, np.int32),
                 np.array(cen, np.float64).reshape(-1, 3), np.array(ex, np.float64),
                 np.array(co, np.float64))


@dataclass
class Problem:
    name: str
    a: np.ndarray            # [3,3] lattice vectors as rows, Bohr
    kmesh: tuple             # Gamma-including mesh
    ao: Basis
    aux: Basis
    omega: float | None      # None: derive from gmesh and eps_lr
    gmesh: tuple | None      # None: derive from omega and eps_lr
    eps_sr: float
    eps_lr: float
    atoms: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))

    @property
    def nk(self) -> int:
        return int(np.prod(self.kmesh))


def even_tempered(l: int, center, alpha0: float, beta: float, n: int):
    return [(l, center, [alpha0 * beta ** i], [1.0]) for i in range(n)]


def fcc_cell(a: float) -> np.ndarray:
    return 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])


def _random_ao_atom(rng, center, spec=((0, (3, 2, 1)), (1, (2, 1)), (2, (1,))),
                    lo=0.1, hi=7000.0):
    shells = []
    for l, nprims in spec:
        for npr in nprims:
            e = np.sort(np.exp(rng.uniform(np.log(lo), np.log(hi), size=npr)))[::-1]
            c = rng.uniform(0.2, 1.0, size=npr)
            shells.append((l, center, e, c))
    return shells


def _etb_atom(center, counts=(8, 5, 2, 1), alpha0=0.2, beta=2.0):
    shells = []
    for l, n in enumerate(counts):
        shells += even_tempered(l, center, alpha0, beta, n)
    return shells


def config1() -> Problem:
    """Gamma-only cubic cell a = 4.0 Bohr, atoms at (0,0,0) and (2,2,2);
    per atom uncontracted AO s {13.0, 1.96, 0.44} and p {0.8}; aux s, p, d
    even-tempered 0.2*2.5^n, n = 0..5; omega = 0.5; eps = 1e-10."""
    a = 4.0 * np.eye(3)
    atoms = np.array([[0.0, 0.0, 0.0], [2.0, 2.0, 2.0]])
    ao, aux = [], []
    for c in atoms:
        for e in (13.0, 1.96, 0.44):
            ao.append((0, c, [e], [1.0]))
        ao.append((1, c, [0.8], [1.0]))
        for l in range(3):
            aux += even_tempered(l, c, 0.2, 2.5, 6)
    return Problem("cubic a=4.0 2-atom Gamma (12 AO, 120 aux)", a, (1, 1, 1), make_basis(ao),
                   make_basis(aux), 0.5, None, 1e-10, 1e-10, atoms)


def config2(kmesh=(2, 2, 2), seed_offset=2) -> Problem:
    """FCC two-atom cell a = 6.74 Bohr; per atom 3s2p1d AO shells with
    log-uniform random exponents in [0.1, 7000] and random contraction
    coefficients in [0.2, 1]; even-tempered aux (beta = 2, from 0.2) s x8,
    p x5, d x2, f x1 per atom; eps = 1e-8; G mesh 7^3, omega from the LR cutoff."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    A = 6.74
    a = fcc_cell(A)
    atoms = np.array([[0.0, 0.0, 0.0], [A / 4, A / 4, A / 4]])
    ao, aux = [], []
    for c in atoms:
        ao += _random_ao_atom(rng, c)
        aux += _etb_atom(c)
    name = "FCC a=6.74 2-atom k=%dx%dx%d (30 AO, 90 aux)" % tuple(kmesh)
    return Problem(name, a, tuple(kmesh), make_basis(ao), make_basis(aux), None, (7, 7, 7),
                   1e-8, 1e-8, atoms)


def config3(kmesh=(4, 4, 4)) -> Problem:
    p = config2(kmesh, seed_offset=2)
    p.name = p.name.replace("k=", "mixed k=")
    return p


def config5() -> Problem:
    """Rocksalt conventional cubic cell a = 8.0 Bohr, 8 atoms, 4x4x4 mesh;
    every atom draws its AO shells like the FCC two-atom cell (3s2p1d) and
    carries the same ETB aux."""
    rng = np.random.default_rng(SEED_BASE + 5)
    A = 8.0
    a = A * np.eye(3)
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]]) * A
    atoms = np.concatenate([fcc, fcc + np.array([A / 2, 0, 0])])
    ao, aux = [], []
    for c in atoms:
        ao += _random_ao_atom(rng, c)
        aux += _etb_atom(c)
    return Problem("rocksalt a=8.0 8-atom k=4x4x4 (120 AO, 360 aux)", a, (4, 4, 4),
                   make_basis(ao), make_basis(aux), None, (7, 7, 7), 1e-8, 1e-8, atoms)


def config4(ncell=32) -> list:
    """32 heterogeneous cells: 1-8 atoms at random positions (at most one
    per 40 Bohr^3, at least 1.5 Bohr apart), cubic or FCC lattices with a in
    U[5, 10] Bohr; per atom 2-4 random AO shells (an s
    shell plus shells of random l <= 3, 1-2 primitives, exponents
    log-uniform in [0.15, 50]); an ETB aux set (from 0.25, beta 2.0, l <= 3)
    of about 3x the AO count; k-meshes from 1x1x1 to 3x3x3.  The batched j3c
    covers the diagonal k pairs (k, k) of each cell."""
    rng = np.random.default_rng(SEED_BASE + 4)
    probs = []
    for ic in range(ncell):
        natm = int(rng.integers(1, 9))
        A = float(rng.uniform(5.0, 10.0))
        fcc = bool(rng.integers(0, 2))
        a = fcc_cell(A) if fcc else A * np.eye(3)
        # at least 40 Bohr^3 per atom (solid-state densities) and 1.5 Bohr
        # between atoms, periodic images included
        natm = max(1, min(natm, int(abs(np.linalg.det(a)) // 40.0)))
        atoms = []
        img = np.array([(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)]) @ a
        while len(atoms) < natm:
            c = rng.uniform(0, 1, size=3) @ a
            if all(np.min(np.linalg.norm(c - (b + img), axis=1)) >= 1.5 for b in atoms):
                atoms.append(c)
        atoms = np.array(atoms)
        ao, aux = [], []
        for c in atoms:
            nsh = int(rng.integers(2, 5))
            ls = [0] + [int(rng.integers(0, 4)) for _ in range(nsh - 1)]
            spec = tuple((l, (int(rng.integers(1, 3)),)) for l in sorted(ls))
            ao += _random_ao_atom(rng, c, spec=spec, lo=0.15, hi=50.0)
        nao = sum((s_[0] + 1) * (s_[0] + 2) // 2 for s_ in ao)
        per_atom = max(1, int(round(3 * nao / natm)))
        for c in atoms:
            counts = [0, 0, 0, 0]
            tot, l = 0, 0
            while tot < per_atom:
                counts[l] += 1
                tot += (l + 1) * (l + 2) // 2
                l = (l + 1) % 4
            aux += _etb_atom(c, counts=tuple(counts), alpha0=0.25, beta=2.0)
        n = int(rng.integers(1, 4))
        probs.append(Problem("batch cell %d" % ic, a, (n, n, n), make_basis(ao), make_basis(aux),
                             None, (7, 7, 7), 1e-8, 1e-8, atoms))
    return probs


def kpairs_diag(nk: int) -> np.ndarray:
    return np.array([(i, i) for i in range(nk)], dtype=np.int32)


def tiny(kmesh=(1, 1, 1), lmax_ao=1, lmax_aux=2, seed=7, a=3.2, natm=1) -> Problem:
    """A tiny cubic cell for brute-force checks: few compact shells."""
    rng = np.random.default_rng(SEED_BASE + 100 + seed)
    cell = a * np.eye(3)
    atoms = rng.uniform(0, a, size=(natm, 3))
    ao, aux = [], []
    for c in atoms:
        for l in range(lmax_ao + 1):
            npr = 2 if l == 0 else 1
            e = np.sort(rng.uniform(0.8, 4.0, size=npr))[::-1]
            ao.append((l, c, e, rng.uniform(0.3, 1.0, size=npr)))
        for l in range(lmax_aux + 1):
            aux.append((l, c, [float(rng.uniform(1.0, 3.0))], [1.0]))
    return Problem("tiny", cell, tuple(kmesh), make_basis(ao), make_basis(aux), 0.9, None,
                   1e-12, 1e-12, atoms)


def kpairs_all(nk: int) -> np.ndarray:
    return np.array([(i, j) for i in range(nk) for j in range(nk)], dtype=np.int32)


def _mesh_neg(k: int, kmesh) -> int:
    n1, n2 = kmesh[1], kmesh[2]
    a = (k // (n1 * n2), (k // n2) % n1, k % n2)
    return ((-a[0]) % kmesh[0] * n1 + (-a[1]) % n1) * n2 + (-a[2]) % n2


def df_synthetic(kmesh=(2, 1, 1), naux=24, nao=6, nocc=2, seed=0, cond=1e-7, rank=None):
    """Seeded inputs of the density-fitting consumers: per k a Hermitian metric
    J^k = Q diag(lam) Q^H (Q random unitary, real at k = -k; J^{-k} = conj(J^k))
    with lam log-spaced from 1 down to cond, or, with rank < naux, the last
    naux - rank eigenvalues exactly zero (a linearly dependent aux set); a
    random complex j3c tensor V over every k pair ([nk*nk][naux][nao][nao],
    pairs in kpairs_all order); closed-shell densities D^k = 2 C C^H with C
    random orthonormal (nao x nocc), D^{-k} = conj(D^k)."""
    rng = np.random.default_rng(SEED_BASE + 300 + seed)
    nk = int(np.prod(kmesh))
    J = np.zeros((nk, naux, naux), dtype=np.complex128)
    D = np.zeros((nk, nao, nao), dtype=np.complex128)
    lam = np.logspace(0.0, np.log10(cond), naux)
    if rank is not None:
        lam[rank:] = 0.0
    done = [False] * nk
    for k in range(nk):
        if done[k]:
            continue
        kn = _mesh_neg(k, kmesh)
        X = rng.normal(size=(naux, naux)) + (1j * rng.normal(size=(naux, naux)) if kn != k else 0.0)
        Q, _ = np.linalg.qr(X)
        M = (Q * lam) @ Q.conj().T
        J[k] = 0.5 * (M + M.conj().T)
        C0 = rng.normal(size=(nao, nocc)) + (1j * rng.normal(size=(nao, nocc)) if kn != k else 0.0)
        C, _ = np.linalg.qr(C0)
        M = 2.0 * C @ C.conj().T
        D[k] = 0.5 * (M + M.conj().T)
        J[kn], D[kn] = np.conj(J[k]), np.conj(D[k])
        done[k] = done[kn] = True
    V = rng.normal(size=(nk * nk, naux, nao, nao)) + 1j * rng.normal(size=(nk * nk, naux, nao, nao))
    return J, V, D
