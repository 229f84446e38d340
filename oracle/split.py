"""Plain FP64 reference of the compact/diffuse split of j3c (test infrastructure).

TEST INFRASTRUCTURE ONLY (tests, smoke check, bench CPU leg).  The paper (its
compact/diffuse paragraph, Fig. 1 and Eq. VPmunu_FT) splits the primitive
Gaussians of both bases at an exponent alpha_cut into compact (C/c) and
diffuse (D/d) sets.  Of the six integral types (aux C or D) x (pair cc, cd or
dd), the four with a diffuse aux function or a dd pair are evaluated entirely
in reciprocal space with the plain Coulomb kernel (Eq. VPmunu_FT, q = 0
removed) on the plane-wave box of the long-range part; only (C|cc) and (C|cd)
go through the range separation.

The paper picks, per box, the largest omega and alpha_cut that keep every
integral at the target precision; it gives no formula.  Reading used here:
the slowest-decaying factor of a reciprocal-space type is the transform of a
dd pair density, e^{-q^2 / 4(a_mu + a_nu)}, and the box of the long-range
part ends where e^{-q^2/4 omega^2} reaches eps, so dd pairs converge on that
box when a_mu + a_nu <= omega^2: alpha_cut = omega^2 / 2 (a diffuse aux
function alone, with e^{-q^2/4 a_P}, would allow a_P <= omega^2).

This module evaluates the split route by brute force: contracted shells are
cut into a compact and a diffuse sub-shell (the function is linear in its
primitives; each sub-shell is renormalised by the oracle, so its weight in
the parent is the ratio of the normalised coefficients of any one of its
primitives), every sub-shell triple is computed by route R1 (range separated)
and by route R2 (plain kernel on the given box), each block takes the route of
its type, and the sub-shells are summed back into the parent functions.

Pins: tests/test_oracle_split.py (recombination reproduces the unsplit
tensor; the split on the long-range box is as accurate as the range-separated
route on that box against converged sums, and a cutoff past the reading is
not).
"""
from __future__ import annotations

import numpy as np

import oracle


class _Basis:
    """A shell list with the attributes the oracle reads."""

    def __init__(self, l, nprim, center, exps, coeffs):
        self.l = np.asarray(l, dtype=np.int32)
        self.nprim = np.asarray(nprim, dtype=np.int32)
        self.prim_off = np.concatenate([[0], np.cumsum(self.nprim)[:-1]]).astype(np.int32)
        self.center = np.asarray(center, dtype=np.float64).reshape(-1, 3)
        self.exps = np.asarray(exps, dtype=np.float64)
        self.coeffs = np.asarray(coeffs, dtype=np.float64)
        self.nfunc = int(sum((int(x) + 1) * (int(x) + 2) // 2 for x in self.l))


def alpha_cut(omega: float) -> float:
    """The reading of the header: dd pairs converge on the long-range box."""
    return 0.5 * omega * omega


def split_basis(b, acut: float):
    """(sub-basis, R, kind): R [parent functions][sub functions] holds each
    sub-function's weight in its parent function; kind[j] is 'c' or 'd' per
    sub function (a primitive with exponent > acut is compact)."""
    l, nprim = np.asarray(b.l), np.asarray(b.nprim)
    po = np.asarray(b.prim_off)
    cen = np.asarray(b.center, dtype=np.float64).reshape(-1, 3)
    ex, co = np.asarray(b.exps, dtype=np.float64), np.asarray(b.coeffs, dtype=np.float64)
    subs = []   # (parent shell, kind, primitive indices)
    for s in range(len(l)):
        idx = np.arange(po[s], po[s] + nprim[s])
        for kind, m in (("c", ex[idx] > acut), ("d", ex[idx] <= acut)):
            if m.any():
                subs.append((s, kind, idx[m]))
    sb = _Basis([l[s] for s, _, _ in subs], [len(i) for _, _, i in subs], [cen[s] for s, _, _ in subs],
                np.concatenate([ex[i] for _, _, i in subs]), np.concatenate([co[i] for _, _, i in subs]))
    cn_full, cn_sub = oracle.norm_coeffs(b), oracle.norm_coeffs(sb)
    nc = lambda x: (int(x) + 1) * (int(x) + 2) // 2
    pf0 = np.concatenate([[0], np.cumsum([nc(x) for x in l])]).astype(int)
    R = np.zeros((b.nfunc if hasattr(b, "nfunc") else int(pf0[-1]), sb.nfunc))
    kind = []
    j0, p0 = 0, 0
    for (s, k, idx) in subs:
        w = cn_full[idx[0]] / cn_sub[p0]
        for c in range(nc(l[s])):
            R[pf0[s] + c, j0 + c] = w
            kind.append(k)
        j0 += nc(l[s])
        p0 += len(idx)
    return sb, R, np.array(kind)


def recombine(Vs, Rx, Ra):
    """V[pair][P][mu][nu] of the parent bases from the sub-basis tensor."""
    return np.einsum("Pp,ipmn,Mm,Nn->iPMN", Rx, Vs, Ra, Ra, optimize=True)


def j3c_split(cell_a, kmesh, ao, aux, omega, kpairs, gmesh, *, acut=None, eps_sr=1e-10, eps_lr=1e-10):
    """V by the split route: (C|cc), (C|cd) range separated (SR + G0 + LR on
    ``gmesh``), the other four types with the plain kernel on the same box."""
    acut = alpha_cut(omega) if acut is None else acut
    sa, Ra, ka = split_basis(ao, acut)
    sx, Rx, kx = split_basis(aux, acut)
    v_rs = oracle.j3c(cell_a, kmesh, sa, sx, omega, kpairs, eps_sr=eps_sr, eps_lr=eps_lr, gmesh=gmesh)
    v_g = oracle.j3c_fullG(cell_a, kmesh, sa, sx, kpairs, gmesh, eps_lr=1e-14)
    dd = (ka[:, None] == "d") & (ka[None, :] == "d")
    rs = (kx[:, None, None] == "c") & ~dd[None, :, :]
    return recombine(np.where(rs[None], v_rs, v_g), Rx, Ra)
