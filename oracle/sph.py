"""Plain FP64 reference of the Cartesian -> real solid harmonic transform (test infrastructure).

TEST INFRASTRUCTURE ONLY (tests, smoke check, bench CPU leg).  The paper works
in spherical AO and aux bases (cc-pVDZ, GTH-DZVP); the library computes every
integral over Cartesian shells and converts afterwards.  A spherical function
of shell l, order m, is a fixed combination of the shell's Cartesian functions,
    chi_{l m} = sum_c s_{m c} chi_c ,
with s the monomial coefficients of the real regular solid harmonic (Racah
normalisation, no Condon-Shortley phase)
    C_l^m = sqrt((2 - delta_m0) (l-m)!/(l+m)!) r^l P_l^m(cos theta) cos(m phi),  m >= 0
    S_l^m = sqrt(2 (l-m)!/(l+m)!)           r^l P_l^m(cos theta) sin(m phi),  m >= 1,
ordered m = -l .. l (S_l^{|m|} for m < 0, C_l^m for m >= 0), Cartesian
components in lexicographic order.  Since a Cartesian shell carries the norm of
its x^l component and int |C_l^m|^2 dOmega = int x^{2l} dOmega = 4 pi/(2l+1),
every spherical function inherits unit norm.

Here the coefficients come from evaluating the harmonic (scipy's associated
Legendre function, its Condon-Shortley factor (-1)^m removed) at random points and
solving for the monomial coefficients of degree l by least squares; the integral
tensors transform as V^sph = s_aux (x) s_ao (x) s_ao V^cart, J^sph = s J s^T.

Pins: tests/test_oracle_sph.py (textbook forms for l <= 2, harmonicity, unit
norm and orthogonality through the oracle's own overlap integrals).
"""
from __future__ import annotations

import math

import numpy as np


def cart_components(l: int):
    """(lx, ly, lz) of a Cartesian shell in lexicographic order"""
    return [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]


def _harmonic(l: int, m: int, xyz: np.ndarray) -> np.ndarray:
    from scipy.special import lpmv
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    r = np.sqrt(x * x + y * y + z * z)
    ct = z / r
    phi = np.arctan2(y, x)
    am = abs(m)
    plm = lpmv(am, l, ct) * (-1.0) ** am          # remove the Condon-Shortley phase
    if m == 0:
        return r ** l * plm
    norm = math.sqrt(2.0 * math.factorial(l - am) / math.factorial(l + am))
    ang = np.cos(am * phi) if m > 0 else np.sin(am * phi)
    return norm * r ** l * plm * ang


def coefficients(l: int) -> np.ndarray:
    """s [2l+1][ncart]: row m + l holds the monomial coefficients of order m"""
    comps = cart_components(l)
    rng = np.random.default_rng(1234 + l)
    pts = rng.normal(size=(max(64, 8 * len(comps)), 3))
    M = np.stack([pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c for a, b, c in comps], axis=1)
    s = np.zeros((2 * l + 1, len(comps)))
    for m in range(-l, l + 1):
        s[m + l], *_ = np.linalg.lstsq(M, _harmonic(l, m, pts), rcond=None)
    return s


def basis_matrix(ls) -> np.ndarray:
    """block-diagonal transform [nsph][ncart] of a basis with shell momenta ls"""
    blocks = [coefficients(int(l)) for l in ls]
    ns = sum(b.shape[0] for b in blocks)
    nc = sum(b.shape[1] for b in blocks)
    S = np.zeros((ns, nc))
    i = j = 0
    for b in blocks:
        S[i:i + b.shape[0], j:j + b.shape[1]] = b
        i += b.shape[0]
        j += b.shape[1]
    return S


def j3c(V, ao_l, aux_l):
    """V^sph[pair][P][mu][nu] from V^cart[pair][P][mu][nu]"""
    Sa, Sx = basis_matrix(ao_l), basis_matrix(aux_l)
    return np.einsum("Pp,ipmn,Mm,Nn->iPMN", Sx, np.asarray(V), Sa, Sa, optimize=True)


def j2c(J, aux_l):
    """J^sph[k] = s J^cart[k] s^T"""
    Sx = basis_matrix(aux_l)
    return np.einsum("Pp,kpq,Qq->kPQ", Sx, np.asarray(J), Sx, optimize=True)
