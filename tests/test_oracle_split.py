"""Pins of the compact/diffuse split route (oracle/split.py) on a small cubic
cell whose AO and aux primitives straddle the cutoff (a contracted shell with
one compact and one diffuse primitive included): cutting shells into compact
and diffuse sub-shells and summing them back reproduces the unsplit tensor;
against converged sums (tight screening, box for eps_lr = 1e-15) the split
route on the long-range box is no less accurate than the range-separated route
on that box, while a cutoff 16 times the reading moves compact functions to the
plain-kernel sum, which that box cannot converge."""
import numpy as np
import pytest

from oracle import split
from paper_2102_02989_gb300 import inputs
from rules_ref import gmesh_for

A = 4.0 * np.eye(3)
C1, C2 = np.zeros(3), np.array([1.7, 2.1, 1.9])
KM = (2, 1, 1)
W = 0.9


def _bases():
    ao = inputs.make_basis([(0, C1, [3.0, 0.3], [0.6, 0.5]), (1, C1, [0.25], [1.0]), (0, C2, [12.0], [1.0]),
                            (0, C2, [0.7], [1.0]), (1, C1, [0.75], [1.0]), (1, C2, [2.2, 0.35], [0.7, 0.4])])
    aux = inputs.make_basis([(0, C1, [25.0], [1.0]), (0, C1, [0.3], [1.0]), (1, C2, [0.5], [1.0]),
                             (2, C2, [0.2], [1.0]), (2, C1, [1.2], [1.0])])
    return ao, aux


def test_sub_shells_sum_back_to_the_parent(orc):
    ao, aux = _bases()
    kp = inputs.kpairs_all(2)
    gm = gmesh_for(A, W, 1e-8, KM)
    # screening acts on primitive-pair coefficients, which the sub-shells renormalise:
    # the identity is checked with screening below rounding
    whole = orc.j3c(A, KM, ao, aux, W, kp, eps_sr=1e-15, eps_lr=1e-16, gmesh=gm)
    sa, Ra, ka = split.split_basis(ao, split.alpha_cut(W))
    sx, Rx, kx = split.split_basis(aux, split.alpha_cut(W))
    assert set(ka) == {"c", "d"} and set(kx) == {"c", "d"}
    assert sa.nfunc > ao.nfunc          # the contracted shells that straddle the cut were split
    parts = orc.j3c(A, KM, sa, sx, W, kp, eps_sr=1e-15, eps_lr=1e-16, gmesh=gm)
    got = split.recombine(parts, Rx, Ra)
    assert np.max(np.abs(got - whole)) < 1e-11 * np.max(np.abs(whole))


def test_split_route_accuracy_on_the_long_range_box(orc):
    ao, aux = _bases()
    kp = inputs.kpairs_all(2)
    gm = gmesh_for(A, W, 1e-8, KM)
    ref = orc.j3c(A, KM, ao, aux, W, kp, eps_sr=1e-14, eps_lr=1e-15, gmesh=gmesh_for(A, W, 1e-15, KM))
    rs = orc.j3c(A, KM, ao, aux, W, kp, eps_sr=1e-10, eps_lr=1e-8, gmesh=gm)
    err_rs = np.max(np.abs(rs - ref))
    sp = split.j3c_split(A, KM, ao, aux, W, kp, gm, eps_sr=1e-10, eps_lr=1e-8)
    err_sp = np.max(np.abs(sp - ref))
    assert err_sp <= err_rs + 1e-9, (err_sp, err_rs)
    bad = split.j3c_split(A, KM, ao, aux, W, kp, gm, acut=16 * split.alpha_cut(W), eps_sr=1e-10, eps_lr=1e-8)
    assert np.max(np.abs(bad - ref)) > 100 * err_rs
