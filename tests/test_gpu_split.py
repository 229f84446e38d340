"""The compact/diffuse split route on the GPU (cdsplit.j3c_split: split bases,
range-separated j3c restricted to (C|cc)/(C|cd), plain-kernel G sum, combine)
against the oracle's split route (oracle/split.py) on a cell whose primitives
straddle the cut, and against converged sums: no less accurate than the plain
range-separated route on the same box.  FP64; parity tolerance 1e-10 (the same
screening thresholds and box on both sides)."""
import numpy as np
import pytest

from oracle import split
from paper_2102_02989_gb300 import inputs
from rules_ref import gmesh_for

pytestmark = pytest.mark.gpu
A = 4.0 * np.eye(3)
C1, C2 = np.zeros(3), np.array([1.7, 2.1, 1.9])
KM = (2, 1, 1)
W = 0.9


@pytest.fixture(scope="module")
def rs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    return rsgdf


def _bases():
    ao = inputs.make_basis([(0, C1, [3.0, 0.3], [0.6, 0.5]), (1, C1, [0.25], [1.0]), (0, C2, [12.0], [1.0]),
                            (0, C2, [0.7], [1.0]), (1, C1, [0.75], [1.0]), (1, C2, [2.2, 0.35], [0.7, 0.4])])
    aux = inputs.make_basis([(0, C1, [25.0], [1.0]), (0, C1, [0.3], [1.0]), (1, C2, [0.5], [1.0]),
                             (2, C2, [0.2], [1.0]), (2, C1, [1.2], [1.0])])
    return ao, aux


def test_split_route_parity_and_accuracy(rs, orc):
    from paper_2102_02989_gb300 import cdsplit
    ao, aux = _bases()
    kp = inputs.kpairs_all(2)
    gm = gmesh_for(A, W, 1e-8, KM)
    ref_split = split.j3c_split(A, KM, ao, aux, W, kp, gm, eps_sr=1e-12, eps_lr=1e-14)
    got = cdsplit.j3c_split(A, KM, ao, aux, kp, omega=W, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14).cpu().numpy()
    assert np.max(np.abs(got - ref_split)) < 1e-10
    conv = orc.j3c(A, KM, ao, aux, W, kp, eps_sr=1e-14, eps_lr=1e-15, gmesh=gmesh_for(A, W, 1e-15, KM))
    plain = rs.rsgdf_j3c(A, KM, ao, aux, kp, omega=W, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14).cpu().numpy()
    assert np.max(np.abs(got - conv)) <= np.max(np.abs(plain - conv)) + 1e-9


def test_plain_kernel_lr_equals_the_full_reciprocal_sum(rs, orc):
    """rsgdf_j3c_lr with the plain kernel is route R2 on the given box."""
    ao, aux = _bases()
    kp = inputs.kpairs_all(2)
    gm = gmesh_for(A, W, 1e-8, KM)
    ref = orc.j3c_fullG(A, KM, ao, aux, kp, gm, eps_lr=1e-14)
    got = rs.rsgdf_j3c_lr(A, KM, ao, aux, kp, omega=W, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14,
                          kernel=rs.RSGDF_KERNEL_PLAIN).cpu().numpy()
    assert np.max(np.abs(got - ref)) < 1e-10


MIXED_REL = 1e-6   # stated bound of the mixed path: whole j3c within 1e-6 of max |V| of the oracle


def test_mixed_split_route_within_the_stated_bound(rs, orc):
    """The split route in the mixed path (split-TF32 tensor-core G sums for both
    the erf and the plain kernel, double-float phase contractions, FP64 SR)
    against the oracle's FP64 split route: within the mixed path's stated
    bound, and no less accurate against converged sums than the FP64 plain
    route plus that bound."""
    from paper_2102_02989_gb300 import cdsplit
    ao, aux = _bases()
    kp = inputs.kpairs_all(2)
    gm = gmesh_for(A, W, 1e-8, KM)
    ref_split = split.j3c_split(A, KM, ao, aux, W, kp, gm, eps_sr=1e-12, eps_lr=1e-14)
    got = cdsplit.j3c_split(A, KM, ao, aux, kp, omega=W, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14,
                            precision=rs.RSGDF_MIXED).cpu().numpy()
    scale = np.max(np.abs(ref_split))
    assert scale > 0.1
    err = np.max(np.abs(got - ref_split))
    assert err < 1e-10 + MIXED_REL * scale, (err, scale)
    conv = orc.j3c(A, KM, ao, aux, W, kp, eps_sr=1e-14, eps_lr=1e-15, gmesh=gmesh_for(A, W, 1e-15, KM))
    plain = rs.rsgdf_j3c(A, KM, ao, aux, kp, omega=W, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14).cpu().numpy()
    assert np.max(np.abs(got - conv)) <= np.max(np.abs(plain - conv)) + 1e-9 + MIXED_REL * scale


def test_mixed_split_on_the_tuned_fcc_box(rs):
    """FCC a = 6.74 at 2x2x2 on the 11^3 box (the box the tuner picks for the
    mixed path), every aux shell and k pair: the mixed split route against
    the FP64 split route within the stated mixed bound (the FP64 split route
    itself is held to the oracle's split route by the small-cell test)."""
    from paper_2102_02989_gb300 import cdsplit
    p = inputs.config2((2, 2, 2))
    gm = (11, 11, 11)
    w, _ = rs.rsgdf_params(p.a, p.kmesh, gmesh=gm, eps_lr=p.eps_lr)
    kp = inputs.kpairs_all(p.nk)
    opt = dict(omega=w, gmesh=gm, eps_screen=p.eps_sr, eps_lr=p.eps_lr)
    v64 = cdsplit.j3c_split(p.a, p.kmesh, p.ao, p.aux, kp, **opt)
    vmx = cdsplit.j3c_split(p.a, p.kmesh, p.ao, p.aux, kp, precision=rs.RSGDF_MIXED, **opt)
    scale = v64.abs().max().item()
    err = (vmx - v64).abs().max().item()
    assert err < MIXED_REL * scale, (err, scale)
