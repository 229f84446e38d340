"""Cartesian -> spherical transforms on the GPU (rsgdf_cart2sph_j3c/j2c)
against the oracle (oracle/sph.py): the transform alone on the oracle's own
Cartesian tensors (element by element, 1e-13 of the largest element: a sparse
sum of at most 64 products), and the whole path, GPU j3c/j2c then the GPU
transform, against the oracle's integrals transformed by the oracle (the j3c
parity tolerance)."""
import numpy as np
import pytest

from oracle import sph
from paper_2102_02989_gb300 import inputs
from rules_ref import gmesh_for

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def rs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    return rsgdf


@pytest.fixture(scope="module")
def case(orc):
    km = (2, 1, 1)
    p = inputs.tiny(kmesh=km, lmax_ao=2, lmax_aux=3, natm=2, seed=11)
    gm = gmesh_for(p.a, p.omega, 1e-12, km)
    kp = inputs.kpairs_all(2)
    V = orc.j3c(p.a, km, p.ao, p.aux, p.omega, kp, eps_sr=1e-12, eps_lr=1e-12, gmesh=gm)
    J = orc.j2c(p.a, km, p.aux, p.omega, [0, 1], eps_sr=1e-12, eps_lr=1e-12, gmesh=gm)
    return p, km, gm, kp, V, J


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def test_transform_alone(rs, case):
    p, km, gm, kp, V, J = case
    ref = sph.j3c(V, p.ao.l, p.aux.l)
    got = rs.rsgdf_cart2sph_j3c(p.ao, p.aux, _dev(V)).cpu().numpy()
    assert got.shape == ref.shape == (4, rs.rsgdf_sph_nfunc(p.aux), rs.rsgdf_sph_nfunc(p.ao), rs.rsgdf_sph_nfunc(p.ao))
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
    refj = sph.j2c(J, p.aux.l)
    gotj = rs.rsgdf_cart2sph_j2c(p.aux, _dev(J)).cpu().numpy()
    assert np.max(np.abs(gotj - refj)) < 1e-13 * np.max(np.abs(refj))


def test_transform_of_a_shell_range(rs, case):
    p, km, gm, kp, V, J = case
    l = np.asarray(p.aux.l)
    s0, s1 = 1, len(l) - 1
    f0 = int(sum((int(x) + 1) * (int(x) + 2) // 2 for x in l[:s0]))
    f1 = int(sum((int(x) + 1) * (int(x) + 2) // 2 for x in l[:s1]))
    ref = sph.j3c(V[:, f0:f1], p.ao.l, l[s0:s1])
    got = rs.rsgdf_cart2sph_j3c(p.ao, p.aux, _dev(V[:, f0:f1]), shells=(s0, s1)).cpu().numpy()
    assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))


def test_gpu_integrals_then_transform(rs, case):
    p, km, gm, kp, V, J = case
    Vg = rs.rsgdf_j3c(p.a, km, p.ao, p.aux, kp, omega=p.omega, gmesh=gm, eps_screen=1e-12, eps_lr=1e-12)
    got = rs.rsgdf_cart2sph_j3c(p.ao, p.aux, Vg).cpu().numpy()
    assert np.max(np.abs(got - sph.j3c(V, p.ao.l, p.aux.l))) < TOL
    Jg, _, _ = rs.rsgdf_j2c(p.a, km, p.aux, [0, 1], cholesky=False, omega=p.omega, gmesh=gm, eps_screen=1e-12,
                            eps_lr=1e-12)
    gotj = rs.rsgdf_cart2sph_j2c(p.aux, Jg).cpu().numpy()
    assert np.max(np.abs(gotj - sph.j2c(J, p.aux.l))) < TOL
