"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Both sides run at the same screening threshold; FP64 results agree to 1e-10
absolute (terms that sit exactly on a screening boundary may be decided
differently by the two independent restatements of the rule; at the tight
thresholds used here such a term is below 1e-11)."""
import numpy as np
import pytest

from paper_2102_02989_gb300 import inputs
from rules_ref import gmesh_for, omega_for

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


def _np(t):
    return t.detach().cpu().numpy()


@pytest.mark.parametrize("km,lao,lax,natm", [((1, 1, 1), 1, 2, 1), ((2, 2, 1), 2, 3, 2), ((2, 1, 1), 1, 1, 1)])
def test_sr_tiny(rs, orc, km, lao, lax, natm):
    p = inputs.tiny(kmesh=km, lmax_ao=lao, lmax_aux=lax, natm=natm, seed=3)
    nk = int(np.prod(km))
    kp = inputs.kpairs_all(nk)
    w, eps = 0.9, 1e-12
    gm = gmesh_for(p.a, w, 1e-14, km)
    ref = orc.j3c(p.a, km, p.ao, p.aux, w, kp, eps_sr=eps, eps_lr=1e-14, gmesh=gm, lr=False)
    got = _np(rs.rsgdf_j3c_sr(p.a, km, p.ao, p.aux, kp, omega=w, gmesh=gm, eps_screen=eps, eps_lr=1e-14))
    assert np.max(np.abs(ref)) > 0.1
    assert np.max(np.abs(got - ref)) < TOL


@pytest.mark.parametrize("km", [(1, 1, 1), (2, 2, 1)])
def test_lr_tiny(rs, orc, km):
    p = inputs.tiny(kmesh=km, lmax_ao=2, lmax_aux=3, natm=2, seed=5)
    nk = int(np.prod(km))
    kp = inputs.kpairs_all(nk)
    w = 0.9
    gm = gmesh_for(p.a, w, 1e-14, km)
    ref = orc.j3c(p.a, km, p.ao, p.aux, w, kp, eps_lr=1e-14, gmesh=gm, sr=False, g0=False)
    import torch
    out = torch.zeros(ref.shape, dtype=torch.complex128, device="cuda")
    got = _np(rs.rsgdf_j3c_lr(p.a, km, p.ao, p.aux, kp, out=out, omega=w, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14))
    assert np.max(np.abs(got - ref)) < TOL


def test_j3c_fused_equals_parts(rs, orc):
    km = (2, 1, 2)
    p = inputs.tiny(kmesh=km, lmax_ao=2, lmax_aux=2, natm=2, seed=8)
    kp = inputs.kpairs_all(4)[::3]
    w = 1.1
    gm = gmesh_for(p.a, w, 1e-14, km)
    ref = orc.j3c(p.a, km, p.ao, p.aux, w, kp, eps_sr=1e-12, eps_lr=1e-14, gmesh=gm)
    got = _np(rs.rsgdf_j3c(p.a, km, p.ao, p.aux, kp, omega=w, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14))
    assert np.max(np.abs(got - ref)) < TOL
    sr = rs.rsgdf_j3c_sr(p.a, km, p.ao, p.aux, kp, omega=w, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14)
    both = _np(rs.rsgdf_j3c_lr(p.a, km, p.ao, p.aux, kp, out=sr, omega=w, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14))
    assert np.max(np.abs(both - got)) < 1e-12


def test_config1_subset(rs, orc):
    p = inputs.config1()
    sh = (0, 8)
    gm = gmesh_for(p.a, p.omega, p.eps_lr, p.kmesh)
    ref = orc.j3c(p.a, p.kmesh, p.ao, p.aux, p.omega, [(0, 0)], eps_sr=p.eps_sr, eps_lr=p.eps_lr, gmesh=gm, shells=sh)
    got = _np(rs.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, [(0, 0)], shells=sh, omega=p.omega, gmesh=gm,
                           eps_screen=p.eps_sr, eps_lr=p.eps_lr))
    assert np.max(np.abs(got - ref)) < TOL
    st = rs.rsgdf_last_stats()
    assert st["sr_terms"] > 0 and st["gmesh"] == gm


def test_config2_subset(rs, orc):
    p = inputs.config2()
    w = omega_for(p.a, p.gmesh, p.eps_lr, p.kmesh)
    kp = [(0, 0), (1, 6), (3, 2), (7, 7), (5, 0)]
    sh = (13, 16)      # d, d, f aux shells of the first atom: the highest L classes
    eps = 1e-11
    ref = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp, eps_sr=eps, eps_lr=p.eps_lr, gmesh=p.gmesh, shells=sh)
    got = _np(rs.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, kp, shells=sh, gmesh=p.gmesh, eps_screen=eps,
                           eps_lr=p.eps_lr))
    assert np.max(np.abs(got - ref)) < TOL


@pytest.mark.parametrize("km", [(1, 1, 1), (2, 2, 1)])
def test_j2c_and_cholesky(rs, orc, km):
    p = inputs.tiny(kmesh=km, lmax_aux=3, natm=2, seed=2)
    nk = int(np.prod(km))
    kl = list(range(nk))
    w = 0.9
    gm = gmesh_for(p.a, w, 1e-14, km)
    ref = orc.j2c(p.a, km, p.aux, w, kl, eps_sr=1e-12, eps_lr=1e-14, gmesh=gm)
    J, L, info = rs.rsgdf_j2c(p.a, km, p.aux, kl, omega=w, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14)
    J, L, info = _np(J), _np(L), _np(info)
    assert np.max(np.abs(J - ref)) < TOL
    for k in range(nk):
        Lr, piv = orc.cholesky(ref[k])
        assert piv == -1 and info[k] == -1
        assert np.max(np.abs(L[k] - Lr)) < 1e-9


def test_j2c_not_positive_definite_reports_pivot(rs):
    p = inputs.tiny(lmax_aux=1)
    aux = inputs.make_basis([(0, p.aux.center[0], [1.3], [1.0]), (0, p.aux.center[0], [1.3], [1.0])])
    J, L, info = rs.rsgdf_j2c(p.a, (1, 1, 1), aux, [0], omega=0.9, eps_screen=1e-12, eps_lr=1e-14)
    assert int(_np(info)[0]) == 1


def test_kphase_definition(rs):
    import torch
    km = (2, 3, 1)
    nk = 6
    rng = np.random.default_rng(1)
    m = 37
    X = rng.normal(size=(nk, nk, m))
    kp = inputs.kpairs_all(nk)
    got = _np(rs.rsgdf_kphase(inputs.fcc_cell(5.0), km, torch.tensor(X, device="cuda"), kp))
    # plain definition: e^{-i k12.lt} e^{+i k2.dt} with exact fractions
    n = np.array(np.unravel_index(np.arange(nk), km)).T
    ref = np.zeros((len(kp), m), dtype=complex)
    for ip, (k1, k2) in enumerate(kp):
        n12 = n[k2] - n[k1]
        for lt in range(nk):
            for dt in range(nk):
                ph = np.exp(-2j * np.pi * np.sum(n12 * n[lt] / np.array(km))) * np.exp(2j * np.pi * np.sum(n[k2] * n[dt] / np.array(km)))
                ref[ip] += ph * X[lt, dt]
    assert np.max(np.abs(got - ref)) < 1e-12


def test_invalid_arguments_rejected(rs):
    p = inputs.tiny()
    with pytest.raises(rs.RsgdfError) as e:
        rs.rsgdf_j3c(p.a, (1, 1, 1), p.ao, p.aux, [(0, 1)], omega=0.9)
    assert e.value.code == rs.RSGDF_EINVAL
    with pytest.raises(rs.RsgdfError):
        rs.rsgdf_j3c(p.a, (1, 1, 1), p.ao, p.aux, [(0, 0)], omega=0.9, gmesh=(4, 5, 5))


# ---------------------------------------------------------------------------
# Mixed-precision path (RSGDF_MIXED): split-TF32 tensor-core LR contraction.
# Bound: the 3xTF32 products carry ~22 significant bits and each 16-k chunk is
# summed in FP32 before a compensated FP32 accumulation; measured 3e-7 of
# max|V_LR| on the tiny cell (the sum over G cancels); the test bound is
# 1e-6 x max|V_LR| absolute.
# ---------------------------------------------------------------------------
MIXED_REL = 1e-6


@pytest.mark.parametrize("km,lao", [((1, 1, 1), 2), ((2, 2, 1), 2), ((2, 1, 1), 3)])
def test_lr_mixed_tensor_core(rs, orc, km, lao):
    """lao = 3 puts f shells among the AO pairs: their transforms take the
    generic kernel, the others the per-(lmu, lnu) instantiations."""
    import torch
    p = inputs.tiny(kmesh=km, lmax_ao=lao, lmax_aux=3, natm=2, seed=5)
    nk = int(np.prod(km))
    kp = inputs.kpairs_all(nk)
    w = 0.9
    gm = gmesh_for(p.a, w, 1e-14, km)
    ref = orc.j3c(p.a, km, p.ao, p.aux, w, kp, eps_lr=1e-14, gmesh=gm, sr=False, g0=False)
    out = torch.zeros(ref.shape, dtype=torch.complex128, device="cuda")
    got = _np(rs.rsgdf_j3c_lr(p.a, km, p.ao, p.aux, kp, out=out, omega=w, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14,
                              precision=rs.RSGDF_MIXED))
    rs.rsgdf_sync_status()
    scale = np.max(np.abs(ref))
    err = np.max(np.abs(got - ref))
    assert err < MIXED_REL * scale, (err, scale)
    assert err > 0.0   # really a different arithmetic


def test_config2_mixed_lr_error(rs, orc):
    p = inputs.config2()
    w = omega_for(p.a, p.gmesh, p.eps_lr, p.kmesh)
    kp = [(0, 0), (1, 6), (3, 2), (7, 7), (5, 0)]
    sh = (0, 32)
    import torch
    ref = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp, eps_lr=p.eps_lr, gmesh=p.gmesh, shells=sh, sr=False, g0=False)
    out = torch.zeros(ref.shape, dtype=torch.complex128, device="cuda")
    got = _np(rs.rsgdf_j3c_lr(p.a, p.kmesh, p.ao, p.aux, kp, shells=sh, out=out, gmesh=p.gmesh, eps_screen=1e-8,
                              eps_lr=p.eps_lr, precision=rs.RSGDF_MIXED))
    rs.rsgdf_sync_status()
    assert np.max(np.abs(got - ref)) < MIXED_REL * np.max(np.abs(ref))


def test_config2_mixed_full_all_pairs(rs, orc):
    """Mixed path end to end (FP64 SR lattice sums, double-float phase
    contractions on the FP32 pipes, split-TF32 tensor-core LR) on every k pair
    of the 2x2x2 mesh."""
    p = inputs.config2()
    w = omega_for(p.a, p.gmesh, p.eps_lr, p.kmesh)
    kp = inputs.kpairs_all(p.nk)
    sh = (14, 16)
    eps = 1e-11
    ref = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp, eps_sr=eps, eps_lr=p.eps_lr, gmesh=p.gmesh, shells=sh)
    got = _np(rs.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, kp, shells=sh, gmesh=p.gmesh, eps_screen=eps, eps_lr=p.eps_lr,
                           precision=rs.RSGDF_MIXED))
    rs.rsgdf_sync_status()
    assert np.max(np.abs(got - ref)) < MIXED_REL * np.max(np.abs(ref))
    fp = _np(rs.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, kp, shells=sh, gmesh=p.gmesh, eps_screen=eps, eps_lr=p.eps_lr))
    assert np.max(np.abs(fp - ref)) < TOL


@pytest.mark.parametrize("km,sh", [((2, 2, 2), (13, 16)), ((3, 3, 3), (0, 2))])
def test_mixed_sr_phases_fp64_grade(rs, orc, km, sh):
    """The mixed path's Bloch-phase contractions run in double-float
    arithmetic on the FP32 pipes: the SR part (FP64 lattice sums, then both
    phase steps and the G = 0 correction) stays within the FP64 parity bound."""
    p = inputs.config2(km)
    w = omega_for(p.a, p.gmesh, p.eps_lr, p.kmesh)
    kp = inputs.kpairs_all(p.nk)
    if len(kp) > 100:
        kp = kp[np.random.default_rng(1).choice(len(kp), 60, replace=False)]
    eps = 1e-11
    ref = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp, eps_sr=eps, eps_lr=p.eps_lr, gmesh=p.gmesh, shells=sh, lr=False)
    got = _np(rs.rsgdf_j3c_sr(p.a, p.kmesh, p.ao, p.aux, kp, shells=sh, gmesh=p.gmesh, eps_screen=eps,
                              eps_lr=p.eps_lr, precision=rs.RSGDF_MIXED))
    assert np.max(np.abs(ref)) > 0.1
    assert np.max(np.abs(got - ref)) < TOL


@pytest.mark.parametrize("km", [(3, 3, 2), (4, 2, 2)])
def test_phase_contractions_as_mesh_dfts(rs, orc, km):
    """With every k pair requested on a mesh of 16 or more points the phase
    contractions run as separable DFTs over the mesh axes (odd and even
    axis lengths here): SR + G0 + LR, the LR-only accumulate path and the
    mixed path against the oracle."""
    import torch
    p = inputs.tiny(kmesh=km, lmax_ao=1, lmax_aux=2, natm=2, seed=6)
    nk = int(np.prod(km))
    kp = inputs.kpairs_all(nk)
    w = 0.9
    gm = gmesh_for(p.a, w, 1e-14, km)
    opt = dict(omega=w, gmesh=gm, eps_screen=1e-12, eps_lr=1e-14)
    ref = orc.j3c(p.a, km, p.ao, p.aux, w, kp, eps_sr=1e-12, eps_lr=1e-14, gmesh=gm)
    got = _np(rs.rsgdf_j3c(p.a, km, p.ao, p.aux, kp, **opt))
    assert np.max(np.abs(ref)) > 0.1
    assert np.max(np.abs(got - ref)) < TOL
    lref = orc.j3c(p.a, km, p.ao, p.aux, w, kp, eps_lr=1e-14, gmesh=gm, sr=False, g0=False)
    out = torch.full(ref.shape, 0.5 + 0.25j, dtype=torch.complex128, device="cuda")
    lgot = _np(rs.rsgdf_j3c_lr(p.a, km, p.ao, p.aux, kp, out=out, **opt)) - (0.5 + 0.25j)
    assert np.max(np.abs(lgot - lref)) < TOL
    mix = _np(rs.rsgdf_j3c(p.a, km, p.ao, p.aux, kp, precision=rs.RSGDF_MIXED, **opt))
    rs.rsgdf_sync_status()
    assert np.max(np.abs(mix - ref)) < MIXED_REL * np.max(np.abs(ref))
    # the SR part of the mixed path (double-float DFT passes) stays FP64-grade
    sref = orc.j3c(p.a, km, p.ao, p.aux, w, kp, eps_sr=1e-12, eps_lr=1e-14, gmesh=gm, lr=False)
    smix = _np(rs.rsgdf_j3c_sr(p.a, km, p.ao, p.aux, kp, precision=rs.RSGDF_MIXED, **opt))
    assert np.max(np.abs(smix - sref)) < TOL
