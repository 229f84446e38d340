"""Density-fitting consumers on the GPU (rsgdf_df_metric, rsgdf_df_fit,
rsgdf_df_jk) against the oracle (oracle/dfjk.py), element by element where the
result is unique (the Cholesky transform, B and J/K from it, the eigenvalues,
T^H T) and through the invariant J/K matrices where it is not (eigen-route
rows carry an arbitrary phase).

Tolerances (FP64 both sides, different summation orders): 1e-10 of the largest
element for the Cholesky route, whose error grows as cond(L) eps ~ 1e3 eps
here; 1e-9 for the eigen route, where T scales as lam^{-1/2} down to the cut,
and for T J T^H = I the Jacobi stopping floor over the smallest kept eigenvalue."""
import numpy as np
import pytest

from oracle import dfjk
from paper_2102_02989_gb300 import inputs
from rules_ref import gmesh_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    return rsgdf


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.complex128)).cuda()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("naux", [1, 33, 70])
def test_cholesky_route_elementwise(rs, naux):
    J, _, _ = inputs.df_synthetic((3, 1, 1), naux=naux, nao=2, cond=1e-6, seed=10 + naux)
    T, lam, kept, info = rs.rsgdf_df_metric(_dev(J), rs.RSGDF_FIT_CHOLESKY, rel=1e-10)
    To, route, ko, piv = dfjk.metric_transforms(J, "cholesky", rel=1e-10)
    assert info.cpu().tolist() == [0] * 3 and kept.cpu().tolist() == ko == [naux] * 3
    assert _rel(T.cpu().numpy(), To) < 1e-10
    assert float(lam.abs().max()) == 0.0


@pytest.mark.parametrize("naux", [1, 33, 70, 130])   # 130: working matrix beyond shared memory
def test_eigen_route_unique_parts(rs, naux):
    J, _, _ = inputs.df_synthetic((3, 1, 1), naux=naux, nao=2, cond=1e-6, seed=20 + naux)
    T, lam, kept, info = rs.rsgdf_df_metric(_dev(J), rs.RSGDF_FIT_EIGEN, rel=1e-8)
    info = info.cpu().numpy()
    assert np.all((info >= 1) & (info <= rs.RSGDF_DF_SWEEPS)), info
    T, lam = T.cpu().numpy(), lam.cpu().numpy()
    for k in range(3):
        To, lo, ko = dfjk.transform_eigen(J[k], rel=1e-8)
        assert int(kept[k]) == ko == naux
        assert np.max(np.abs(lam[k] - lo)) < 1e-13 * lo[0]
        assert _rel(T[k].conj().T @ T[k], To.conj().T @ To) < 1e-9
        # the sweeps stop once every |a_pq| <= 1e-15 ||J||_F (or the relative test
        # passes), so T J T^H = I holds to about that over the smallest kept eigenvalue
        tol = 3e-15 * np.linalg.norm(J[k]) / lo[ko - 1] + 1e-12
        assert np.max(np.abs(T[k] @ J[k] @ T[k].conj().T - np.eye(naux))) < tol


def test_auto_falls_back_per_k_on_a_singular_metric(rs):
    naux, rank = 40, 35
    Jg, _, _ = inputs.df_synthetic((2, 1, 1), naux=naux, nao=2, cond=1e-5, seed=30)
    Js, _, _ = inputs.df_synthetic((2, 1, 1), naux=naux, nao=2, rank=rank, seed=31)
    J = np.concatenate([Jg[:1], Js[:1], Jg[1:], Js[1:]])
    T, lam, kept, info = rs.rsgdf_df_metric(_dev(J), rs.RSGDF_FIT_AUTO, rel=1e-10)
    info, kept, T = info.cpu().numpy(), kept.cpu().numpy(), T.cpu().numpy()
    To, route, ko, piv = dfjk.metric_transforms(J, "auto", rel=1e-10)
    assert route == ["cholesky", "eigen", "cholesky", "eigen"]
    assert info[0] == 0 and info[2] == 0 and 1 <= info[1] <= 40 and 1 <= info[3] <= 40
    assert kept.tolist() == ko == [naux, rank, naux, rank]
    for k in range(4):
        assert _rel(T[k].conj().T @ T[k], To[k].conj().T @ To[k]) < 1e-9
    assert _rel(T[0], To[0]) < 1e-10 and _rel(T[2], To[2]) < 1e-10
    # the Cholesky method alone reports the failing pivot and leaves T zero there
    T, lam, kept, info = rs.rsgdf_df_metric(_dev(J), rs.RSGDF_FIT_CHOLESKY, rel=1e-10)
    assert info.cpu().tolist() == [0, -1 - rank, 0, -1 - rank]
    assert kept.cpu().tolist() == [naux, 0, naux, 0]
    assert float(T[1].abs().max()) == 0.0


@pytest.mark.parametrize("kmesh,naux,nao,pairs", [((2, 2, 1), 30, 7, "all"), ((2, 1, 1), 70, 40, "some"),
                                                  ((1, 1, 1), 1, 1, "all")])
def test_fit_and_jk_elementwise(rs, kmesh, naux, nao, pairs):
    nk = int(np.prod(kmesh))
    J, V, D = inputs.df_synthetic(kmesh, naux=naux, nao=nao, nocc=max(1, nao // 3), cond=1e-5, seed=40 + nao)
    kp = inputs.kpairs_all(nk)
    if pairs == "some":
        sel = [1, 3]          # (0,1) and (1,1): k = 0 has no diagonal pair
        kp, V = kp[sel], V[sel]
    To, _, _, _ = dfjk.metric_transforms(J, "cholesky", rel=0.0)
    Bo = dfjk.fit(To, V, kp, kmesh)
    Jo, Ko, _ = dfjk.jk(Bo, kp, kmesh, D)
    T, _, _, info = rs.rsgdf_df_metric(_dev(J), rs.RSGDF_FIT_AUTO, rel=0.0)
    assert info.cpu().tolist() == [0] * nk
    a = np.eye(3) * 5.0
    B = rs.rsgdf_df_fit(a, kmesh, T, _dev(V), kp)
    assert _rel(B.cpu().numpy(), Bo) < 1e-10
    # the fit alone, from the oracle's transform
    B2 = rs.rsgdf_df_fit(a, kmesh, _dev(To), _dev(V), kp)
    assert _rel(B2.cpu().numpy(), Bo) < 1e-12
    Jm, Km = rs.rsgdf_df_jk(a, kmesh, B2, kp, _dev(D))
    Jm, Km = Jm.cpu().numpy(), Km.cpu().numpy()
    assert _rel(Km, Ko) < 1e-12
    if pairs == "some":
        assert float(np.max(np.abs(Jm[0]))) == 0.0
    assert _rel(Jm, Jo) < 1e-12
    ej, ek = dfjk.energies(Jm, Km, D)
    oj, ok = dfjk.energies(Jo, Ko, D)
    assert abs(ej - oj) < 1e-12 * abs(oj) and abs(ek - ok) < 1e-12 * abs(ok)
    # one of the two matrices alone
    Jx, Kx = rs.rsgdf_df_jk(a, kmesh, B2, kp, _dev(D), with_j=False)
    assert Jx is None and _rel(Kx.cpu().numpy(), Ko) < 1e-12


def test_eigen_route_jk_on_a_linearly_dependent_metric(rs):
    kmesh = (3, 1, 1)
    J, V, D = inputs.df_synthetic(kmesh, naux=24, nao=5, nocc=2, rank=20, seed=50)
    kp = inputs.kpairs_all(3)
    To, route, ko, _ = dfjk.metric_transforms(J, "auto", rel=1e-10)
    assert route == ["eigen"] * 3
    Jo, Ko, _ = dfjk.jk(dfjk.fit(To, V, kp, kmesh), kp, kmesh, D)
    T, _, kept, _ = rs.rsgdf_df_metric(_dev(J), rs.RSGDF_FIT_AUTO, rel=1e-10)
    assert kept.cpu().tolist() == ko
    a = np.eye(3) * 5.0
    Jm, Km = rs.rsgdf_df_jk(a, kmesh, rs.rsgdf_df_fit(a, kmesh, T, _dev(V), kp), kp, _dev(D))
    assert _rel(Jm.cpu().numpy(), Jo) < 1e-9 and _rel(Km.cpu().numpy(), Ko) < 1e-9


def test_physical_metric_needs_the_fallback(rs, orc):
    """The FCC cell's even-tempered aux metric (from the oracle's j2c) is not
    positive definite in floating point: the Cholesky route fails and the
    automatic choice takes the eigen route; fitted J/K of the oracle's j3c
    match the oracle's."""
    p = inputs.config2((2, 1, 1))
    w = 0.5
    gm = gmesh_for(p.a, w, 1e-8, p.kmesh)
    J = orc.j2c(p.a, p.kmesh, p.aux, w, [0, 1], eps_sr=1e-10, eps_lr=1e-10, gmesh=gm)
    kp = inputs.kpairs_all(2)
    V = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp, eps_sr=1e-8, eps_lr=1e-8, gmesh=gm)
    nao = V.shape[-1]
    D = inputs.df_synthetic(p.kmesh, naux=2, nao=nao, nocc=nao // 4, seed=60)[2]
    To, route, ko, piv = dfjk.metric_transforms(J, "auto", rel=1e-6)
    assert "eigen" in route
    lam0 = [np.linalg.eigvalsh(0.5 * (J[k] + J[k].conj().T))[::-1] for k in range(2)]
    for k in range(2):   # no eigenvalue within 1% of the cut
        cut = 1e-6 * lam0[k][0]
        assert np.min(np.abs(lam0[k] / cut - 1.0)) > 0.01
    Jo, Ko, _ = dfjk.jk(dfjk.fit(To, V, kp, p.kmesh), kp, p.kmesh, D)
    T, _, kept, info = rs.rsgdf_df_metric(_dev(J), rs.RSGDF_FIT_AUTO, rel=1e-6)
    info = info.cpu().numpy()
    assert [("eigen" if i >= 1 else "cholesky") for i in info] == route
    assert kept.cpu().tolist() == ko
    Jm, Km = rs.rsgdf_df_jk(p.a, p.kmesh, rs.rsgdf_df_fit(p.a, p.kmesh, T, _dev(V), kp), kp, _dev(D))
    Jm, Km = Jm.cpu().numpy(), Km.cpu().numpy()
    assert _rel(Jm, Jo) < 1e-9 and _rel(Km, Ko) < 1e-9
    ej, ek = dfjk.energies(Jm, Km, D)
    oj, ok = dfjk.energies(Jo, Ko, D)
    assert abs(ej - oj) < 1e-9 * abs(oj) and abs(ek - ok) < 1e-9 * abs(ok)


def test_jk_from_pair_shards_with_summed_rho(rs):
    """Two pair shards processed one after the other on one GPU, as two ranks
    would (rho summed, then J and K summed), equal J/K over every pair; the
    library's rho equals the oracle's."""
    from paper_2102_02989_gb300 import shard
    kmesh = (2, 2, 1)
    J, V, D = inputs.df_synthetic(kmesh, naux=30, nao=7, nocc=2, cond=1e-5, seed=80)
    kp = inputs.kpairs_all(4)
    To, _, _, _ = dfjk.metric_transforms(J, "cholesky", rel=0.0)
    Jo, Ko, rho_o = dfjk.jk(dfjk.fit(To, V, kp, kmesh), kp, kmesh, D)
    a = np.eye(3) * 5.0
    T = _dev(To)
    Dd = _dev(D)
    parts = shard.pair_shards(len(kp), 2)
    Bs = [rs.rsgdf_df_fit(a, kmesh, T, _dev(V[s]), kp[s]) for s in parts]
    rhos = [rs.rsgdf_df_rho(a, kmesh, B, kp[s], Dd) for B, s in zip(Bs, parts)]
    rho = rhos[0] + rhos[1]
    assert _rel(rho.cpu().numpy(), rho_o) < 1e-12
    out = [rs.rsgdf_df_jk(a, kmesh, B, kp[s], Dd, rho=rho) for B, s in zip(Bs, parts)]
    Jm = (out[0][0] + out[1][0]).cpu().numpy()
    Km = (out[0][1] + out[1][1]).cpu().numpy()
    assert _rel(Jm, Jo) < 1e-12 and _rel(Km, Ko) < 1e-12
