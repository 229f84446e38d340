"""Host checks of the HF-energy error proxy: invariance of the fitted
energies under a change of aux basis (V -> T V, J -> T J T^H; a factor
applied on the wrong side or a missing conjugate breaks it), signs
(E_J >= 0, E_K <= 0 for a PSD density), quadratic scaling, the k-symmetry of
the synthetic density, a zero error for identical tensors, and the removal
of an exactly linearly dependent aux function."""
import numpy as np

from paper_2102_02989_gb300 import hfproxy, inputs


def _problem(kmesh, naux=5, nao=4, seed=0):
    rng = np.random.default_rng(seed)
    nk = int(np.prod(kmesh))
    kp = np.array([(i, j) for i in range(nk) for j in range(nk)], np.int32)
    V = rng.normal(size=(len(kp), naux, nao, nao)) + 1j * rng.normal(size=(len(kp), naux, nao, nao))
    J = []
    for _ in range(nk):
        A = rng.normal(size=(naux, naux)) + 1j * rng.normal(size=(naux, naux))
        J.append(A @ A.conj().T + naux * np.eye(naux))
    return kp, V, np.array(J)


def test_aux_basis_invariance():
    km = (2, 1, 2)
    kp, V, J = _problem(km)
    rng = np.random.default_rng(4)
    D = hfproxy.densities(km, V.shape[-1], 2, seed=1)
    e0 = hfproxy.energies(V, kp, km, hfproxy.fit_transforms(J, 0.0), D)
    # the Cholesky inverse is another fitting transform of the same metric
    e0c = hfproxy.energies(V, kp, km, [np.linalg.inv(np.linalg.cholesky(Jk)) for Jk in J], D)
    assert np.allclose(e0, e0c, rtol=1e-10, atol=1e-12)
    # a k12-dependent invertible change of the aux basis
    nk = len(J)
    T = [rng.normal(size=J.shape[1:]) + 1j * rng.normal(size=J.shape[1:]) + 3 * np.eye(J.shape[1]) for _ in range(nk)]
    V2 = np.array([np.einsum("pq,qmn->pmn", T[hfproxy.k12(a, b, km)], V[i]) for i, (a, b) in enumerate(kp)])
    J2 = np.array([T[k] @ J[k] @ T[k].conj().T for k in range(nk)])
    e1 = hfproxy.energies(V2, kp, km, hfproxy.fit_transforms(J2, 0.0), D)
    assert np.allclose(e0, e1, rtol=1e-10, atol=1e-12)


def test_signs_scaling_and_zero_error():
    km = (2, 2, 1)
    kp, V, J = _problem(km, seed=3)
    W = hfproxy.fit_transforms(J)
    D = hfproxy.densities(km, V.shape[-1], 2, seed=2)
    ej, ek = hfproxy.energies(V, kp, km, W, D)
    assert ej >= 0 and ek <= 0
    ej2, ek2 = hfproxy.energies(2.0 * V, kp, km, W, D)
    assert abs(ej2 - 4 * ej) < 1e-10 * abs(ej) and abs(ek2 - 4 * ek) < 1e-10 * abs(ek)
    assert hfproxy.energy_error(V, V, kp, km, J)["dE"] == 0.0


def test_linear_dependence_dropped():
    """A duplicated aux function makes J singular; the thresholded transform
    drops the null direction and the energies equal those without the copy."""
    km = (1, 1, 1)
    kp, V, J = _problem(km, naux=4, seed=7)
    V2 = np.concatenate([V, V[:, :1]], axis=1)
    J2 = np.zeros((1, 5, 5), complex)
    J2[0, :4, :4] = J[0]
    J2[0, 4, :4] = J[0, 0]
    J2[0, :4, 4] = J[0, :, 0]
    J2[0, 4, 4] = J[0, 0, 0]
    D = hfproxy.densities(km, V.shape[-1], 2, seed=3)
    e = hfproxy.energies(V, kp, km, hfproxy.fit_transforms(J), D)
    e2 = hfproxy.energies(V2, kp, km, hfproxy.fit_transforms(J2), D)
    assert np.allclose(e, e2, rtol=1e-8)


def test_density_k_symmetry():
    km = (3, 2, 1)
    D = hfproxy.densities(km, 6, 2, seed=5)
    for k in range(6):
        assert np.allclose(D[hfproxy.kneg(k, km)], np.conj(D[k]))
        assert np.allclose(D[k], D[k].conj().T)
        assert abs(np.trace(D[k]).real - 4.0) < 1e-12
        assert np.min(np.linalg.eigvalsh(D[k])) > -1e-12
    assert hfproxy.k12(1, 0, km) == hfproxy.kneg(1, km)


def test_energies_equal_the_df_oracle_jk():
    """The proxy's energies (eigen-route fit, energies from B directly) equal
    those of the DF oracle's J/K matrices on the same tensors and metric."""
    from oracle import dfjk
    kmesh = (2, 2, 1)
    J, V, D = inputs.df_synthetic(kmesh, naux=14, nao=5, nocc=2, cond=1e-4, seed=90)
    kp = inputs.kpairs_all(4)
    ej, ek = hfproxy.energies(V, kp, kmesh, hfproxy.fit_transforms(J, 1e-6), D)
    T, _, _, _ = dfjk.metric_transforms(J, "eigen", rel=1e-6)
    Jm, Km, _ = dfjk.jk(dfjk.fit(T, V, kp, kmesh), kp, kmesh, D)
    oj, ok = dfjk.energies(Jm, Km, D)
    assert abs(ej - oj) < 1e-10 * abs(oj) and abs(ek - ok) < 1e-10 * abs(ok)
