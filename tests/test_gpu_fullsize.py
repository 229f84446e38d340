"""The bench workloads at full size (FCC cell, every aux shell, every k pair),
in the launch configuration bench.py times, checked against the oracle on
sampled outputs: a few aux shells (an s, a d and an f shell, whose classes
carry most of the SR work) and a few k pairs, computed by the oracle one
sample at a time at the same screening threshold.

Tolerances: FP64 path 10 eps (both sides screen at eps = 1e-8 by independent
restatements of the same rules; a term on a boundary may be kept by one side
only); mixed path the same plus the stated bound of its LR part (1e-6 of the
largest element)."""
import numpy as np
import pytest

from paper_2102_02989_gb300 import inputs
from rules_ref import omega_for

pytestmark = pytest.mark.gpu
EPS = 1e-8
MIXED_REL = 1e-6


@pytest.fixture(scope="module")
def rs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    return rsgdf


@pytest.mark.parametrize("km,mixed", [((2, 2, 2), False), ((2, 2, 2), True), ((4, 4, 4), True)])
def test_full_workload_sampled(rs, orc, km, mixed):
    import torch
    p = inputs.config2(km)
    w, gm = rs.rsgdf_params(p.a, p.kmesh, gmesh=p.gmesh, eps_lr=p.eps_lr)
    assert abs(w - omega_for(p.a, p.gmesh, p.eps_lr, p.kmesh)) < 1e-14
    kp = inputs.kpairs_all(p.nk)
    prec = rs.RSGDF_MIXED if mixed else rs.RSGDF_FP64
    V = rs.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, kp, gmesh=gm, eps_screen=EPS, eps_lr=p.eps_lr, precision=prec)
    rs.rsgdf_sync_status()
    rng = np.random.default_rng(sum(km) + 10 * mixed)
    l = np.asarray(p.aux.l)
    shells = [int(rng.choice(np.where(l == lv)[0])) for lv in (0, 2, 3)]
    pairs = sorted(set([0] + [int(x) for x in rng.choice(len(kp), 3, replace=False)]))
    for s in shells:
        f0 = int(sum((int(x) + 1) * (int(x) + 2) // 2 for x in l[:s]))
        nf = (int(l[s]) + 1) * (int(l[s]) + 2) // 2
        got = V[torch.tensor(pairs, device=V.device)][:, f0:f0 + nf].cpu().numpy()
        ref = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp[pairs], eps_sr=EPS, eps_lr=p.eps_lr, gmesh=gm,
                      shells=(s, s + 1))
        assert np.max(np.abs(ref)) > 1e-3
        tol = 10 * EPS + (MIXED_REL * np.max(np.abs(ref)) if mixed else 0.0)
        err = np.max(np.abs(got - ref))
        assert err < tol, (s, pairs, err, tol)
    del V
    torch.cuda.empty_cache()


def test_headline_learned_mixed_sampled(rs, orc):
    """The headline path as bench.py times it: learned screening (a network
    trained on the items of the cubic Gamma cell and of an FCC cell with
    another basis draw, not the timed one) together with the mixed-precision
    path, FCC 2x2x2, every aux shell and every k pair, sampled against the
    oracle.  Tolerance: the FP64 path's 10 eps, another 10 eps for the items
    the network prunes (each predicted below eps/10 behind a calibrated
    margin), plus the mixed LR bound."""
    import torch
    from paper_2102_02989_gb300 import screening
    p1 = inputs.config1()
    _, gm1 = rs.rsgdf_params(p1.a, p1.kmesh, omega=p1.omega, eps_lr=p1.eps_lr)
    pt = inputs.config2(seed_offset=12)
    wt, gmt = rs.rsgdf_params(pt.a, pt.kmesh, gmesh=pt.gmesh, eps_lr=pt.eps_lr)
    X, t = screening.items_dataset([(p1.a, p1.kmesh, p1.ao, p1.aux, p1.omega, gm1, p1.eps_lr),
                                    (pt.a, pt.kmesh, pt.ao, pt.aux, wt, gmt, pt.eps_lr)], eps_screen=EPS)
    m, _ = screening.train_screen(X, t, seed=0, eps_screen=EPS)
    p = inputs.config2((2, 2, 2))
    w, gm = rs.rsgdf_params(p.a, p.kmesh, gmesh=p.gmesh, eps_lr=p.eps_lr)
    kp = inputs.kpairs_all(p.nk)
    V = rs.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, kp, gmesh=gm, eps_screen=EPS, eps_lr=p.eps_lr,
                     precision=rs.RSGDF_MIXED, screening=rs.RSGDF_SCREEN_LEARNED, mlp=m.h)
    st = rs.rsgdf_last_stats()
    rs.rsgdf_sync_status()
    assert st["sr_items_pruned"] > 0
    rng = np.random.default_rng(29)
    l = np.asarray(p.aux.l)
    shells = [int(rng.choice(np.where(l == lv)[0])) for lv in (0, 1, 2, 3)]
    pairs = sorted(set([0] + [int(x) for x in rng.choice(len(kp), 3, replace=False)]))
    for s in shells:
        f0 = int(sum((int(x) + 1) * (int(x) + 2) // 2 for x in l[:s]))
        nf = (int(l[s]) + 1) * (int(l[s]) + 2) // 2
        got = V[torch.tensor(pairs, device=V.device)][:, f0:f0 + nf].cpu().numpy()
        ref = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp[pairs], eps_sr=EPS, eps_lr=p.eps_lr, gmesh=gm,
                      shells=(s, s + 1))
        assert np.max(np.abs(ref)) > 1e-3
        tol = 20 * EPS + MIXED_REL * np.max(np.abs(ref))
        err = np.max(np.abs(got - ref))
        assert err < tol, (s, pairs, err, tol)
    del V
    torch.cuda.empty_cache()
