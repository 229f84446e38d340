"""Batched j3c on the GPU: one persistent SR launch per angular-momentum class
over many cells, optional CUDA-graph capture and replay, autotuned SR tiles.

The batched results are checked against the FP64 oracle (tiny cells, all k
pairs and diagonal-only pairs, 1e-10), against the single-cell calls of the
same library on the 32-cell heterogeneous workload (same arithmetic, only the
order of the atomic accumulations differs), and against the oracle on a
sample (aux shell, k pair) of two of the 32 cells."""
import numpy as np
import pytest

from paper_2102_02989_gb300 import inputs
from rules_ref import gmesh_for, omega_for

pytestmark = pytest.mark.gpu
TOL = 1e-10
SAME = 1e-11   # batched vs single-cell: atomics in another order


@pytest.fixture(scope="module")
def rs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    return rsgdf


@pytest.fixture(scope="module")
def cells():
    return inputs.config4()


def _np(t):
    return t.detach().cpu().numpy()


def _diag(p):
    return inputs.kpairs_diag(int(np.prod(p.kmesh)))


def test_batch_tiny_vs_oracle(rs, orc):
    """Three tiny cells of different meshes; the third asks only for diagonal
    pairs (X folded over the aux image cell)."""
    w, eps = 0.9, 1e-12
    ps = [inputs.tiny(kmesh=(1, 1, 1), lmax_ao=1, lmax_aux=2, natm=1, seed=3),
          inputs.tiny(kmesh=(2, 2, 1), lmax_ao=2, lmax_aux=2, natm=2, seed=8),
          inputs.tiny(kmesh=(2, 1, 2), lmax_ao=1, lmax_aux=3, natm=2, seed=5)]
    kps = [inputs.kpairs_all(1), inputs.kpairs_all(4), inputs.kpairs_diag(4)]
    outs = rs.rsgdf_j3c_batch([(p.a, p.kmesh, p.ao, p.aux) for p in ps], kps, omega=w, eps_screen=eps, eps_lr=1e-14)
    for p, kp, o in zip(ps, kps, outs):
        gm = gmesh_for(p.a, w, 1e-14, p.kmesh)
        ref = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp, eps_sr=eps, eps_lr=1e-14, gmesh=gm)
        assert np.max(np.abs(ref)) > 0.1
        assert np.max(np.abs(_np(o) - ref)) < TOL


def test_batch_equals_single_calls(rs, cells):
    """Every cell of the 32-cell batch equals the single-cell call."""
    probs = [(p.a, p.kmesh, p.ao, p.aux) for p in cells]
    kps = [_diag(p) for p in cells]
    outs = rs.rsgdf_j3c_batch(probs, kps, gmesh=(7, 7, 7), eps_screen=1e-8, eps_lr=1e-8)
    st = rs.rsgdf_last_stats()
    assert st["sr_items"] > 1000000
    for p, kp, o in zip(cells, kps, outs):
        ref = _np(rs.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, kp, gmesh=(7, 7, 7), eps_screen=1e-8, eps_lr=1e-8))
        got = _np(o)
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) < SAME * max(1.0, np.max(np.abs(ref)))
        # diagonal pairs: V^{kk}_{P nu mu} = conj V^{kk}_{P mu nu}
        assert np.max(np.abs(got - np.conj(np.swapaxes(got, 2, 3)))) < 1e-10


def test_batch_graph_and_autotune(rs, cells):
    """Graph capture + replay and the autotuned tiles reproduce the plain run;
    new output pointers are captured anew."""
    import torch
    probs = [(p.a, p.kmesh, p.ao, p.aux) for p in cells]
    kps = [_diag(p) for p in cells]
    opt = dict(gmesh=(7, 7, 7), eps_screen=1e-8, eps_lr=1e-8)
    plain = [_np(o) for o in rs.rsgdf_j3c_batch(probs, kps, **opt)]
    s = torch.cuda.Stream()
    b = rs.Batch(probs, kps, flags=rs.RSGDF_BATCH_GRAPH | rs.RSGDF_BATCH_AUTOTUNE, stream=s, **opt)
    outs = b.outputs()
    for rep in range(3):
        for o in outs:
            o.fill_(7.0)   # stale values must be overwritten
        b.run(outs, stream=s)
        s.synchronize()
        for o, r in zip(outs, plain):
            assert np.max(np.abs(_np(o) - r)) < SAME * max(1.0, np.max(np.abs(r)))
    tiles = b.tiles()
    st = rs.rsgdf_last_stats()
    assert st["n_launch"] > 32
    assert any(g > 0 for g in tiles["grid"])
    for L in range(10):
        if tiles["grid"][L]:
            assert 1 <= tiles["bc"][L] <= 16 and tiles["grab"][L] in (1, 4)
    outs2 = b.outputs()
    b.run(outs2, stream=s)
    s.synchronize()
    for o, r in zip(outs2, plain):
        assert np.max(np.abs(_np(o) - r)) < SAME * max(1.0, np.max(np.abs(r)))
    # the legacy default stream (internal capture stream, ordered by events)
    outs3 = b.outputs()
    b.run(outs3)
    torch.cuda.synchronize()
    for o, r in zip(outs3, plain):
        assert np.max(np.abs(_np(o) - r)) < SAME * max(1.0, np.max(np.abs(r)))
    b.close()


@pytest.mark.parametrize("ic", [1, 9])
def test_batch_sample_vs_oracle(rs, orc, cells, ic):
    """Full-size batch, sampled: one aux shell and two diagonal k pairs of a
    large cell against the oracle at the same screening."""
    probs = [(p.a, p.kmesh, p.ao, p.aux) for p in cells]
    kps = [_diag(p) for p in cells]
    outs = rs.rsgdf_j3c_batch(probs, kps, gmesh=(7, 7, 7), eps_screen=1e-8, eps_lr=1e-8)
    p = cells[ic]
    nk = int(np.prod(p.kmesh))
    w = omega_for(p.a, (7, 7, 7), 1e-8, p.kmesh)
    rng = np.random.default_rng(ic)
    sh = int(rng.integers(0, len(p.aux.l)))
    ks = sorted(set([0, int(rng.integers(0, nk))]))
    kp = np.array([(k, k) for k in ks], np.int32)
    ref = orc.j3c(p.a, p.kmesh, p.ao, p.aux, w, kp, eps_sr=1e-8, eps_lr=1e-8, gmesh=(7, 7, 7), shells=(sh, sh + 1))
    f0 = int(sum((l + 1) * (l + 2) // 2 for l in p.aux.l[:sh]))
    nf = (p.aux.l[sh] + 1) * (p.aux.l[sh] + 2) // 2
    got = _np(outs[ic])[ks][:, f0:f0 + nf]
    assert np.max(np.abs(ref)) > 1e-3
    # both sides screen at eps = 1e-8 by independent restatements of the same
    # rules; a term on a boundary may be kept by one side only (each <= eps)
    assert np.max(np.abs(got - ref)) < 10 * 1e-8


def test_batch_errors(rs):
    import ctypes as C
    lib = rs.load()
    h = C.c_void_p()
    o = rs._opts(gmesh=(7, 7, 7))
    rc = lib.rsgdf_j3c_batch_create(0, None, C.byref(o), None, None, 0, C.byref(h))
    assert rc == rs.RSGDF_EINVAL
    p = inputs.tiny()
    with pytest.raises(rs.RsgdfError) as e:
        rs.Batch([(p.a, p.kmesh, p.ao, p.aux)], [np.array([[0, 1]])], gmesh=(7, 7, 7))
    assert "cell 0" in str(e.value)
