"""The allocation-free k-phase entry point (rsgdf_kphase_noalloc) against the
ordinary one, through the C ABI, on two calls in a row.

Callers that cannot allocate device memory while they run (applications that
own all device memory through their own pool, steady-state loops that must not
meet an allocation failure mid-step) use the no-alloc variant; its scratch is a fixed static device array shared by every
call, so a second call must give the same answer as the first.  This file is
collected last on purpose."""
import numpy as np
import pytest

from paper_2102_02989_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    return rsgdf


def test_kphase_noalloc_matches_kphase_twice(rs):
    import torch
    km = (2, 2, 2)
    nk = 8
    rng = np.random.default_rng(17)
    a = inputs.fcc_cell(6.74)
    kp = inputs.kpairs_all(nk)
    for m in (1000, 3333):
        X = torch.tensor(rng.normal(size=(nk, nk, m)), device="cuda")
        ref = rs.rsgdf_kphase(a, km, X, kp)
        for call in range(2):
            out = torch.full((len(kp), m), complex(float("nan"), 0.0), dtype=torch.complex128, device="cuda")
            rs.rsgdf_kphase_noalloc(a, km, X, kp, out)
            torch.cuda.synchronize()
            assert torch.max(torch.abs(out - ref)).item() < 1e-12, (m, call)


def test_kphase_noalloc_rejects_oversize(rs):
    import torch
    km = (2, 2, 2)
    X = torch.zeros((8, 8, 1), dtype=torch.float64, device="cuda")
    kp = inputs.kpairs_all(8)
    # m such that 16 * Nk * m bytes exceed the 64 MiB static array
    m = (64 << 20) // (16 * 8) + 1
    big = torch.zeros((8, 8, m), dtype=torch.float64, device="cuda")
    out = torch.zeros((len(kp), m), dtype=torch.complex128, device="cuda")
    with pytest.raises(rs.RsgdfError) as e:
        rs.rsgdf_kphase_noalloc((6.74 / 2) * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0.0]]), km, big, kp, out)
    assert e.value.code == rs.RSGDF_EINVAL
    del X
