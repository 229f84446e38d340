"""Device-side error paths in the forms that fault no GPU:

- a bounded device wait that runs out: the self-test CTA waits, with the
  same bounded poll as the tensor-core contraction, on a barrier nothing
  arrives at; the kernel returns, rsgdf_sync_status reports RSGDF_ETIMEOUT,
  and the device stays usable (a j3c afterwards still matches the oracle);
- a scratch budget too small for the call: RSGDF_ENOMEM, as when the device
  allocator fails, and the next call with the budget lifted is correct."""
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


def small_case():
    km = (2, 1, 1)
    p = inputs.tiny(kmesh=km, lmax_ao=1, lmax_aux=2, natm=2, seed=3)
    return p, km, inputs.kpairs_all(2)


def test_bounded_wait_gives_up_and_reports(rs, orc):
    rs.rsgdf_sync_status()
    rs.rsgdf_selftest_wait(True, 1000)      # control: the barrier completes
    rs.rsgdf_sync_status()
    rs.rsgdf_selftest_wait(False, 2000)     # nothing arrives: the wait runs out
    with pytest.raises(rs.RsgdfError) as e:
        rs.rsgdf_sync_status()
    assert e.value.code == rs.RSGDF_ETIMEOUT
    rs.rsgdf_sync_status()                  # the flag was cleared by the report
    # the context is still usable and correct
    p, km, kp = small_case()
    w, gm = rs.rsgdf_params(p.a, km, omega=0.9, eps_lr=1e-13)
    got = rs.rsgdf_j3c(p.a, km, p.ao, p.aux, kp, omega=w, gmesh=gm, eps_screen=1e-12, eps_lr=1e-13)
    rs.rsgdf_sync_status()
    ref = orc.j3c(p.a, km, p.ao, p.aux, w, kp, eps_sr=1e-12, eps_lr=1e-13, gmesh=gm)
    assert np.max(np.abs(got.cpu().numpy() - ref)) < 1e-10


@pytest.mark.parametrize("limit", [1024, 1 << 16])
def test_scratch_budget_reports_enomem(rs, orc, limit):
    p, km, kp = small_case()
    w, gm = rs.rsgdf_params(p.a, km, omega=0.9, eps_lr=1e-13)
    opt = dict(omega=w, gmesh=gm, eps_screen=1e-12, eps_lr=1e-13)
    rs.rsgdf_set_scratch_limit(limit)
    try:
        with pytest.raises(rs.RsgdfError) as e:
            rs.rsgdf_j3c(p.a, km, p.ao, p.aux, kp, **opt)
        assert e.value.code == rs.RSGDF_ENOMEM
        assert "limit" in rs.rsgdf_last_error()
    finally:
        rs.rsgdf_set_scratch_limit(0)
    rs.rsgdf_sync_status()
    got = rs.rsgdf_j3c(p.a, km, p.ao, p.aux, kp, **opt)
    rs.rsgdf_sync_status()
    ref = orc.j3c(p.a, km, p.ao, p.aux, w, kp, eps_sr=1e-12, eps_lr=1e-13, gmesh=gm)
    assert np.max(np.abs(got.cpu().numpy() - ref)) < 1e-10
