"""The allocation-free k-phase entry point (rsgdf_kphase_noalloc) against the
ordinary one, through the C ABI, on two calls in a row.

Some callers cannot let a library allocate device memory while they run:
applications that own all device memory through their own pool, and
steady-state loops that must not meet an allocation failure (or an allocator
synchronisation) in the middle of a step.  The no-alloc variant serves them;
its scratch is one fixed static device array shared by every call, so a
second call must give the same answer as the first, and the device's
stream-ordered memory pool (where the library's other entry points take their
scratch) must not grow during its calls.  This file is collected last on
purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2102_02989_gb300 import inputs

pytestmark = pytest.mark.gpu
POOL_USED_MEM_CURRENT, POOL_USED_MEM_HIGH = 0x7, 0x8   # cudaMemPoolAttr


@pytest.fixture(scope="module")
def rs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    return rsgdf


class Pool:
    """The current device's default memory pool, through the CUDA runtime the
    library links against."""

    def __init__(self, lib):
        self.lib = lib
        dev = C.c_int()
        assert lib.cudaGetDevice(C.byref(dev)) == 0
        self.pool = C.c_void_p()
        assert lib.cudaDeviceGetDefaultMemPool(C.byref(self.pool), dev.value) == 0

    def get(self, attr):
        v = C.c_uint64()
        assert self.lib.cudaMemPoolGetAttribute(self.pool, attr, C.byref(v)) == 0
        return v.value

    def reset_high(self):
        z = C.c_uint64(0)
        assert self.lib.cudaMemPoolSetAttribute(self.pool, POOL_USED_MEM_HIGH, C.byref(z)) == 0


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


def test_kphase_noalloc_allocates_nothing(rs):
    import torch
    km = (2, 2, 2)
    nk, m = 8, 2048
    a = inputs.fcc_cell(6.74)
    kp = inputs.kpairs_all(nk)
    X = torch.tensor(np.random.default_rng(3).normal(size=(nk, nk, m)), device="cuda")
    out = torch.empty((len(kp), m), dtype=torch.complex128, device="cuda")
    pool = Pool(rs.load())
    rs.rsgdf_kphase_noalloc(a, km, X, kp, out)   # first call on the device: address look-up
    torch.cuda.synchronize()
    # the probe sees the ordinary entry point's scratch
    pool.reset_high()
    base = pool.get(POOL_USED_MEM_CURRENT)
    rs.rsgdf_kphase(a, km, X, kp)
    torch.cuda.synchronize()
    assert pool.get(POOL_USED_MEM_HIGH) > base
    # ... and nothing from the no-alloc variant
    torch.cuda.synchronize()
    pool.reset_high()
    base = pool.get(POOL_USED_MEM_CURRENT)
    torch_before = torch.cuda.memory_allocated()
    for _ in range(3):
        rs.rsgdf_kphase_noalloc(a, km, X, kp, out)
    torch.cuda.synchronize()
    assert pool.get(POOL_USED_MEM_HIGH) == base
    assert torch.cuda.memory_allocated() == torch_before


def test_kphase_noalloc_rejects_oversize(rs):
    import torch
    km = (2, 2, 2)
    kp = inputs.kpairs_all(8)
    # m such that 16 * Nk * m bytes exceed the 64 MiB static array
    m = (64 << 20) // (16 * 8) + 1
    big = torch.zeros((8, 8, m), dtype=torch.float64, device="cuda")
    out = torch.zeros((len(kp), m), dtype=torch.complex128, device="cuda")
    with pytest.raises(rs.RsgdfError) as e:
        rs.rsgdf_kphase_noalloc(inputs.fcc_cell(6.74), km, big, kp, out)
    assert e.value.code == rs.RSGDF_EINVAL
