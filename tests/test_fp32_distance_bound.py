"""The error bound behind the SR kernel's FP32 distance test (CPU only).

The kernel decides Rc <= Rc_cut and the window floor(Rc / DR) of a candidate
translation from the FP32 squared distance r2f = |fl(h) - fl(l')|^2 whenever the
interval [r2f - e2f, r2f + e2f] leaves no doubt, with

    e2f = 8 u fcut (|h| + lim + fcut),   lim = fcut + |h| + 1e-3,   u = 2^-24,

twice the derived bound 4 u fcut (|h| + lim) + 3 u fcut^2 (each component carries
at most 2u(|h_x| + |l'_x|)(1 + u) of rounding from fl(h), fl(l') and the
difference; the sum of squares adds 3u r2).  These tests emulate the kernel's
FP32 arithmetic (with and without fused multiply-adds in the sum of squares) on
candidates that pass its pre-filter and check that the exact squared distance
never leaves [r2f - e2f/2, r2f + e2f/2], and that the pre-filter margin of the
candidate radius (fcut = rcut + 1e-3) exceeds the same error."""
import numpy as np

U = 2.0 ** -24


def _f32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def _fma32(a, b, c):
    # a*b is exact in FP64 for FP32 a, b; one rounding of the sum to FP32
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _cases(rng, n, rcut, hmax):
    h = rng.uniform(-1, 1, size=(n, 3)) * (hmax / np.sqrt(3))
    d = rng.normal(size=(n, 3))
    d *= (rng.uniform(0, 1, size=(n, 1)) ** (1 / 3) * (rcut + 1e-3)) / np.linalg.norm(d, axis=1, keepdims=True)
    lp = h - d                        # candidate lattice vectors with |h - l'| <= fcut
    # round l' to a few decimals of a lattice-like grid: the kernel's l' come from FP64 vectors
    return h, np.round(lp, 9)


def _kernel_r2f(h, lp, fused):
    fx, fy, fz = (_f32(h[:, i]) for i in range(3))
    lx, ly, lz = (_f32(lp[:, i]) for i in range(3))
    ex, ey, ez = fx - lx, fy - ly, fz - lz          # FP32 differences
    if fused:
        return _fma32(ez, ez, _fma32(ey, ey, ex * ex))
    return (ex * ex + ey * ey) + ez * ez


def _e2f(h, rcut):
    fcut = np.float32(rcut) + np.float32(1e-3)
    hf = np.sqrt(np.sum(_f32(h).astype(np.float64) ** 2, axis=1))
    return 8.0 * U * fcut * (hf + fcut + 1e-3 + hf + fcut), fcut


def test_fp32_squared_distance_within_half_the_kernel_margin():
    rng = np.random.default_rng(7)
    for rcut, hmax in ((2.0, 3.0), (15.0, 6.0), (40.0, 10.0), (120.0, 20.0)):
        h, lp = _cases(rng, 200000, rcut, hmax)
        exact = np.sum((h - lp) ** 2, axis=1)
        e2f, _ = _e2f(h, rcut)
        for fused in (False, True):
            r2f = _kernel_r2f(h, lp, fused).astype(np.float64)
            worst = np.max(np.abs(r2f - exact) / (0.5 * e2f))
            assert worst <= 1.0, (rcut, hmax, fused, worst)


def test_prefilter_margin_exceeds_the_rounding():
    # a translation with Rc <= rcut must pass the FP32 pre-filter r2f <= fcut^2
    rng = np.random.default_rng(8)
    for rcut, hmax in ((1.0, 3.0), (15.0, 6.0), (60.0, 12.0)):
        h, lp = _cases(rng, 200000, rcut, hmax)
        d = h - lp
        d *= (rcut / np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-300))   # exactly on the radius
        lp = h - d
        _, fcut = _e2f(h, rcut)
        for fused in (False, True):
            r2f = _kernel_r2f(h, lp, fused)
            assert np.all(r2f <= fcut * fcut), (rcut, fused)
