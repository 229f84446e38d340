"""Plain FP64 CPU oracle for the RSGDF j3c / j2c integrals.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports this package and this package never imports the product.  It
shares no code with the CUDA path; only the seeded input generator (which holds
none of the method's arithmetic) feeds both.

The C source (``rsgdf_oracle.c``) evaluates every integral term by term with the
McMurchie-Davidson scheme.  Route R1 is the paper's range-separated evaluation
(Eqs. Coulomb_RS, VPmunu_SR, VPmunu_LR, AFT_pairden, BvK_latsum_LR and the
screening of the Supplementary Material); route R2 is the plain reciprocal-space
definition (Eq. VPmunu_FT) on a large G box, used to check R1 on tiny cells.

Every pin of these functions lives in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "rsgdf_oracle.c")
_lock = threading.Lock()
_lib = None

KERNEL_COULOMB, KERNEL_ERF, KERNEL_ERFC = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=gnu11",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class _Basis(C.Structure):
    _fields_ = [("nshell", C.c_int), ("l", C.c_void_p), ("nprim", C.c_void_p),
                ("prim_off", C.c_void_p), ("center", C.c_void_p),
                ("exps", C.c_void_p), ("coeffs", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("omega", C.c_double), ("eps_sr", C.c_double), ("eps_lr", C.c_double),
                ("gmesh", C.c_int * 3), ("do_sr", C.c_int), ("do_g0", C.c_int),
                ("do_lr", C.c_int), ("direct_phase", C.c_int)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.or_boys.argtypes = [C.c_int, C.c_double, C.c_void_p]
            _lib.or_prim3c.argtypes = [C.c_int, C.c_double, C.c_int, C.c_double, C.c_void_p,
                                       C.c_int, C.c_double, C.c_void_p, C.c_int, C.c_double,
                                       C.c_void_p, C.c_void_p]
            _lib.or_prim2c.argtypes = [C.c_int, C.c_double, C.c_int, C.c_double, C.c_void_p,
                                       C.c_int, C.c_double, C.c_void_p, C.c_void_p]
            _lib.or_prim_ovlp.argtypes = [C.c_int, C.c_double, C.c_void_p, C.c_int, C.c_double,
                                          C.c_void_p, C.c_void_p]
            _lib.or_prim_ft.argtypes = [C.c_int, C.c_double, C.c_void_p, C.c_int, C.c_double,
                                        C.c_void_p, C.c_void_p, C.c_void_p]
            _lib.or_norm_coeffs.argtypes = [C.c_void_p, C.c_void_p]
            _lib.or_j3c.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
            _lib.or_j3c_fullG.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                          C.c_void_p, C.c_void_p]
            _lib.or_j2c.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_void_p, C.c_void_p]
            _lib.or_j2c_fullG.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
            _lib.or_cholesky.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
            _lib.or_cholesky.restype = C.c_int
            _lib.or_sr_bounds.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_double,
                                          C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_int,
                                          C.c_void_p, C.c_void_p, C.c_void_p]
            _lib.or_aux_charge.argtypes = [C.c_void_p, C.c_void_p]
            _lib.or_count_nf_cells.argtypes = [C.c_void_p]
            _lib.or_count_nf_cells.restype = C.c_int
            _lib.or_num_threads.restype = C.c_int
            _lib.or_set_num_threads.argtypes = [C.c_int]
            _lib.or_flops_end.argtypes = [C.c_void_p]
            _lib.or_flops_ncat.restype = C.c_int
        return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class _BasisRef:
    """Holds contiguous copies of a basis and the ctypes struct that points at them."""

    def __init__(self, b):
        self.l = np.ascontiguousarray(b.l, dtype=np.int32)
        self.nprim = np.ascontiguousarray(b.nprim, dtype=np.int32)
        self.prim_off = np.ascontiguousarray(b.prim_off, dtype=np.int32)
        self.center = np.ascontiguousarray(b.center, dtype=np.float64).reshape(-1, 3)
        self.exps = np.ascontiguousarray(b.exps, dtype=np.float64)
        self.coeffs = np.ascontiguousarray(b.coeffs, dtype=np.float64)
        self.s = _Basis(len(self.l), _p(self.l), _p(self.nprim), _p(self.prim_off),
                        _p(self.center), _p(self.exps), _p(self.coeffs))
        self.nfunc = int(sum((l + 1) * (l + 2) // 2 for l in self.l))

    def ref(self):
        return C.byref(self.s)


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def boys(mmax: int, T: float) -> np.ndarray:
    out = np.zeros(mmax + 1)
    lib().or_boys(mmax, float(T), _p(out))
    return out


def prim3c(kernel, omega, lc, g, Cc, la, a, A, lb, b, B):
    out = np.zeros(ncart(lc) * ncart(la) * ncart(lb))
    v = [np.ascontiguousarray(x, dtype=np.float64) for x in (Cc, A, B)]
    lib().or_prim3c(kernel, omega, lc, g, _p(v[0]), la, a, _p(v[1]), lb, b, _p(v[2]), _p(out))
    return out.reshape(ncart(lc), ncart(la), ncart(lb))


def prim2c(kernel, omega, lc, g, Cc, ld, e, D):
    out = np.zeros(ncart(lc) * ncart(ld))
    v = [np.ascontiguousarray(x, dtype=np.float64) for x in (Cc, D)]
    lib().or_prim2c(kernel, omega, lc, g, _p(v[0]), ld, e, _p(v[1]), _p(out))
    return out.reshape(ncart(lc), ncart(ld))


def prim_ovlp(la, a, A, lb, b, B):
    out = np.zeros(ncart(la) * ncart(lb))
    v = [np.ascontiguousarray(x, dtype=np.float64) for x in (A, B)]
    lib().or_prim_ovlp(la, a, _p(v[0]), lb, b, _p(v[1]), _p(out))
    return out.reshape(ncart(la), ncart(lb))


def prim_ft(la, a, A, lb, b, B, q):
    out = np.zeros(ncart(la) * ncart(lb), dtype=np.complex128)
    v = [np.ascontiguousarray(x, dtype=np.float64) for x in (A, B, q)]
    lib().or_prim_ft(la, a, _p(v[0]), lb, b, _p(v[1]), _p(v[2]), _p(out))
    return out.reshape(ncart(la), ncart(lb))


def norm_coeffs(basis) -> np.ndarray:
    r = _BasisRef(basis)
    out = np.zeros_like(r.exps)
    lib().or_norm_coeffs(r.ref(), _p(out))
    return out


def aux_charge(aux) -> np.ndarray:
    r = _BasisRef(aux)
    out = np.zeros(r.nfunc)
    lib().or_aux_charge(r.ref(), _p(out))
    return out


def _a9(cell_a):
    return np.ascontiguousarray(np.asarray(cell_a, dtype=np.float64).reshape(9))


def _i3(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32).reshape(3))


def _opts(omega, eps_sr, eps_lr, gmesh, sr, g0, lr, direct):
    o = _Opts()
    o.omega, o.eps_sr, o.eps_lr = float(omega), float(eps_sr), float(eps_lr)
    for i in range(3):
        o.gmesh[i] = int(gmesh[i]) if gmesh is not None else 1
    o.do_sr, o.do_g0, o.do_lr, o.direct_phase = int(sr), int(g0), int(lr), int(direct)
    return o


def aux_shell_nfunc(aux, s0, s1):
    return int(sum(ncart(int(l)) for l in np.asarray(aux.l)[s0:s1]))


def j3c(cell_a, kmesh, ao, aux, omega, kpairs, *, eps_sr=1e-10, eps_lr=1e-10, gmesh=None,
        shells=None, sr=True, g0=True, lr=True, direct_phase=False, return_counts=False):
    """Route R1: V[pair][P][mu][nu] (complex128) for aux shells ``shells`` = (s0, s1)."""
    ra, rx = _BasisRef(ao), _BasisRef(aux)
    s0, s1 = shells if shells is not None else (0, len(rx.l))
    kp = np.ascontiguousarray(np.asarray(kpairs, dtype=np.int32).reshape(-1, 2))
    nP = aux_shell_nfunc(aux, s0, s1)
    V = np.zeros((len(kp), nP, ra.nfunc, ra.nfunc), dtype=np.complex128)
    cnt = np.zeros(2, dtype=np.int64)
    if lr and gmesh is None:
        raise ValueError("LR needs a G mesh")
    o = _opts(omega, eps_sr, eps_lr, gmesh, sr, g0, lr, direct_phase)
    lib().or_j3c(_p(_a9(cell_a)), _p(_i3(kmesh)), ra.ref(), rx.ref(), C.byref(o), s0, s1,
                 len(kp), _p(kp), _p(V), _p(cnt))
    if return_counts:
        return V, {"terms": int(cnt[0]), "integrals": int(cnt[1])}
    return V


def j3c_fullG(cell_a, kmesh, ao, aux, kpairs, gmesh, *, eps_lr=1e-14, shells=None):
    """Route R2: the whole Coulomb integral (q = 0 removed) in reciprocal space."""
    ra, rx = _BasisRef(ao), _BasisRef(aux)
    s0, s1 = shells if shells is not None else (0, len(rx.l))
    kp = np.ascontiguousarray(np.asarray(kpairs, dtype=np.int32).reshape(-1, 2))
    nP = aux_shell_nfunc(aux, s0, s1)
    V = np.zeros((len(kp), nP, ra.nfunc, ra.nfunc), dtype=np.complex128)
    o = _opts(1.0, 1e-14, eps_lr, gmesh, 0, 0, 0, 0)
    lib().or_j3c_fullG(_p(_a9(cell_a)), _p(_i3(kmesh)), ra.ref(), rx.ref(), C.byref(o),
                       _p(_i3(gmesh)), s0, s1, len(kp), _p(kp), _p(V))
    return V


def j2c(cell_a, kmesh, aux, omega, klist, *, eps_sr=1e-10, eps_lr=1e-10, gmesh=None,
        sr=True, g0=True, lr=True):
    rx = _BasisRef(aux)
    kl = np.ascontiguousarray(np.asarray(klist, dtype=np.int32).reshape(-1))
    J = np.zeros((len(kl), rx.nfunc, rx.nfunc), dtype=np.complex128)
    if lr and gmesh is None:
        raise ValueError("LR needs a G mesh")
    o = _opts(omega, eps_sr, eps_lr, gmesh, sr, g0, lr, 0)
    lib().or_j2c(_p(_a9(cell_a)), _p(_i3(kmesh)), rx.ref(), C.byref(o), len(kl), _p(kl), _p(J))
    return J


def j2c_fullG(cell_a, kmesh, aux, klist, gmesh):
    rx = _BasisRef(aux)
    kl = np.ascontiguousarray(np.asarray(klist, dtype=np.int32).reshape(-1))
    J = np.zeros((len(kl), rx.nfunc, rx.nfunc), dtype=np.complex128)
    o = _opts(1.0, 1e-14, 1e-14, None, 0, 0, 0, 0)
    lib().or_j2c_fullG(_p(_a9(cell_a)), _p(_i3(kmesh)), rx.ref(), C.byref(o), _p(_i3(gmesh)),
                       len(kl), _p(kl), _p(J))
    return J


def cholesky(A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    Lo = np.zeros_like(A)
    rc = lib().or_cholesky(n, _p(A), _p(Lo))
    return Lo, (rc - 1 if rc else -1)


def sr_bounds(cell_a, omega, eps, aux, P, ao, mu, nu):
    ra, rx = _BasisRef(ao), _BasisRef(aux)
    rc = np.zeros(1)
    r12 = np.zeros(512)
    nw = np.zeros(1, dtype=np.int32)
    lib().or_sr_bounds(_p(_a9(cell_a)), _p(_i3((1, 1, 1))), float(omega), float(eps), rx.ref(),
                       int(P), ra.ref(), int(mu), int(nu), _p(rc), _p(r12), _p(nw))
    return float(rc[0]), r12[: int(nw[0])].copy()


def count_nf_cells(cell_a) -> int:
    return int(lib().or_count_nf_cells(_p(_a9(cell_a))))


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> None:
    lib().or_set_num_threads(int(n))


# Categories of the instrumented operation counter (rsgdf_oracle.c, in its order).
FLOP_CATEGORIES = ("sep_T", "boys_calls", "boys_orders", "combine", "seed", "hermite", "per_combination")
# Counting convention for one Boys evaluation of orders 0..m: the tabulated
# Taylor scheme -- F_m(T) and e^{-T} each from a degree-6 polynomial about the
# nearest grid point (6 fused multiply-adds, 12 flops), then m downward steps
# F_n = (2T F_{n+1} + e^{-T})/(2n+1) (one FMA and one multiply, 3 flops).
BOYS_BASE_FLOPS = 24
BOYS_STEP_FLOPS = 3


def sr_term_op_counts(lc, la, lb, omega=0.4, T=2.0):
    """Operation counts of one SR (erfc-kernel) primitive integral of class
    (lc | la lb), tallied by the instrumented oracle while it evaluates the
    integral (Eq. VPmunu_SR; the auxiliary function G_n and the Hermite
    integrals R_tuv of the McMurchie-Davidson scheme).  Returns a dict over
    FLOP_CATEGORIES.  The centres are placed so that the separation gives the
    requested T at unit exponents; the counts do not depend on it."""
    lib()
    g, a, b = 1.0, 1.0, 1.0
    p = a + b
    alpha = p * g / (p + g)
    r = (float(T) / alpha) ** 0.5
    A = np.zeros(3)
    B = np.zeros(3)
    Cc = np.array([r, 0.0, 0.0])
    out = np.zeros(len(FLOP_CATEGORIES), dtype=np.int64)
    assert int(_lib.or_flops_ncat()) == len(FLOP_CATEGORIES)
    _lib.or_flops_begin()
    try:
        prim3c(KERNEL_ERFC, float(omega), lc, g, Cc, la, a, A, lb, b, B)
    finally:
        _lib.or_flops_end(_p(out))
    return dict(zip(FLOP_CATEGORIES, (int(x) for x in out)))


def sr_term_flops(lc, la, lb):
    """FP64 flops of the part of one SR primitive term that depends on its
    lattice translation: separation and T, two Boys evaluations (counted by
    the convention above), the erfc combination, the Hermite seeds and
    recursion.  Per-combination constants are excluded."""
    c = sr_term_op_counts(lc, la, lb)
    boys = BOYS_BASE_FLOPS * c["boys_calls"] + BOYS_STEP_FLOPS * c["boys_orders"]
    return c["sep_T"] + boys + c["combine"] + c["seed"] + c["hermite"]
