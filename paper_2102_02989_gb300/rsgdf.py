"""Thin Python binding of the C ABI in ``include/rsgdf.h`` (ctypes).

Argument marshalling only: every step of the j3c / j2c / k-phase paths runs in
the CUDA library ``_build/librsgdf.so``.  PyTorch supplies device memory and the
current CUDA stream.  There is no CPU fallback: if the library cannot be loaded
or no sm_103a device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "librsgdf.so")
_lock = threading.Lock()
_lib = None

RSGDF_OK, RSGDF_EINVAL, RSGDF_ENOMEM, RSGDF_ENOTPD, RSGDF_ETIMEOUT, RSGDF_EDEVICE, RSGDF_ENOTIMPL = 0, -1, -2, -3, -4, -5, -6
RSGDF_FP64, RSGDF_MIXED = 0, 1
RSGDF_SCREEN_BOUND, RSGDF_SCREEN_LEARNED = 0, 1
RSGDF_BATCH_GRAPH, RSGDF_BATCH_AUTOTUNE = 1, 2
RSGDF_FIT_CHOLESKY, RSGDF_FIT_EIGEN, RSGDF_FIT_AUTO = 0, 1, 2
RSGDF_KERNEL_ERF, RSGDF_KERNEL_PLAIN = 0, 1
RSGDF_DF_NMAX, RSGDF_DF_SWEEPS = 1024, 40

# names exported by the library (every declaration of include/rsgdf.h)
EXPORTS = ("rsgdf_j2c", "rsgdf_j3c_sr", "rsgdf_j3c_lr", "rsgdf_j3c", "rsgdf_kphase", "rsgdf_kphase_noalloc",
           "rsgdf_last_stats", "rsgdf_params", "rsgdf_last_error", "rsgdf_probe_fp64", "rsgdf_sync_status",
           "rsgdf_mlp_nparams", "rsgdf_mlp_create", "rsgdf_mlp_destroy", "rsgdf_mlp_get_params",
           "rsgdf_mlp_set_margin", "rsgdf_mlp_set_base", "rsgdf_mlp_forward", "rsgdf_mlp_loss_grad", "rsgdf_mlp_train",
           "rsgdf_sr_items", "rsgdf_j3c_batch_create", "rsgdf_j3c_batch_run", "rsgdf_j3c_batch_destroy",
           "rsgdf_j3c_batch_tiles", "rsgdf_j3c_batch", "rsgdf_df_metric", "rsgdf_df_fit", "rsgdf_df_jk", "rsgdf_df_rho",
           "rsgdf_sph_coefficients", "rsgdf_sph_nfunc", "rsgdf_cart2sph_j3c", "rsgdf_cart2sph_j2c",
           "rsgdf_split_basis", "rsgdf_sr_items_split", "rsgdf_split_combine", "rsgdf_set_scratch_limit",
           "rsgdf_selftest_wait")
RSGDF_MLP_NFEAT = 10


class RsgdfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("rsgdf error %d: %s" % (code, msg))
        self.code = code


class _Basis(C.Structure):
    _fields_ = [("nshell", C.c_int), ("l", C.c_void_p), ("nprim", C.c_void_p),
                ("prim_off", C.c_void_p), ("center", C.c_void_p), ("exps", C.c_void_p),
                ("coeffs", C.c_void_p)]


class _Cell(C.Structure):
    _fields_ = [("a", C.c_double * 9), ("kmesh", C.c_int * 3)]


class _Opts(C.Structure):
    _fields_ = [("omega", C.c_double), ("gmesh", C.c_int * 3), ("eps_screen", C.c_double),
                ("eps_lr", C.c_double), ("precision", C.c_int), ("screening", C.c_int),
                ("mlp", C.c_void_p), ("stream", C.c_void_p), ("split_alpha", C.c_double), ("kernel", C.c_int)]


class _Problem(C.Structure):
    _fields_ = [("cell", C.c_void_p), ("ao", C.c_void_p), ("aux", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("sr_terms", C.c_longlong), ("sr_integrals", C.c_longlong),
                ("sr_flops", C.c_longlong), ("aft_units", C.c_longlong),
                ("lr_flops", C.c_longlong), ("omega", C.c_double), ("gmesh", C.c_int * 3),
                ("n_launch", C.c_int), ("sr_ms", C.c_double), ("aft_ms", C.c_double),
                ("lr_gemm_ms", C.c_double), ("phase_ms", C.c_double), ("other_ms", C.c_double),
                ("sr_terms_by_L", C.c_longlong * 10), ("sr_prim_terms", C.c_longlong),
                ("sr_items", C.c_longlong), ("sr_items_pruned", C.c_longlong),
                ("sr_ms_by_L", C.c_double * 10), ("sr_prim_terms_by_L", C.c_longlong * 10),
                ("sr_prim_terms_skipped", C.c_longlong)]

    def asdict(self):
        return {"sr_terms": self.sr_terms, "sr_integrals": self.sr_integrals,
                "sr_flops": self.sr_flops, "aft_units": self.aft_units, "lr_flops": self.lr_flops,
                "omega": self.omega, "gmesh": tuple(self.gmesh), "n_launch": self.n_launch,
                "sr_ms": self.sr_ms, "aft_ms": self.aft_ms, "lr_gemm_ms": self.lr_gemm_ms,
                "phase_ms": self.phase_ms, "other_ms": self.other_ms,
                "sr_terms_by_L": list(self.sr_terms_by_L), "sr_prim_terms": self.sr_prim_terms,
                "sr_items": self.sr_items, "sr_items_pruned": self.sr_items_pruned,
                "sr_ms_by_L": list(self.sr_ms_by_L), "sr_prim_terms_by_L": list(self.sr_prim_terms_by_L),
                "sr_prim_terms_skipped": self.sr_prim_terms_skipped}


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load the CUDA library (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _b
        if _b.needs_build():
            _b.build()
        if not os.path.exists(_LIB_PATH):
            raise ImportError("librsgdf.so is missing: run paper_2102_02989_gb300.build.build()")
        lib = C.CDLL(_LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        lib.rsgdf_j2c.argtypes = [vp, vp, vp, i, vp, vp, vp, vp]
        for n in ("rsgdf_j3c_sr", "rsgdf_j3c_lr", "rsgdf_j3c"):
            getattr(lib, n).argtypes = [vp, vp, vp, vp, i, vp, i, i, vp]
        lib.rsgdf_kphase.argtypes = [vp, vp, C.c_longlong, i, vp, vp, vp]
        lib.rsgdf_kphase_noalloc.argtypes = [vp, vp, C.c_longlong, i, vp, vp, vp]
        lib.rsgdf_last_stats.argtypes = [vp]
        lib.rsgdf_params.argtypes = [vp, vp, vp, vp]
        lib.rsgdf_last_error.restype = C.c_char_p
        lib.rsgdf_probe_fp64.argtypes = [vp, vp]
        lib.rsgdf_sync_status.argtypes = [vp]
        lib.rsgdf_set_scratch_limit.argtypes = [C.c_longlong]
        lib.rsgdf_selftest_wait.argtypes = [i, C.c_longlong, vp]
        lib.rsgdf_mlp_nparams.argtypes = [i]
        lib.rsgdf_mlp_create.argtypes = [i, vp, vp, vp, vp]
        lib.rsgdf_mlp_destroy.argtypes = [vp]
        lib.rsgdf_mlp_get_params.argtypes = [vp, vp]
        lib.rsgdf_mlp_set_margin.argtypes = [vp, C.c_float]
        lib.rsgdf_mlp_set_base.argtypes = [vp, C.c_int, C.c_float, C.c_float, vp]
        lib.rsgdf_mlp_forward.argtypes = [vp, vp, C.c_longlong, vp, vp]
        lib.rsgdf_mlp_loss_grad.argtypes = [vp, vp, vp, C.c_longlong, C.c_float, vp, vp, vp]
        lib.rsgdf_mlp_train.argtypes = [vp, vp, vp, C.c_longlong, i, i, C.c_float, C.c_float, C.c_uint, vp, vp]
        lib.rsgdf_sr_items.argtypes = [vp, vp, vp, vp, i, i, vp, vp, vp]
        lib.rsgdf_j3c_batch_create.argtypes = [i, vp, vp, vp, vp, i, vp]
        lib.rsgdf_j3c_batch_run.argtypes = [vp, vp, vp]
        lib.rsgdf_j3c_batch_destroy.argtypes = [vp]
        lib.rsgdf_j3c_batch_tiles.argtypes = [vp, vp, vp, vp]
        lib.rsgdf_j3c_batch.argtypes = [i, vp, vp, vp, vp, vp]
        lib.rsgdf_df_metric.argtypes = [vp, i, i, i, C.c_double, vp, vp, vp, vp, vp]
        lib.rsgdf_df_fit.argtypes = [vp, vp, i, i, i, vp, vp, vp, vp]
        lib.rsgdf_df_jk.argtypes = [vp, vp, i, i, i, vp, vp, vp, vp, vp, vp]
        lib.rsgdf_df_rho.argtypes = [vp, vp, i, i, i, vp, vp, vp, vp]
        lib.rsgdf_sph_coefficients.argtypes = [i, vp]
        lib.rsgdf_sph_nfunc.argtypes = [vp, vp]
        lib.rsgdf_cart2sph_j3c.argtypes = [vp, vp, i, i, i, vp, vp, vp]
        lib.rsgdf_cart2sph_j2c.argtypes = [vp, i, vp, vp, vp]
        lib.rsgdf_split_basis.argtypes = [vp, C.c_double] + [vp] * 11
        lib.rsgdf_sr_items_split.argtypes = [vp, vp, vp, vp, C.c_double, vp]
        lib.rsgdf_split_combine.argtypes = [vp, vp, C.c_double, i, vp, vp, vp, vp]
        for n in EXPORTS:
            if n != "rsgdf_last_error":
                getattr(lib, n).restype = C.c_int
        _lib = lib
        return lib


def _check(rc):
    if rc != RSGDF_OK:
        raise RsgdfError(rc, load().rsgdf_last_error().decode())


class _BasisRef:
    def __init__(self, b):
        self.l = np.ascontiguousarray(b.l, dtype=np.int32)
        self.nprim = np.ascontiguousarray(b.nprim, dtype=np.int32)
        self.prim_off = np.ascontiguousarray(b.prim_off, dtype=np.int32)
        self.center = np.ascontiguousarray(b.center, dtype=np.float64)
        self.exps = np.ascontiguousarray(b.exps, dtype=np.float64)
        self.coeffs = np.ascontiguousarray(b.coeffs, dtype=np.float64)
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        self.s = _Basis(len(self.l), p(self.l), p(self.nprim), p(self.prim_off), p(self.center),
                        p(self.exps), p(self.coeffs))
        self.nfunc = int(sum((int(l) + 1) * (int(l) + 2) // 2 for l in self.l))

    def ref(self):
        return C.byref(self.s)


def _cell(a, kmesh):
    c = _Cell()
    av = np.asarray(a, dtype=np.float64).reshape(9)
    for k in range(9):
        c.a[k] = float(av[k])
    for k in range(3):
        c.kmesh[k] = int(kmesh[k])
    return c


def _stream_ptr(stream):
    import torch
    if stream is None and not torch.cuda.is_available():
        return C.c_void_p(0)   # host-only calls (planning); device calls fail with RSGDF_EDEVICE
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _opts(omega=None, gmesh=None, eps_screen=1e-8, eps_lr=1e-8, precision=RSGDF_FP64,
          screening=RSGDF_SCREEN_BOUND, mlp=None, stream=None, split_alpha=0.0, kernel=RSGDF_KERNEL_ERF):
    o = _Opts()
    o.split_alpha, o.kernel = float(split_alpha), int(kernel)
    o.omega = float(omega) if omega else 0.0
    for k in range(3):
        o.gmesh[k] = int(gmesh[k]) if gmesh is not None else 0
    o.eps_screen, o.eps_lr = float(eps_screen), float(eps_lr)
    o.precision, o.screening = int(precision), int(screening)
    o.mlp = mlp
    o.stream = _stream_ptr(stream)
    return o


def _nfunc(b, s0, s1):
    return int(sum((int(l) + 1) * (int(l) + 2) // 2 for l in np.asarray(b.l)[s0:s1]))


def rsgdf_params(a, kmesh, omega=None, gmesh=None, eps_lr=1e-8):
    lib = load()
    c = _cell(a, kmesh)
    o = _Opts()
    o.omega = float(omega) if omega else 0.0
    for k in range(3):
        o.gmesh[k] = int(gmesh[k]) if gmesh is not None else 0
    o.eps_screen, o.eps_lr = 1e-8, float(eps_lr)
    w = C.c_double()
    g = (C.c_int * 3)()
    _check(lib.rsgdf_params(C.byref(c), C.byref(o), C.byref(w), g))
    return float(w.value), tuple(int(x) for x in g)


def _j3c_call(name, a, kmesh, ao, aux, kpairs, shells=None, out=None, **opt):
    import torch
    lib = load()
    ra, rx = _BasisRef(ao), _BasisRef(aux)
    s0, s1 = shells if shells is not None else (0, len(rx.l))
    kp = np.ascontiguousarray(np.asarray(kpairs, dtype=np.int32).reshape(-1, 2))
    nP = _nfunc(aux, s0, s1)
    shape = (len(kp), nP, ra.nfunc, ra.nfunc)
    if out is None:
        out = torch.zeros(shape, dtype=torch.complex128, device="cuda")
    assert out.is_cuda and out.dtype == torch.complex128 and tuple(out.shape) == shape and out.is_contiguous()
    c = _cell(a, kmesh)
    o = _opts(**opt)
    rc = getattr(lib, name)(C.byref(c), ra.ref(), rx.ref(), C.byref(o), len(kp),
                            kp.ctypes.data_as(C.c_void_p), s0, s1, C.c_void_p(out.data_ptr()))
    _check(rc)
    return out


def rsgdf_j3c_sr(a, kmesh, ao, aux, kpairs, shells=None, out=None, **opt):
    """SR part incl. the G = 0 correction; overwrites ``out`` [pair][P][mu][nu] (complex128, cuda)."""
    return _j3c_call("rsgdf_j3c_sr", a, kmesh, ao, aux, kpairs, shells, out, **opt)


def rsgdf_j3c_lr(a, kmesh, ao, aux, kpairs, shells=None, out=None, **opt):
    """LR part; ADDED to ``out``."""
    return _j3c_call("rsgdf_j3c_lr", a, kmesh, ao, aux, kpairs, shells, out, **opt)


def rsgdf_j3c(a, kmesh, ao, aux, kpairs, shells=None, out=None, **opt):
    """SR + G = 0 + LR; overwrites ``out``."""
    return _j3c_call("rsgdf_j3c", a, kmesh, ao, aux, kpairs, shells, out, **opt)


def rsgdf_j2c(a, kmesh, aux, klist, cholesky=True, **opt):
    import torch
    lib = load()
    rx = _BasisRef(aux)
    kl = np.ascontiguousarray(np.asarray(klist, dtype=np.int32).reshape(-1))
    J = torch.zeros((len(kl), rx.nfunc, rx.nfunc), dtype=torch.complex128, device="cuda")
    L = torch.zeros_like(J) if cholesky else None
    info = torch.full((len(kl),), -2, dtype=torch.int32, device="cuda")
    c = _cell(a, kmesh)
    o = _opts(**opt)
    _check(lib.rsgdf_j2c(C.byref(c), rx.ref(), C.byref(o), len(kl), kl.ctypes.data_as(C.c_void_p),
                         C.c_void_p(J.data_ptr()), C.c_void_p(L.data_ptr()) if L is not None else None,
                         C.c_void_p(info.data_ptr())))
    return J, L, info


def rsgdf_kphase(a, kmesh, X, kpairs, out=None, stream=None):
    """V[pair][i] = sum_{lt,dt} e^{-i k12.lt} e^{i k2.dt} X[lt][dt][i]; X float64 cuda [Nk][Nk][m]."""
    import torch
    lib = load()
    assert X.is_cuda and X.dtype == torch.float64 and X.is_contiguous()
    nk = int(np.prod(kmesh))
    m = X.numel() // (nk * nk)
    kp = np.ascontiguousarray(np.asarray(kpairs, dtype=np.int32).reshape(-1, 2))
    if out is None:
        out = torch.empty((len(kp), m), dtype=torch.complex128, device="cuda")
    c = _cell(a, kmesh)
    _check(lib.rsgdf_kphase(C.byref(c), C.c_void_p(X.data_ptr()), m, len(kp),
                            kp.ctypes.data_as(C.c_void_p), C.c_void_p(out.data_ptr()),
                            _stream_ptr(stream)))
    return out


def rsgdf_kphase_noalloc(a, kmesh, X, kpairs, out, stream=None):
    """rsgdf_kphase without device allocation: ``out`` (complex128 cuda
    [npair][m]) must be given; the library's scratch is a static device array
    of RSGDF_NOALLOC_SCRATCH_BYTES shared by all calls."""
    import torch
    lib = load()
    assert X.is_cuda and X.dtype == torch.float64 and X.is_contiguous()
    assert out.is_cuda and out.dtype == torch.complex128 and out.is_contiguous()
    nk = int(np.prod(kmesh))
    m = X.numel() // (nk * nk)
    kp = np.ascontiguousarray(np.asarray(kpairs, dtype=np.int32).reshape(-1, 2))
    assert tuple(out.shape) == (len(kp), m)
    c = _cell(a, kmesh)
    _check(lib.rsgdf_kphase_noalloc(C.byref(c), C.c_void_p(X.data_ptr()), m, len(kp),
                                    kp.ctypes.data_as(C.c_void_p), C.c_void_p(out.data_ptr()),
                                    _stream_ptr(stream)))
    return out


def _cplx_cuda(x, name):
    import torch
    assert x.is_cuda and x.dtype == torch.complex128 and x.is_contiguous(), name + ": complex128 contiguous cuda tensor"
    return C.c_void_p(x.data_ptr())


def rsgdf_df_metric(J, method=RSGDF_FIT_AUTO, rel=1e-6, stream=None):
    """Fitting transforms of the metrics J [nk][naux][naux] (complex128 cuda):
    returns (T, lam, nkept, info) with T_k^H T_k = (J^k)^{-1} on the kept part
    (Cholesky T = L^{-1}; eigen route: canonical orthogonalisation)."""
    import torch
    lib = load()
    Jp = _cplx_cuda(J, "J")
    nk, naux = int(J.shape[0]), int(J.shape[1])
    T = torch.empty_like(J)
    lam = torch.empty((nk, naux), dtype=torch.float64, device=J.device)
    nkept = torch.empty(nk, dtype=torch.int32, device=J.device)
    info = torch.empty(nk, dtype=torch.int32, device=J.device)
    _check(lib.rsgdf_df_metric(Jp, naux, nk, int(method), float(rel), C.c_void_p(T.data_ptr()),
                               C.c_void_p(lam.data_ptr()), C.c_void_p(nkept.data_ptr()),
                               C.c_void_p(info.data_ptr()), _stream_ptr(stream)))
    return T, lam, nkept, info


def rsgdf_df_fit(a, kmesh, T, V, kpairs, out=None, stream=None):
    """B[pair] = T[k12] V[pair]; T [Nk][naux][naux], V [npair][naux][nao][nao] (complex128 cuda)."""
    import torch
    lib = load()
    kp = np.ascontiguousarray(np.asarray(kpairs, dtype=np.int32).reshape(-1, 2))
    naux, nao = int(V.shape[1]), int(V.shape[2])
    if out is None:
        out = torch.empty_like(V)
    c = _cell(a, kmesh)
    _check(lib.rsgdf_df_fit(C.byref(c), _cplx_cuda(T, "T"), naux, nao, len(kp), kp.ctypes.data_as(C.c_void_p),
                            _cplx_cuda(V, "V"), _cplx_cuda(out, "out"), _stream_ptr(stream)))
    return out


def rsgdf_df_rho(a, kmesh, B, kpairs, D, stream=None):
    """rho_P = sum over the listed (k, k) pairs of Tr[B^kk_P D^k] (complex128 cuda [naux])."""
    import torch
    lib = load()
    kp = np.ascontiguousarray(np.asarray(kpairs, dtype=np.int32).reshape(-1, 2))
    naux, nao = int(B.shape[1]), int(B.shape[2])
    rho = torch.empty(naux, dtype=torch.complex128, device=B.device)
    c = _cell(a, kmesh)
    _check(lib.rsgdf_df_rho(C.byref(c), _cplx_cuda(B, "B"), naux, nao, len(kp), kp.ctypes.data_as(C.c_void_p),
                            _cplx_cuda(D, "D"), C.c_void_p(rho.data_ptr()), _stream_ptr(stream)))
    return rho


def rsgdf_df_jk(a, kmesh, B, kpairs, D, with_j=True, with_k=True, rho=None, stream=None):
    """Fitted Coulomb and exchange matrices (J, K) [Nk][nao][nao] of the
    densities D [Nk][nao][nao] from B [npair][naux][nao][nao] (complex128 cuda);
    a matrix not asked for is None.  rho: the fitted density summed over all
    pairs (e.g. over processes), else taken from the listed pairs."""
    import torch
    lib = load()
    kp = np.ascontiguousarray(np.asarray(kpairs, dtype=np.int32).reshape(-1, 2))
    naux, nao = int(B.shape[1]), int(B.shape[2])
    Jm = torch.empty_like(D) if with_j else None
    Km = torch.empty_like(D) if with_k else None
    c = _cell(a, kmesh)
    _check(lib.rsgdf_df_jk(C.byref(c), _cplx_cuda(B, "B"), naux, nao, len(kp), kp.ctypes.data_as(C.c_void_p),
                           _cplx_cuda(D, "D"), C.c_void_p(rho.data_ptr() if rho is not None else 0),
                           C.c_void_p(Jm.data_ptr() if with_j else 0),
                           C.c_void_p(Km.data_ptr() if with_k else 0), _stream_ptr(stream)))
    return Jm, Km


def rsgdf_sph_coefficients(l):
    """[(2l+1)][ncart] monomial coefficients of the real solid harmonics (host)."""
    out = np.zeros((2 * l + 1, (l + 1) * (l + 2) // 2))
    _check(load().rsgdf_sph_coefficients(int(l), out.ctypes.data_as(C.c_void_p)))
    return out


def rsgdf_sph_nfunc(basis):
    n = C.c_int(0)
    _check(load().rsgdf_sph_nfunc(_BasisRef(basis).ref(), C.byref(n)))
    return n.value


def rsgdf_cart2sph_j3c(ao, aux, V, shells=None, stream=None):
    """V [npair][nP][nao][nao] over Cartesian functions -> the same over spherical ones."""
    import torch
    ra, rx = _BasisRef(ao), _BasisRef(aux)
    s0, s1 = shells if shells else (0, len(rx.l))
    nsx = sum(2 * int(l) + 1 for l in rx.l[s0:s1])
    nsa = sum(2 * int(l) + 1 for l in ra.l)
    ncx = sum((int(l) + 1) * (int(l) + 2) // 2 for l in rx.l[s0:s1])
    assert tuple(V.shape[1:]) == (ncx, ra.nfunc, ra.nfunc), "V must be [npair][nP][nao][nao] over Cartesian functions"
    out = torch.empty((V.shape[0], nsx, nsa, nsa), dtype=torch.complex128, device=V.device)
    _check(load().rsgdf_cart2sph_j3c(ra.ref(), rx.ref(), s0, s1, int(V.shape[0]), _cplx_cuda(V, "V"),
                                     _cplx_cuda(out, "out"), _stream_ptr(stream)))
    return out


def rsgdf_cart2sph_j2c(aux, J, stream=None):
    """J [nk][naux][naux] over Cartesian functions -> the same over spherical ones."""
    import torch
    rx = _BasisRef(aux)
    ns = sum(2 * int(l) + 1 for l in rx.l)
    assert tuple(J.shape[1:]) == (rx.nfunc, rx.nfunc), "J must be [nk][naux][naux] over Cartesian functions"
    out = torch.empty((J.shape[0], ns, ns), dtype=torch.complex128, device=J.device)
    _check(load().rsgdf_cart2sph_j2c(rx.ref(), int(J.shape[0]), _cplx_cuda(J, "J"), _cplx_cuda(out, "out"),
                                     _stream_ptr(stream)))
    return out


def rsgdf_split_basis(basis, alpha_cut):
    """Compact/diffuse split (host): dict of the split basis' arrays (l, nprim,
    prim_off, center, exps, coeffs) plus parent, kind (0 compact, 1 diffuse)
    and weight per sub-shell."""
    lib = load()
    rb = _BasisRef(basis)
    ns, npt = C.c_int(0), C.c_int(0)
    nul = [None] * 9
    _check(lib.rsgdf_split_basis(rb.ref(), float(alpha_cut), C.byref(ns), C.byref(npt), *nul))
    n, m = ns.value, npt.value
    out = {"l": np.zeros(n, np.int32), "nprim": np.zeros(n, np.int32), "prim_off": np.zeros(n, np.int32),
           "center": np.zeros((n, 3)), "exps": np.zeros(m), "coeffs": np.zeros(m), "parent": np.zeros(n, np.int32),
           "kind": np.zeros(n, np.int32), "weight": np.zeros(n)}
    p = lambda k: out[k].ctypes.data_as(C.c_void_p)
    _check(lib.rsgdf_split_basis(rb.ref(), float(alpha_cut), C.byref(ns), C.byref(npt), p("l"), p("nprim"),
                                 p("prim_off"), p("center"), p("exps"), p("coeffs"), p("parent"), p("kind"),
                                 p("weight")))
    return out


def rsgdf_sr_items_split(a, kmesh, ao, aux, alpha_cut, **opt):
    """Host planner only: {"items": (unsplit, split, split range-separated types),
    "terms": the same as candidate primitive terms}."""
    lib = load()
    ra, rx = _BasisRef(ao), _BasisRef(aux)
    n = (C.c_longlong * 6)()
    o = _opts(**opt)
    _check(lib.rsgdf_sr_items_split(C.byref(_cell(a, kmesh)), ra.ref(), rx.ref(), C.byref(o), float(alpha_cut), n))
    return {"items": tuple(int(x) for x in n[:3]), "terms": tuple(int(x) for x in n[3:])}


def rsgdf_split_combine(ao, aux, alpha_cut, V_rs, V_g, stream=None):
    """V over the input bases from the range-separated (V_rs) and plain-kernel
    (V_g) tensors over the split bases (complex128 cuda)."""
    import torch
    ra, rx = _BasisRef(ao), _BasisRef(aux)
    out = torch.empty((V_rs.shape[0], rx.nfunc, ra.nfunc, ra.nfunc), dtype=torch.complex128, device=V_rs.device)
    nsub = lambda b: int(sum((int(l) + 1) * (int(l) + 2) // 2 for l in rsgdf_split_basis(b, alpha_cut)["l"]))
    want = (nsub(aux), nsub(ao), nsub(ao))
    assert tuple(V_rs.shape[1:]) == want and V_g.shape == V_rs.shape, "V_rs, V_g must be over the split bases"
    _check(load().rsgdf_split_combine(ra.ref(), rx.ref(), float(alpha_cut), int(V_rs.shape[0]),
                                      _cplx_cuda(V_rs, "V_rs"), _cplx_cuda(V_g, "V_g"), _cplx_cuda(out, "out"),
                                      _stream_ptr(stream)))
    return out


def rsgdf_last_stats() -> dict:
    s = Stats()
    _check(load().rsgdf_last_stats(C.byref(s)))
    return s.asdict()


def rsgdf_sync_status(stream=None) -> None:
    """Synchronise the stream; raise RsgdfError(RSGDF_ETIMEOUT) if a bounded device wait gave up."""
    _check(load().rsgdf_sync_status(_stream_ptr(stream)))


def rsgdf_set_scratch_limit(nbytes: int) -> None:
    """Largest device scratch (bytes) one call may hold; 0 = no limit."""
    _check(load().rsgdf_set_scratch_limit(int(nbytes)))


def rsgdf_selftest_wait(arrive: bool, limit: int, stream=None) -> None:
    """Enqueue the bounded-wait self-test; read its outcome with rsgdf_sync_status."""
    _check(load().rsgdf_selftest_wait(1 if arrive else 0, int(limit), _stream_ptr(stream)))


def rsgdf_last_error() -> str:
    return load().rsgdf_last_error().decode()


def rsgdf_probe_fp64(stream=None) -> float:
    v = C.c_double()
    _check(load().rsgdf_probe_fp64(C.byref(v), _stream_ptr(stream)))
    return float(v.value)


class Mlp:
    """Handle of the learned-screening network (parameters on the device)."""

    def __init__(self, params, mean, std):
        lib = load()
        p = np.ascontiguousarray(params, dtype=np.float32)
        mu = np.ascontiguousarray(mean, dtype=np.float32)
        sd = np.ascontiguousarray(std, dtype=np.float32)
        self.F = len(mu)
        assert len(p) == lib.rsgdf_mlp_nparams(self.F)
        h = C.c_void_p()
        _check(lib.rsgdf_mlp_create(self.F, p.ctypes.data_as(C.c_void_p), mu.ctypes.data_as(C.c_void_p),
                                    sd.ctypes.data_as(C.c_void_p), C.byref(h)))
        self.h = h

    @staticmethod
    def nparams(F=RSGDF_MLP_NFEAT):
        return int(load().rsgdf_mlp_nparams(F))

    def close(self):
        if getattr(self, "h", None):
            load().rsgdf_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.zeros(self.nparams(self.F), dtype=np.float32)
        _check(load().rsgdf_mlp_get_params(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def set_margin(self, margin):
        _check(load().rsgdf_mlp_set_margin(self.h, float(margin)))

    def set_base(self, feature, lo=-20.0, hi=20.0, guard=None):
        """guard: per class L = 0..9 (sequence of 10 floats) or None (all 0)"""
        g = np.zeros(10, np.float32) if guard is None else np.ascontiguousarray(guard, dtype=np.float32)
        assert g.shape == (10,)
        self._guard = g
        _check(load().rsgdf_mlp_set_base(self.h, int(feature), float(lo), float(hi), g.ctypes.data_as(C.c_void_p)))

    def forward(self, X, stream=None):
        import torch
        assert X.is_cuda and X.dtype == torch.float32 and X.is_contiguous()
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        _check(load().rsgdf_mlp_forward(self.h, C.c_void_p(X.data_ptr()), X.shape[0], C.c_void_p(y.data_ptr()),
                                        _stream_ptr(stream)))
        return y

    def loss_grad(self, X, t, tau=0.5, stream=None):
        loss = C.c_float()
        g = np.zeros(self.nparams(self.F), dtype=np.float32)
        _check(load().rsgdf_mlp_loss_grad(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(t.data_ptr()), X.shape[0],
                                          float(tau), C.byref(loss), g.ctypes.data_as(C.c_void_p),
                                          _stream_ptr(stream)))
        return float(loss.value), g

    def train(self, X, t, epochs=20, batch=1024, lr=1e-3, tau=0.5, seed=0, stream=None):
        loss = C.c_float()
        _check(load().rsgdf_mlp_train(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(t.data_ptr()), X.shape[0],
                                      int(epochs), int(batch), float(lr), float(tau), int(seed), C.byref(loss),
                                      _stream_ptr(stream)))
        return float(loss.value)


def rsgdf_sr_items(a, kmesh, ao, aux, shells=None, features=True, magnitudes=False, **opt):
    """(n_items, features [n][10] float32 cuda or None, log10 magnitudes [n] or None)"""
    import torch
    lib = load()
    ra, rx = _BasisRef(ao), _BasisRef(aux)
    s0, s1 = shells if shells is not None else (0, len(rx.l))
    c = _cell(a, kmesh)
    o = _opts(**opt)
    n = C.c_longlong()
    _check(lib.rsgdf_sr_items(C.byref(c), ra.ref(), rx.ref(), C.byref(o), s0, s1, C.byref(n), None, None))
    nn = int(n.value)
    feat = torch.zeros((nn, RSGDF_MLP_NFEAT), dtype=torch.float32, device="cuda") if features else None
    mag = torch.zeros(nn, dtype=torch.float32, device="cuda") if magnitudes else None
    if nn and (features or magnitudes):
        _check(lib.rsgdf_sr_items(C.byref(c), ra.ref(), rx.ref(), C.byref(o), s0, s1, C.byref(n),
                                  C.c_void_p(feat.data_ptr()) if feat is not None else None,
                                  C.c_void_p(mag.data_ptr()) if mag is not None else None))
    return nn, feat, mag


class Batch:
    """Handle of a batched j3c over many cells (plans and device buffers kept;
    runs issue kernels only, optionally replaying a captured CUDA graph).
    problems: list of (a, kmesh, ao, aux); kpairs: list of [npair][2] arrays."""

    def __init__(self, problems, kpairs, flags=0, **opt):
        lib = load()
        self.cells = [_cell(a, km) for (a, km, _, _) in problems]
        self.refs = [(_BasisRef(ao), _BasisRef(aux)) for (_, _, ao, aux) in problems]
        self.kp = [np.ascontiguousarray(np.asarray(k, dtype=np.int32).reshape(-1, 2)) for k in kpairs]
        n = len(problems)
        self.pr = (_Problem * n)()
        for p in range(n):
            self.pr[p].cell = C.cast(C.pointer(self.cells[p]), C.c_void_p)
            self.pr[p].ao = C.cast(C.pointer(self.refs[p][0].s), C.c_void_p)
            self.pr[p].aux = C.cast(C.pointer(self.refs[p][1].s), C.c_void_p)
        npair = np.array([len(k) for k in self.kp], dtype=np.int32)
        kcat = np.ascontiguousarray(np.concatenate(self.kp).reshape(-1))
        self.opts = _opts(**opt)
        h = C.c_void_p()
        _check(lib.rsgdf_j3c_batch_create(n, C.cast(self.pr, C.c_void_p), C.byref(self.opts),
                                          npair.ctypes.data_as(C.c_void_p), kcat.ctypes.data_as(C.c_void_p),
                                          int(flags), C.byref(h)))
        self.h = h
        self.shapes = [(len(self.kp[p]), self.refs[p][1].nfunc, self.refs[p][0].nfunc, self.refs[p][0].nfunc)
                       for p in range(n)]

    def outputs(self):
        import torch
        return [torch.zeros(s, dtype=torch.complex128, device="cuda") for s in self.shapes]

    def run(self, outs=None, stream=None):
        import torch
        if outs is None:
            outs = self.outputs()
        for o, s in zip(outs, self.shapes):
            assert o.is_cuda and o.dtype == torch.complex128 and tuple(o.shape) == s and o.is_contiguous()
        ptrs = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        _check(load().rsgdf_j3c_batch_run(self.h, C.cast(ptrs, C.c_void_p), _stream_ptr(stream)))
        return outs

    def tiles(self):
        g, b, r = (np.zeros(10, np.int32) for _ in range(3))
        _check(load().rsgdf_j3c_batch_tiles(self.h, g.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p),
                                            r.ctypes.data_as(C.c_void_p)))
        return {"grid": g.tolist(), "bc": b.tolist(), "grab": r.tolist()}

    def close(self):
        if getattr(self, "h", None):
            load().rsgdf_j3c_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rsgdf_j3c_batch(problems, kpairs, outs=None, **opt):
    """One-shot batched j3c; returns the list of outputs."""
    import torch
    lib = load()
    cells = [_cell(a, km) for (a, km, _, _) in problems]
    refs = [(_BasisRef(ao), _BasisRef(aux)) for (_, _, ao, aux) in problems]
    kp = [np.ascontiguousarray(np.asarray(k, dtype=np.int32).reshape(-1, 2)) for k in kpairs]
    n = len(problems)
    pr = (_Problem * n)()
    for p in range(n):
        pr[p].cell = C.cast(C.pointer(cells[p]), C.c_void_p)
        pr[p].ao = C.cast(C.pointer(refs[p][0].s), C.c_void_p)
        pr[p].aux = C.cast(C.pointer(refs[p][1].s), C.c_void_p)
    if outs is None:
        outs = [torch.zeros((len(kp[p]), refs[p][1].nfunc, refs[p][0].nfunc, refs[p][0].nfunc),
                            dtype=torch.complex128, device="cuda") for p in range(n)]
    npair = np.array([len(k) for k in kp], dtype=np.int32)
    kcat = np.ascontiguousarray(np.concatenate(kp).reshape(-1))
    o = _opts(**opt)
    ptrs = (C.c_void_p * n)(*[x.data_ptr() for x in outs])
    _check(lib.rsgdf_j3c_batch(n, C.cast(pr, C.c_void_p), C.byref(o), npair.ctypes.data_as(C.c_void_p),
                               kcat.ctypes.data_as(C.c_void_p), C.cast(ptrs, C.c_void_p)))
    return outs
