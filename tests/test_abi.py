"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/rsgdf.h declares; argument errors come back as status codes before
any device work (so they are checked without a GPU); the host-side omega /
G-mesh rule agrees with its restatement in the tests."""
import os
import re

import numpy as np
import pytest

from paper_2102_02989_gb300 import inputs
from rules_ref import gmesh_for, omega_for

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rs():
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    return rsgdf


def test_header_symbols_exported(rs):
    hdr = open(os.path.join(ROOT, "include", "rsgdf.h")).read()
    names = set(re.findall(r"^\s*(?:int|const char \*)\s*(rsgdf_\w+)\s*\(", hdr, re.M))
    assert names, "no declarations found"
    lib = rs.load()
    for n in names:
        assert hasattr(lib, n), n
    assert names <= set(rs.EXPORTS)


def test_params_rule_matches(rs):
    for p in (inputs.config1(), inputs.config2(), inputs.config2((4, 4, 4))):
        if p.omega:
            w, gm = rs.rsgdf_params(p.a, p.kmesh, omega=p.omega, eps_lr=p.eps_lr)
            assert gm == gmesh_for(p.a, p.omega, p.eps_lr, p.kmesh)
        else:
            w, gm = rs.rsgdf_params(p.a, p.kmesh, gmesh=p.gmesh, eps_lr=p.eps_lr)
            assert abs(w - omega_for(p.a, p.gmesh, p.eps_lr, p.kmesh)) < 1e-14


@pytest.mark.parametrize("bad", ["npair", "kidx", "shells", "eps", "gmesh_even", "lmax", "exp"])
def test_argument_errors_without_device(rs, bad):
    p = inputs.tiny()
    kw = dict(omega=0.9, eps_screen=1e-10, eps_lr=1e-10)
    kp, sh, ao = [(0, 0)], None, p.ao
    if bad == "kidx":
        kp = [(0, 3)]
    if bad == "shells":
        sh = (2, 2)
    if bad == "eps":
        kw["eps_screen"] = 0.0
    if bad == "gmesh_even":
        kw["gmesh"] = (6, 7, 7)
    if bad == "lmax":
        ao = inputs.make_basis([(4, (0, 0, 0), [1.0], [1.0])])
    if bad == "exp":
        ao = inputs.make_basis([(0, (0, 0, 0), [-1.0], [1.0])])
    lib = rs.load()
    import ctypes as C
    ra, rx = rs._BasisRef(ao), rs._BasisRef(p.aux)
    o = rs._Opts()
    o.omega, o.eps_screen, o.eps_lr = kw["omega"], kw["eps_screen"], kw["eps_lr"]
    for i in range(3):
        o.gmesh[i] = kw.get("gmesh", (0, 0, 0))[i]
    c = rs._cell(p.a, (1, 1, 1))
    kpa = np.ascontiguousarray(np.asarray(kp, np.int32).reshape(-1, 2))
    npair = 0 if bad == "npair" else len(kpa)
    s0, s1 = sh if sh else (0, len(rx.l))
    rc = lib.rsgdf_j3c(C.byref(c), ra.ref(), rx.ref(), C.byref(o), npair, kpa.ctypes.data_as(C.c_void_p), s0, s1,
                       C.c_void_p(16))
    assert rc == rs.RSGDF_EINVAL, (bad, rc, rs.rsgdf_last_error())
    assert rs.rsgdf_last_error() != ""


def test_python_constants_match_header(rs):
    hdr = open(os.path.join(ROOT, "include", "rsgdf.h")).read()
    defs = dict(re.findall(r"^#define (RSGDF_\w+) \(?(-?\d+)", hdr, re.M))
    for name in ("RSGDF_FIT_CHOLESKY", "RSGDF_FIT_EIGEN", "RSGDF_FIT_AUTO", "RSGDF_DF_NMAX", "RSGDF_DF_SWEEPS",
                 "RSGDF_FP64", "RSGDF_MIXED", "RSGDF_EINVAL"):
        assert int(defs[name]) == getattr(rs, name), name


@pytest.mark.parametrize("bad", ["naux0", "naux_big", "method", "rel", "overlap", "nullT"])
def test_df_metric_argument_errors_without_device(rs, bad):
    import ctypes as C
    lib = rs.load()
    naux, nk, method, rel = 8, 2, rs.RSGDF_FIT_AUTO, 1e-6
    J, T = C.c_void_p(1 << 20), C.c_void_p(1 << 30)
    if bad == "naux0":
        naux = 0
    if bad == "naux_big":
        naux = rs.RSGDF_DF_NMAX + 1
    if bad == "method":
        method = 3
    if bad == "rel":
        rel = 1.0
    if bad == "overlap":
        T = C.c_void_p((1 << 20) + 16)
    if bad == "nullT":
        T = C.c_void_p(0)
    rc = lib.rsgdf_df_metric(J, naux, nk, method, rel, T, None, None, None, None)
    assert rc == rs.RSGDF_EINVAL, (bad, rc, rs.rsgdf_last_error())


@pytest.mark.parametrize("bad", ["kidx", "npair", "overlap", "dup", "noout"])
def test_df_fit_jk_argument_errors_without_device(rs, bad):
    import ctypes as C
    lib = rs.load()
    c = rs._cell(4.0 * np.eye(3), (2, 1, 1))
    kp = [(0, 0), (0, 1), (1, 1)]
    if bad == "kidx":
        kp = [(0, 2)]
    if bad == "dup":
        kp = [(0, 1), (0, 1)]
    kpa = np.ascontiguousarray(np.asarray(kp, np.int32).reshape(-1, 2))
    npair = 0 if bad == "npair" else len(kpa)
    ptr = lambda x: C.c_void_p(x)
    naux, nao = 8, 3
    V, Bo = 1 << 20, 1 << 30
    if bad == "overlap":
        Bo = V + 16
    if bad in ("kidx", "npair", "overlap"):
        rc = lib.rsgdf_df_fit(C.byref(c), ptr(1 << 34), naux, nao, npair, kpa.ctypes.data_as(C.c_void_p), ptr(V),
                              ptr(Bo), None)
        assert rc == rs.RSGDF_EINVAL, (bad, rc, rs.rsgdf_last_error())
    if bad in ("kidx", "npair", "dup", "noout"):
        out = ptr(0) if bad == "noout" else ptr(1 << 36)
        rc = lib.rsgdf_df_jk(C.byref(c), ptr(V), naux, nao, npair, kpa.ctypes.data_as(C.c_void_p), ptr(1 << 35),
                             ptr(0), out, ptr(0), None)
        assert rc == rs.RSGDF_EINVAL, (bad, rc, rs.rsgdf_last_error())
        if bad == "noout":
            return
        rc = lib.rsgdf_df_rho(C.byref(c), ptr(V), naux, nao, npair, kpa.ctypes.data_as(C.c_void_p), ptr(1 << 35),
                              ptr(1 << 36), None)
        assert rc == rs.RSGDF_EINVAL, (bad, rc, rs.rsgdf_last_error())


def test_sph_coefficients_match_the_oracle(rs):
    from oracle import sph
    for l in range(4):
        assert np.max(np.abs(rs.rsgdf_sph_coefficients(l) - sph.coefficients(l))) < 1e-13
    p = inputs.tiny(lmax_ao=2, lmax_aux=3)
    assert rs.rsgdf_sph_nfunc(p.aux) == sum(2 * int(l) + 1 for l in p.aux.l)


@pytest.mark.parametrize("bad", ["l", "range", "npair", "overlap", "nk"])
def test_cart2sph_argument_errors_without_device(rs, bad):
    import ctypes as C
    lib = rs.load()
    if bad == "l":
        assert lib.rsgdf_sph_coefficients(4, C.c_void_p(16)) == rs.RSGDF_EINVAL
        return
    p = inputs.tiny(lmax_ao=1, lmax_aux=2)
    ra, rx = rs._BasisRef(p.ao), rs._BasisRef(p.aux)
    if bad == "nk":
        assert lib.rsgdf_cart2sph_j2c(rx.ref(), 0, C.c_void_p(1 << 20), C.c_void_p(1 << 30), None) == rs.RSGDF_EINVAL
        return
    s0, s1, npair, out = 0, len(rx.l), 2, 1 << 30
    if bad == "range":
        s1 = len(rx.l) + 1
    if bad == "npair":
        npair = 0
    if bad == "overlap":
        out = (1 << 20) + 32
    rc = lib.rsgdf_cart2sph_j3c(ra.ref(), rx.ref(), s0, s1, npair, C.c_void_p(1 << 20), C.c_void_p(out), None)
    assert rc == rs.RSGDF_EINVAL, (bad, rc, rs.rsgdf_last_error())


@pytest.mark.parametrize("bad", ["alpha", "plain_j3c", "plain_sr", "kernel"])
def test_split_options_rejected_without_device(rs, bad):
    import ctypes as C
    lib = rs.load()
    p = inputs.tiny()
    ra, rx = rs._BasisRef(p.ao), rs._BasisRef(p.aux)
    o = rs._opts(omega=0.9, eps_screen=1e-10, eps_lr=1e-10)
    name = "rsgdf_j3c"
    if bad == "alpha":
        o.split_alpha = -1.0
    if bad == "plain_j3c":
        o.kernel = rs.RSGDF_KERNEL_PLAIN
    if bad == "plain_sr":
        o.kernel, name = rs.RSGDF_KERNEL_PLAIN, "rsgdf_j3c_sr"
    if bad == "kernel":
        o.kernel = 7
    c = rs._cell(p.a, (1, 1, 1))
    kpa = np.zeros((1, 2), np.int32)
    rc = getattr(lib, name)(C.byref(c), ra.ref(), rx.ref(), C.byref(o), 1, kpa.ctypes.data_as(C.c_void_p), 0,
                            len(rx.l), C.c_void_p(16))
    assert rc == rs.RSGDF_EINVAL, (bad, rc, rs.rsgdf_last_error())


def test_error_control_arguments_without_device(rs):
    lib = rs.load()
    assert lib.rsgdf_set_scratch_limit(-1) == rs.RSGDF_EINVAL
    assert lib.rsgdf_set_scratch_limit(0) == rs.RSGDF_OK
    assert lib.rsgdf_selftest_wait(0, 0, None) == rs.RSGDF_EINVAL
    assert "limit" in rs.rsgdf_last_error()
