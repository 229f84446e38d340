"""The host planner's worker pool: plans made from two host threads at once,
many times over, all equal a serial plan (CPU only; the planner and a small
driver are compiled here with g++).

A worker that joined a parallel loop after its caller had returned could take
indices of the next loop and leave some of its entries uncomputed: a rare
race that changed SR screening radii, and with them j3c results, from one
call to the next."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2102_02989_gb300 import inputs, rsgdf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2102_02989_gb300", "csrc")


@pytest.fixture(scope="module")
def stress_lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    out = str(tmp_path_factory.mktemp("planner") / "libplanner_stress.so")
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           os.path.join(CSRC, "planner.cpp"), os.path.join(ROOT, "tests", "native", "planner_stress.cpp"),
           "-o", out, "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    lib = C.CDLL(out)
    lib.planner_stress.restype = C.c_int
    return lib


def test_concurrent_plans_equal_the_serial_plan(stress_lib):
    p = inputs.config2((2, 2, 2))
    omega, _ = rsgdf.rsgdf_params(p.a, p.kmesh, gmesh=p.gmesh, eps_lr=p.eps_lr)
    cell = rsgdf._cell(p.a, p.kmesh)
    ao, aux = rsgdf._BasisRef(p.ao), rsgdf._BasisRef(p.aux)
    bad = stress_lib.planner_stress(C.byref(cell), ao.ref(), aux.ref(), C.c_double(omega), C.c_double(p.eps_sr), 300)
    assert bad == 0
