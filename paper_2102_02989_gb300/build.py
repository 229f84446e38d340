"""Build the in-tree CUDA library ``_build/librsgdf.so`` for sm_103a.

nvcc compiles every ``csrc/*.cu`` (``-gencode arch=compute_103a,code=sm_103a``),
g++ the host planner; the objects are compiled in parallel and linked with the
shared CUDA runtime.  No cmake; a rebuild happens only when a source is newer
than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "librsgdf.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the RSGDF library needs the CUDA toolkit")


def _sources():
    cu = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cpp = sorted(glob.glob(os.path.join(CSRC, "*.cpp")))
    hdr = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return cu, cpp, hdr


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    cu, cpp, hdr = _sources()
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in cu + cpp + hdr + [__file__])


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    cu, cpp, _ = _sources()
    jobs = []
    for f in cu:
        o = os.path.join(BUILD, os.path.basename(f) + ".o")
        jobs.append(([nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                      "-I", INCLUDE, "-c", f, "-o", o, *extra], o))
    for f in cpp:
        o = os.path.join(BUILD, os.path.basename(f) + ".o")
        jobs.append((["g++", "-O2", "-std=c++17", "-fPIC", "-I", INCLUDE, "-c", f, "-o", o], o))

    def run(job):
        cmd, _ = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.returncode

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        rcs = list(ex.map(run, jobs))
    if any(rcs):
        raise RuntimeError("RSGDF library compilation failed")
    tmp = LIB + ".%d.tmp" % os.getpid()
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode:
        sys.stderr.write(" ".join(link) + "\n" + r.stdout + r.stderr)
        raise RuntimeError("RSGDF library link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
