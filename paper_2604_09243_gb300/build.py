"""In-tree build of libsbr.so for sm_103a (GB300) with nvcc.

Each translation unit is compiled in parallel, then linked into
``paper_2604_09243_gb300/lib/libsbr.so``. Host code is compiled without
floating-point contraction because the aperture-grid convention (Eq. L1-L3)
fixes its FP64 arithmetic order.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libsbr.so")
OBJDIR = os.path.join(ROOT, "_build", "sbr")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsbr")
    return p


def _flags(verbose_ptx: bool):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
                "-I", os.path.join(ROOT, "include")]
    if verbose_ptx:
        f += ["-Xptxas", "-v"]
    return f


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.h"))) + [os.path.join(ROOT, "include", "sbr.h")]


def build(force: bool = False, verbose_ptx: bool = False, jobs: int | None = None) -> str:
    """Compile and link libsbr.so; returns its path. Skips work when up to date."""
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in _deps()):
            return LIB
    os.makedirs(OBJDIR, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nv = nvcc()
    srcs = _sources()
    objs = [os.path.join(OBJDIR, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def compile_one(sv):
        s, o = sv
        r = subprocess.run([nv] + _flags(verbose_ptx) + ["-c", s, "-o", o], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with cf.ThreadPoolExecutor(max_workers=jobs or min(8, len(srcs))) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose_ptx:
        for s, lg in zip(srcs, logs):
            print(f"== {os.path.basename(s)}\n{lg}")
    tmp = LIB + ".tmp"
    r = subprocess.run([nv] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose_ptx="-v" in sys.argv))
