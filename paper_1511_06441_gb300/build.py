"""Builds libcsp.so (the CUDA solver behind include/csp.h) in-tree for sm_103a.

    python -m paper_1511_06441_gb300.build        # or build() from Python

nvcc cross-compiles without a GPU; the library is placed next to this file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import tempfile

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libcsp.so")
SOURCES = ["csp_solver.cu", "csp_event.cu", "csp_batch.cu", "csp_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "csp.h")]
    if not force and not _stale(LIB, deps):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.append("-Xptxas=-v")
    tmpdir = tempfile.mkdtemp(prefix="csp_build_")
    objs = []
    procs = []
    for src in SOURCES:  # one translation unit per process, compiled in parallel
        obj = os.path.join(tmpdir, src.replace(".cu", ".o"))
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc(), *flags, "-c", "-o", obj, os.path.join(CSRC, src)]))
    codes = [p.wait() for p in procs]
    try:
        if any(codes):
            raise subprocess.CalledProcessError(max(codes), "nvcc")
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp] + objs)
    finally:
        shutil.rmtree(tmpdir, ignore_errors=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
