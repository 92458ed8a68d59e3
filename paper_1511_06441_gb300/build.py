"""Builds libcsp.so (the CUDA solver behind include/csp.h) in-tree for sm_103a.

    python -m paper_1511_06441_gb300.build        # or build() from Python

nvcc cross-compiles without a GPU; the library is placed next to this file.
"""
from __future__ import annotations

import json
import os
import shutil
import subprocess
import sys
import tempfile

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libcsp.so")
SOURCES = ["csp_solver.cu", "csp_event.cu", "csp_batch.cu", "csp_server.cu", "csp_info.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SHAPE_JSON = os.path.join(PKG, "shape.json")
# the block-shape build parameters and their defaults (csp_device.cuh, csp_batch.cu)
SHAPE_KEYS = {"tpb": ("CSP_TPB", 512), "ipt": ("CSP_IPT", 4), "nstage": ("CSP_NSTAGE", 3),
              "min_ctas_per_sm": ("CSP_MIN_CTAS_PER_SM", 2), "batch_min_ctas_per_sm": ("CSP_BATCH_MIN_CTAS_PER_SM", 1)}


def shape_flags(shape=None):
    """-D flags for a block shape (a dict of SHAPE_KEYS); None = the tuner's cached choice in
    shape.json, or the defaults without it."""
    if shape is None:
        shape = {}
        if os.path.exists(SHAPE_JSON):
            with open(SHAPE_JSON) as f:
                shape = json.load(f).get("chosen", {})
    flags = []
    for k, (macro, default) in SHAPE_KEYS.items():
        v = int(shape.get(k, default))
        if v <= 0:
            raise ValueError(f"shape {k} must be positive")
        flags.append(f"-D{macro}={v}")
    return flags


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


def build(force: bool = False, verbose: bool = False, shape=None, out: str = "") -> str:
    """Builds the library with the block shape `shape` (None: the cached choice) into `out`
    (default: libcsp.so next to this file)."""
    lib = out or LIB
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "csp.h")]
    if os.path.exists(SHAPE_JSON):
        deps.append(SHAPE_JSON)
    if not force and not _stale(lib, deps):
        return lib
    tmp = lib + f".tmp{os.getpid()}"
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
             *shape_flags(shape)]
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
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
