"""Build the CUDA library (librpca.so) in-tree with nvcc for sm_103a.

The library is plain C ABI (include/rpca.h); the Python side loads it with
ctypes.  Rebuilt when a source is newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "librpca.so")
GENCODE = "arch=compute_103a,code=sm_103a"
UNITS = ["rpca_batch_wide.cu", "rpca_batch_tc.cu", "rpca_wide.cu", "rpca_capi.cu", "rpca_batch.cu", "rpca_server.cu",
         "rpca_noalloc.cu", "rpca_prefilter.cu"]


def _sources():
    out = [os.path.join(ROOT, "include", "rpca.h")]
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librpca.so")


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile librpca.so if needed; return its path."""
    srcs = _sources()
    if not force and os.path.exists(LIB):
        lib_t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= lib_t for s in srcs):
            return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    tmp = LIB + ".tmp"
    # -dlcm=cg: global loads are cached in L2 only; persistent kernels read
    # control data that other CTAs rewrite while they run.
    flags = ["-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xptxas", "-dlcm=cg",
             "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    nvcc = nvcc_path()
    objs = []
    procs = []
    for f in UNITS:  # the units compile in parallel
        obj = os.path.join(LIBDIR, f.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc] + flags + ["-c", "-o", obj, os.path.join(CSRC, f)]
        if verbose:
            print(" ".join(cmd))
        procs.append((f, subprocess.Popen(cmd)))
    failed = [f for f, p in procs if p.wait() != 0]
    if failed:
        raise RuntimeError("nvcc failed on " + ", ".join(failed))
    cmd = [nvcc, "-gencode", GENCODE, "-shared", "-o", tmp] + objs
    if verbose:
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
