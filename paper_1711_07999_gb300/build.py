"""Builds libtrk.so (the CUDA kernels and the C ABI of include/trk.h) in-tree for sm_103a with nvcc.

Translation units compile in parallel; the shared library links the CUDA runtime statically.  Host code
is compiled without floating-point contraction so that the neighbourhood search gives the same ties on
every host architecture; device code without implicit multiply-add contraction, so that a session
computes bit for bit the same through its own launches and through a batch's.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libtrk.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["kernels_geom.cu", "kernels_solve.cu", "kernels_jtj.cu", "kernels_tc.cu", "trk_api.cu", "server.cu", "batch.cu",
           "schedule.cu", "authoring.cu"]
DEPS = ["trk_internal.cuh", "tcgen05.cuh", os.path.join(ROOT, "include", "trk.h")]
# -fmad=false: no implicit multiply-add contraction in device code (the FMAs the kernels want are written
# as fmaf), so a stage body inlined into different kernels rounds identically everywhere.
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo", "-fmad=false",
              "-Xcompiler", "-fPIC,-ffp-contract=off", "-diag-suppress", "177"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    raise RuntimeError("nvcc not found")


def _mtime(p):
    return os.path.getmtime(p) if os.path.exists(p) else 0.0


def build(force: bool = False, verbose: bool = False) -> str:
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, d) if not os.path.isabs(d) else d for d in DEPS]
    newest = max(_mtime(p) for p in deps + [__file__])
    if not force and _mtime(LIB) > newest:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc] + NVCC_FLAGS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout, r.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
