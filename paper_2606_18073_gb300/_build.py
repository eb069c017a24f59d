"""In-tree build of the CUDA library libsgks.so (sm_103a) with nvcc.

The library exposes the C ABI declared in include/sgks.h.  Each translation unit is compiled
in parallel, then linked into one shared object next to this file.  No PyTorch headers are
involved: the library takes plain device pointers and a cudaStream_t.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libsgks.so")
SOURCES = ["k_sketch.cu", "k_small.cu", "k_small2.cu", "k_fp32x.cu", "k_bulk.cu", "k_setup.cu", "k_batch.cu",
           "k_adjoint.cu", "k_gks.cu", "k_conv.cu", "k_batchx.cu", "k_tiles.cu", "sgks_api.cu", "sgks_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-I" + os.path.join(ROOT, "include")]


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the sGKS CUDA library cannot be built")


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libsgks.so if any source is newer than it; return its path."""
    nvcc = _nvcc()
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    headers = [os.path.join(CSRC, "sgks_internal.cuh"), os.path.join(CSRC, "ff.cuh"), os.path.join(CSRC, "batch_common.cuh"), os.path.join(ROOT, "include", "sgks.h")]
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(objdir, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc, *ARCH, *FLAGS, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(objdir, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or _stale(LIB, objs):
        run([nvcc, *ARCH, "-shared", "-Xlinker", "--no-undefined", *objs, "-o", LIB + ".tmp"])
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
