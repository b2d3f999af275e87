"""Build the C-ABI library ``_lib/libmds.so`` in-tree with nvcc for sm_103a.

Translation units are compiled in parallel, then linked into one shared
library (static CUDA runtime, so the library has no dependency beyond the
driver).  ``-Xptxas -v`` resource usage of every kernel is kept in
``_lib/ptxas.log``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libmds.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["pair_kernel.cu", "chunk_kernel.cu", "batch_kernel.cu", "reduce_kernel.cu", "heldout.cu", "noalloc.cu", "tree_prior.cu", "rwmh.cu", "ceiling.cu", "tree_plan.cpp", "api.cpp"]
HEADERS = ["mds_internal.h", "mills_ratio_coeffs.h", "pair_math.cuh", "philox.cuh", "tree_plan.h"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmds")
    return cand


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.join(LIBDIR, "obj"), exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "mds.h")]
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    objs = []
    for src in SOURCES:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(LIBDIR, "obj", src + ".o")
        objs.append(obj)
        if force or _stale(obj, [sp] + hdrs):
            cmd = [nvcc] + common + ["-Xptxas", "-v", "-c", sp, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [nvcc] + common + ["-x", "cu", "-c", sp, "-o", obj]
            jobs.append((src, cmd))
    logs = {}
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            futs = {ex.submit(subprocess.run, cmd, capture_output=True, text=True): src for src, cmd in jobs}
            for f in cf.as_completed(futs):
                src = futs[f]
                r = f.result()
                logs[src] = r.stdout + r.stderr
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}{r.stderr}")
        with open(os.path.join(LIBDIR, "ptxas.log"), "w") as fh:
            for src in sorted(logs):
                fh.write(f"==== {src}\n{logs[src]}\n")
    if force or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}{r.stderr}")
        os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
