"""Builds libufg.so in-tree for sm_103a with nvcc (no cmake): one object per translation unit,
compiled in parallel, the slice kernels once per supported N_x."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libufg.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SLICE_N = (4, 6, 8, 10, 12, 16, 32)
UNITS = ["lattice.cu", "recurrence.cu", "dispatch.cu", "blas.cu", "solvers.cu", "batch.cu",
         "noalloc.cu", "profile.cu", "series.cu"]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(verbose=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if verbose:
        f += ["-Xptxas", "-v"]
    extra = os.environ.get("UFG_NVCC_FLAGS", "").split()
    return f + extra


def _jobs():
    jobs = []
    for u in UNITS:
        src = os.path.join(CSRC, u)
        if os.path.exists(src):
            jobs.append((src, os.path.join(BUILD, u.replace(".cu", ".o")), []))
    for n in SLICE_N:
        jobs.append((os.path.join(CSRC, "slice_inst.cu"), os.path.join(BUILD, "slice_n%d.o" % n),
                     ["-DUFG_N=%d" % n]))
    return jobs


def build(verbose=False, force=False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "ufg.h"))
    hdr_time = max(os.path.getmtime(h) for h in headers)

    def compile_one(job):
        src, obj, extra = job
        if (not force and os.path.exists(obj) and os.path.getmtime(obj) > os.path.getmtime(src)
                and os.path.getmtime(obj) > hdr_time):
            return obj, ""
        cmd = [cc] + _flags(verbose) + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (obj, r.stdout, r.stderr))
        return obj, r.stderr
    jobs = _jobs()
    with ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose:
        for obj, log in results:
            if log:
                sys.stderr.write("== %s\n%s" % (os.path.basename(obj), log))
    objs = [o for o, _ in results]
    if force or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [cc] + ARCH + ["-shared", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
