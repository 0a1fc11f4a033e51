"""Compile libwt.so (sm_103a) in-tree with nvcc, and its debug twin
libwt_debug.so (the same sources with WT_DEBUG_BOUNDS=1: bounds-checked walk
loads that report WT_EBOUNDS).

Each translation unit under csrc/ is compiled in parallel into _build/ (and
_build/debug/), then linked.  No CMake; one -gencode.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwt.so")
SOURCES = ["wt_build.cu", "wt_query.cu", "wt_api.cu", "wt_learned.cu", "wt_batch.cu", "wt_noalloc.cu", "wt_bitvec.cu", "wt_alphabet.cu"]
HEADERS = ["wt_common.cuh", "wt_internal.hpp", "wt_walk.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libwt needs the CUDA toolkit to build")


def _flags():
    return ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


VARIANTS = {
    # name: (library, object directory, extra nvcc flags)
    "release": (LIB, OBJDIR, []),
    # every load of a query walk checked against its array's length (WT_EBOUNDS)
    "debug": (os.path.join(HERE, "libwt_debug.so"), os.path.join(OBJDIR, "debug"), ["-DWT_DEBUG_BOUNDS=1"]),
}


def build(force: bool = False, verbose: bool = False, extra_flags=(), variants=("release", "debug")) -> str:
    """Compile the requested variants (translation units of all of them in one
    parallel pool) and link each library; returns the release library's path."""
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "wt.h")]
    jobs = []
    links = []
    for v in variants:
        lib, objdir, vflags = VARIANTS[v]
        os.makedirs(objdir, exist_ok=True)
        objs = []
        for src in SOURCES:
            s = os.path.join(CSRC, src)
            o = os.path.join(objdir, src.replace(".cu", ".o"))
            objs.append(o)
            if force or _stale(o, [s] + hdrs):
                jobs.append([nvcc(), *_flags(), *vflags, *extra_flags, "-c", s, "-o", o])
        links.append((lib, objs))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(jobs), max(os.cpu_count() or 1, 1))) as ex:
            list(ex.map(run, jobs))
    for lib, objs in links:
        if force or jobs or _stale(lib, objs):
            tmp = lib + ".tmp%d" % os.getpid()
            run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs])
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose=True))
