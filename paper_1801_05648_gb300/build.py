"""Build libfsi.so (the CUDA solver behind include/fsi.h) for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into a shared library next to this file.  Objects go to ``_build/``.
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
BUILD = os.path.join(ROOT, "_build", "fsi")
LIB = os.path.join(HERE, "libfsi.so")
SOURCES = ["spmv.cu", "vec.cu", "sparse_util.cu", "amg.cu", "solver.cu", "fsi_api.cu", "noalloc.cu", "coarse.cu", "learned.cu",
           "assembly.cu", "mlp_tc.cu"]
# throughput probes for the rooflines (include/fsi_peaks.h), a library of their own
PEAKS_LIB = os.path.join(HERE, "libfsi_peaks.so")
PEAKS_SOURCES = ["peaks.cu"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _flags(extra=()):
    return ["-O3", "-std=c++20", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
            "-I", os.path.join(ROOT, "include"), *extra]


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    deps.append(os.path.join(ROOT, "include", "fsi.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    jobs = []
    for src in SOURCES + PEAKS_SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(o, s):
            jobs.append((s, o))

    def run(job):
        s, o = job
        cmd = [cc, "-c", s, "-o", o + ".tmp", *_flags(extra)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(s)}:\n{r.stderr[-8000:]}")
        os.replace(o + ".tmp", o)
        return s, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs) or 1, os.cpu_count() or 4)) as ex:
        for s, err in ex.map(run, jobs):
            if verbose and err:
                print(f"[{os.path.basename(s)}]\n{err}", file=sys.stderr)
    rebuilt = {os.path.basename(src) for src, _ in jobs}
    for lib, srcs in ((LIB, SOURCES), (PEAKS_LIB, PEAKS_SOURCES)):
        objs = [os.path.join(BUILD, src.replace(".cu", ".o")) for src in srcs]
        if rebuilt & set(srcs) or not os.path.exists(lib):
            tmp = lib + f".tmp{os.getpid()}"
            cmd = [cc, "-shared", ARCH, "-o", tmp, *objs, "-lcudart"]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
