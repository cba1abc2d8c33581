"""Build the QTAM CUDA library (libqtam.so) in-tree for sm_103a.

Each .cu file compiles to an object in parallel, then nvcc links the shared
library into ``paper_2603_29785_gb300/lib/``.  A rebuild happens only when a
source or header is newer than the library (or ``force=True``).
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
LIBDIR = os.path.join(HERE, "lib")
BUILDDIR = os.path.join(LIBDIR, "_build")
LIBNAME = "libqtam.so"
SOURCES = ["qtam_api.cu", "kernels_long.cu", "kernels_rows.cu", "qtam_noalloc.cu", "qtam_stream.cu",
           "kernels_tc.cu", "kernels_rows_stream.cu", "kernels_rows_dense.cu", "kernels_rows_pair.cu",
           "kernels_rows_tuned.cu"]
HEADERS = ["fft_core.cuh", "fft_static.cuh", "qtam_internal.h", "tc_sm100.cuh", "rows_common.cuh", "pair_fft.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
                "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the QTAM library needs the CUDA toolkit to build")


def lib_path() -> str:
    return os.path.join(LIBDIR, LIBNAME)


def _inputs():
    yield from (os.path.join(CSRC, s) for s in SOURCES + HEADERS)
    yield os.path.join(ROOT, "include", "qtam.h")
    yield os.path.abspath(__file__)


def up_to_date() -> bool:
    lp = lib_path()
    if not os.path.exists(lp):
        return False
    t = os.path.getmtime(lp)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def _run(cmd, verbose):
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"command failed ({r.returncode}): {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stdout + r.stderr


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    """Compile and link libqtam.so; returns its path."""
    if not force and up_to_date():
        return lib_path()
    os.makedirs(BUILDDIR, exist_ok=True)
    cc = nvcc()
    objs = []
    jobs = []
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for s in SOURCES:
            obj = os.path.join(BUILDDIR, s.replace(".cu", ".o"))
            objs.append(obj)
            cmd = [cc, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, s), "-o", obj]
            jobs.append(ex.submit(_run, cmd, verbose))
        outs = [j.result() for j in jobs]
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = lib_path() + ".tmp"
    _run([cc, *ARCH, "-shared", "-o", tmp, *objs], verbose)
    os.replace(tmp, lib_path())
    return lib_path()


if __name__ == "__main__":
    v = "-v" in sys.argv
    f = "-f" in sys.argv or "--force" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=f or bool(extra), verbose=v or bool(extra), extra_flags=extra))
