"""Build the solver's shared library (C ABI of include/mg.h) for sm_103a with nvcc.

The library is built in-tree under ``paper_0805_3041_gb300/_build/``; the
translation units compile in parallel and are linked with ``nvcc -shared``.
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
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmg_gb300.so")
# the checking build (-DMG_DEBUG: device-side bounds checks that report MG_EBOUNDS)
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(BUILD_DEBUG, "libmg_gb300_debug.so")
SOURCES = ["mg_capi.cu", "kernels_point.cu", "kernels_transfer.cu", "kernels_line.cu", "kernels_coarse.cu",
           "kernels_fast.cu", "kernels_xline.cu", "kernels_march.cu", "kernels_tma.cu", "noalloc.cu",
           "kernels_cg.cu", "kernels_batch.cu", "kernels_ff.cu"]
HEADERS = ["mg_internal.cuh", "coarse_prog.h", "batch_prog.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the solver")


def _inputs():
    out = [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    hdrs = [os.path.join(CSRC, h) for h in HEADERS if os.path.exists(os.path.join(CSRC, h))]
    hdrs.append(os.path.join(ROOT, "include", "mg.h"))
    return out, hdrs


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    srcs, hdrs = _inputs()
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(f) <= t for f in srcs + hdrs + [__file__])


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Build the library (debug=True: the checking build, into its own folder and file)."""
    lib, bdir = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if not force and up_to_date(debug):
        return lib
    os.makedirs(bdir, exist_ok=True)
    srcs, _ = _inputs()
    cc = nvcc()
    objs = []
    mode = ["-DMG_DEBUG"] if debug else []

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *FLAGS, *mode, *extra_flags, "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, debug="--debug" in sys.argv))
