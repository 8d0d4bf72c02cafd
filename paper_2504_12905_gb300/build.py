"""Build liblmrs.so (the CUDA hot path behind include/lmrs.h) in-tree.

Every translation unit is compiled by nvcc for sm_103a only, in parallel,
then linked into ``paper_2504_12905_gb300/_build/liblmrs.so``.  Host code is
compiled with FP contraction disabled (the FP32 list decisions depend on it).
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
OUT_DIR = os.path.join(HERE, "_build")
# the bounds-checked build (LMRS_DEBUG, see include/lmrs.h), beside the release one
OUT_DIR_DEBUG = os.path.join(HERE, "_build_debug")
LIB_NAME = "liblmrs.so"
# hotpath.cu includes preprocess.cu, raster.cu and cg.cu (one translation unit)
SOURCES = ["scene.cu", "hotpath.cu", "binning.cu", "noalloc.cu", "autotune.cu", "server.cu", "view_sampler.cu",
           "peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblmrs")


def library_path(debug: bool = False) -> str:
    return os.path.join(OUT_DIR_DEBUG if debug else OUT_DIR, LIB_NAME)


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
                   "-I" + INCLUDE, "-I" + CSRC] + list(extra)


def _stamp_inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lmrs.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(verbose: bool = False, force: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Builds the library (debug: the bounds-checked LMRS_DEBUG build into
    _build_debug/) unless it is newer than every source; returns its path."""
    out_dir = OUT_DIR_DEBUG if debug else OUT_DIR
    if debug:
        extra_flags = tuple(extra_flags) + ("-DLMRS_DEBUG",)
    os.makedirs(out_dir, exist_ok=True)
    out = library_path(debug)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _stamp_inputs():
        return out
    nv = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        cmd = [nv, "-c", os.path.join(CSRC, src), "-o", obj] + _flags(extra_flags)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nv, "-shared", "-o", tmp] + objs + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv))
