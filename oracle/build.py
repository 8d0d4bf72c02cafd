"""Compile the FP64 oracle (test infrastructure) into ``oracle/_build``.

Plain g++ with OpenMP.  ``-ffp-contract=off`` keeps every floating-point
operation separately rounded, which the FP32 list decisions and the
double/dual instantiations of the forward model rely on.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "lmrs_oracle.cpp")


def library_path() -> str:
    return os.path.join(OUT_DIR, "liblmrs_oracle.so")


def build(verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    out = library_path()
    if os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "lmrs_oracle.h"))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-Wall", "-o", tmp, SRC]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(verbose=True))
