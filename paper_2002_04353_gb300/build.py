"""Builds the CUDA library in-tree: paper_2002_04353_gb300/_build/libalelb.so.

nvcc, one translation unit, sm_103a only.  Host code is compiled without
floating-point contraction so that the static map factors are the plain
IEEE results of the expressions as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc", "alelb.cu")
OUT = os.path.join(HERE, "_build", "libalelb.so")
DEPS = [os.path.join(HERE, "csrc", f) for f in ("alelb.cu", "geom.cuh", "kinetic.cuh", "kernels.cuh")] + [
    os.path.join(ROOT, "include", "alelb.h")]


def nvcc_cmd(out=OUT, extra=()):
    return ["nvcc", "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
            "-Xcompiler", "-fPIC,-ffp-contract=off", "-shared", "-I", os.path.join(ROOT, "include"),
            "-o", out, SRC, *extra]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    stale = not os.path.exists(OUT) or any(os.path.getmtime(d) > os.path.getmtime(OUT) for d in DEPS)
    if force or stale:
        tmp = OUT + f".{os.getpid()}.tmp"
        cmd = nvcc_cmd(tmp)
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
