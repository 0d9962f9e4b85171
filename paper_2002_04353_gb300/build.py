"""Builds the CUDA library in-tree: paper_2002_04353_gb300/_build/libalelb.so.

nvcc, sm_103a only; the translation units compile in parallel and link into
one shared library.  Host code is compiled without
floating-point contraction so that the static map factors are the plain
IEEE results of the expressions as written.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
UNITS = [os.path.join(CSRC, f) for f in ("alelb.cu", "batch.cu", "mlp.cu", "checkpoint.cu", "quad.cu")]
OUT = os.path.join(HERE, "_build", "libalelb.so")
DEPS = UNITS + [os.path.join(CSRC, f) for f in ("geom.cuh", "kinetic.cuh", "kernels.cuh", "tables.h",
                                                 "internal.h", "mlp.cuh", "quad.cuh", "quad_tables.h")] + [
    os.path.join(ROOT, "include", "alelb.h")]
FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
         "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", os.path.join(ROOT, "include")]


def nvcc_cmd(out=OUT, extra=()):
    """One-shot command (all units in one nvcc call), e.g. for -Xptxas -v."""
    return ["nvcc", *FLAGS, "-shared", "-o", out, *UNITS, *extra]


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    stale = not os.path.exists(OUT) or any(os.path.getmtime(d) > os.path.getmtime(OUT) for d in DEPS)
    if force or stale:
        tag = f"{os.getpid()}"
        objs = [os.path.join(os.path.dirname(OUT), os.path.basename(u) + f".{tag}.o") for u in UNITS]
        procs = []
        for u, o in zip(UNITS, objs):
            cmd = ["nvcc", *FLAGS, "-c", "-o", o, u]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            procs.append(subprocess.Popen(cmd))
        codes = [p.wait() for p in procs]
        if any(codes):
            raise subprocess.CalledProcessError(max(codes), "nvcc")
        tmp = OUT + f".{tag}.tmp"
        subprocess.run(["nvcc", "-shared", "-o", tmp, *objs], check=True)
        for o in objs:
            os.remove(o)
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
