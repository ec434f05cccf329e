"""Build the in-tree native libraries: libmanta.so (CUDA, sm_103a) and the
synthetic-input generator.  Cross-compiles without a GPU."""
from __future__ import annotations

import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libmanta.so")

# The product build is the bit-exact build: no FMA contraction, IEEE division
# and square root.  The path is memory-bound, so this costs nothing measurable.
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
              "-Xcompiler", "-fPIC,-fvisibility=hidden", "-shared"]

SOURCES = ["manta.cu"]
DEPS = ["manta.cu", "sim.cuh", "step_kernel.cuh"]


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    deps = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(INCLUDE, "manta.h")]
    if force or _stale(LIB, deps):
        cmd = ["nvcc", *NVCC_FLAGS, "-I", INCLUDE, "-o", LIB, *[os.path.join(CSRC, s) for s in SOURCES]]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        subprocess.check_call(cmd)
    from . import synth
    synth.build(force=force)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
