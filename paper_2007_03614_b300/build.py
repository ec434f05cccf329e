"""Build the in-tree native libraries: libmanta.so (CUDA, sm_103a), its
fast-math variant libmanta_fast.so, and the synthetic-input generator.
Cross-compiles without a GPU."""
from __future__ import annotations

import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libmanta.so")
LIB_FAST = os.path.join(PKG, "libmanta_fast.so")

# The product build is the bit-exact build: no FMA contraction, IEEE division
# and square root.  The path is memory-bound, so this costs nothing measurable.
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
              "-Xcompiler", "-fPIC,-fvisibility=hidden", "-shared"]

# The fast-math variant: FMA contraction, approximate division and square
# root, flush-to-zero.  Same sources and ABI; its trajectories agree with the
# bit-exact build to within the tolerance tested, not bit for bit.
NVCC_FAST_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
                   "--use_fast_math", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-shared"]

SOURCES = ["manta.cu"]
DEPS = ["manta.cu", "sim.cuh", "step_kernel.cuh", "adjoint.cuh"]


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


# Test builds of the same sources: each defines compile-time knobs that move
# the kernel onto paths the product build only takes at sizes a parity test
# cannot afford (a lane-change candidate list that overflows shared memory),
# select the non-default leader-walk batch sizes, or check every device write
# index.  Same ABI; results must equal the product build's bit for bit.
VARIANTS = {
    "lccap": ["-DMANTA_LC_CAP=4"],
    "walk8": ["-DMANTA_WALK_CHUNKS=8", "-DMANTA_FIRST_CHUNKS=4"],
    "walk16": ["-DMANTA_WALK_CHUNKS=16", "-DMANTA_FIRST_CHUNKS=8"],
    # index checks on every device write of the step kernel (manta_debug_checks)
    "check": ["-DMANTA_CHECK_BOUNDS"],
}


def variant_path(name: str) -> str:
    return os.path.join(PKG, f"libmanta_{name}.so")


def build_variant(name: str, force: bool = False) -> str:
    """Build the test variant `name` of libmanta.so (product flags plus its
    defines) and return its path."""
    out = variant_path(name)
    deps = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(INCLUDE, "manta.h"), os.path.abspath(__file__)]
    if force or _stale(out, deps):
        subprocess.check_call(["nvcc", *NVCC_FLAGS, *VARIANTS[name], "-I", INCLUDE, "-o", out,
                               *[os.path.join(CSRC, s) for s in SOURCES]])
    return out


def build(force: bool = False, verbose: bool = False, fast: bool = True) -> str:
    deps = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(INCLUDE, "manta.h")]
    todo = [(LIB, NVCC_FLAGS)] + ([(LIB_FAST, NVCC_FAST_FLAGS)] if fast else [])
    for out, flags in todo:
        if force or _stale(out, deps):
            cmd = ["nvcc", *flags, "-I", INCLUDE, "-o", out, *[os.path.join(CSRC, s) for s in SOURCES]]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            subprocess.check_call(cmd)
    from . import synth
    synth.build(force=force)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
