"""Build the in-tree shared libraries of the package.

    python -m paper_2607_20766_b300.build            # libshape.so + libmolgen.so

libshape.so is compiled for sm_103a only (B300); nvcc cross-compiles it on a
machine without a GPU.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libshape.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_shape(force: bool = False, verbose: bool = False) -> str:
    deps = sources() + glob.glob(os.path.join(HERE, "csrc", "*.h*")) + [os.path.join(ROOT, "include", "shape.h")]
    if not force and not _stale(LIB, deps):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-fopenmp", "-lgomp", "-I", os.path.join(ROOT, "include"),
           "-o", tmp, *sources()]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


def main() -> None:
    from . import synth
    build_shape(force="--force" in sys.argv, verbose="-v" in sys.argv)
    synth.build(force="--force" in sys.argv)
    print(LIB)


if __name__ == "__main__":
    main()
