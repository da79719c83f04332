"""Build libturbogs.so (the C-ABI library of CUDA kernels) in-tree for sm_103a.

    python -m paper_2412_13547_b300.build_native [--force]

nvcc cross-compiles without a GPU. The shared library statically links the
CUDA runtime and is loaded by ``paper_2412_13547_b300.raster`` via ctypes.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
HEADER = os.path.join(ROOT, "include", "turbogs.h")
LIB = os.path.join(PKG, "libturbogs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _newest_input() -> float:
    files = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [HEADER, os.path.abspath(__file__)]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu file to an object (in parallel, one nvcc each) and
    link them into the shared library; skipped when the library is newer than
    every source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    tag = ".tmp%d" % os.getpid()
    objs, procs = [], []
    for src in sources():
        obj = os.path.join(CSRC, os.path.basename(src)[:-3] + tag + ".o")
        cmd = [nvcc] + ARCH + FLAGS + ["-c", "-o", obj, src]
        if verbose:
            print(" ".join(cmd), flush=True)
        procs.append((subprocess.Popen(cmd, cwd=CSRC), cmd))
        objs.append(obj)
    try:
        for pr, cmd in procs:
            if pr.wait() != 0:
                raise subprocess.CalledProcessError(pr.returncode, cmd)
        tmp = LIB + tag
        subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs, check=True, cwd=CSRC)
        os.replace(tmp, LIB)
    finally:
        for pr, _ in procs:
            if pr.poll() is None:
                pr.kill()
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
