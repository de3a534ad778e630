"""Build the CUDA libraries in-tree for sm_103a (nvcc, no GPU needed).

libhetm.so          -- the round library (csrc/*.cu), the C ABI of include/hetm.h
libhetm_testing.so  -- measurement probes (csrc_testing/*.cu), include/hetm_testing.h
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libhetm.so")
LIB_TESTING = os.path.join(HERE, "libhetm_testing.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources(sub="csrc"):
    return sorted(glob.glob(os.path.join(HERE, sub, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cuh")) +
                  glob.glob(os.path.join(ROOT, "include", "*.h")))


def stale(lib, srcs) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in srcs + headers())


def _nvcc(lib, srcs, verbose):
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-fvisibility=hidden", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(HERE, "csrc"), *srcs, "-o", lib + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)


def build(force: bool = False, verbose: bool = False) -> str:
    for lib, sub in ((LIB, "csrc"), (LIB_TESTING, "csrc_testing")):
        srcs = sources(sub)
        if force or stale(lib, srcs):
            _nvcc(lib, srcs, verbose)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
