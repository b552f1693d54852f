"""Build ``libgplhr.so`` (the CUDA hot path and its C ABI) for sm_103a, in tree.

    python -m paper_1506_06829_gb300.build

Translation units are compiled in parallel with nvcc and linked into
``paper_1506_06829_gb300/libgplhr.so``.  No PyTorch headers are involved: the
library's interface is plain C (``include/gplhr.h``).
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libgplhr.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["gplhr.cu", "qz.cpp"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17", "-lineinfo",
           "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")] + ARCH
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-warn-spills"]
    else:
        # host QZ: plain complex multiply/divide formulas, without the Inf/NaN recovery and
        # overflow-avoiding scaling of the default ones (12-16 % faster); the QZ only sees
        # finite pencils, non-finite ones are rejected before it, and entries far below 1e150
        cmd += ["-Xcompiler", "-fcx-limited-range"]
    subprocess.run(cmd, check=True)
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    cmd = [nvcc(), "-shared", "-o", OUT] + objs + ARCH + ["-lcudart"]
    subprocess.run(cmd, check=True)
    if verbose:
        print("built", OUT)
    return OUT


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
