"""Build the CUDA library libal.so in-tree for sm_103a (B300).

    python -m paper_2609_39443_b300.build
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libal.so")
SOURCES = [os.path.join(HERE, "csrc", "al_api.cu"), os.path.join(HERE, "csrc", "al_serve.cu"),
           os.path.join(HERE, "csrc", "al_noalloc.cu")]
HEADERS = [os.path.join(HERE, "csrc", "al_kernels.cuh"), os.path.join(HERE, "csrc", "al_cm.cuh"),
           os.path.join(ROOT, "include", "al.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in SOURCES + HEADERS)


def build(verbose: bool = False, extra=()) -> str:
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"),
           "-Xptxas", "-v" if verbose else "-O3", *extra, "-o", tmp, *SOURCES]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
