"""Build libgray.so (the CUDA library behind include/gray.h) in-tree for sm_103a.

One translation unit, one -gencode, no cmake: ``python -m
paper_1303_5057_gb300.build`` or ``build()`` from Python.
"""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
SRC = os.path.join(PKG, "csrc", "gray.cu")
DEPS = [SRC, os.path.join(PKG, "csrc", "kerr.cuh"), os.path.join(ROOT, "include", "gray.h")]
LIB = os.path.join(PKG, "libgray.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = os.path.join(home, "bin", "nvcc")
    return exe if os.path.exists(exe) else "nvcc"


def command(out=LIB, extra=()):
    return [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
            "-I" + os.path.join(ROOT, "include"), "-o", out, SRC, *extra]


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in DEPS):
            return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = command(tmp, ["-Xptxas", "-v"] if verbose else [])
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv))
