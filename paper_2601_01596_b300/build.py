"""Build the FFCz CUDA library in-tree for sm_103a (B300).

``python -m paper_2601_01596_b300.build`` writes ``libffcz.so`` next to this
file.  The CUDA runtime is linked statically so the library does not depend
on which libcudart the host process (e.g. PyTorch) loaded.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libffcz.so")
SRC = [os.path.join(HERE, "csrc", "ffcz.cu"), os.path.join(HERE, "csrc", "noalloc.cu")]


def deps():
    """Every source the library is built from: the .cu files, every header
    under csrc/ and the public header."""
    csrc = os.path.join(HERE, "csrc")
    return SRC + sorted(os.path.join(csrc, f) for f in os.listdir(csrc) if f.endswith((".cuh", ".h"))) + [
        os.path.join(ROOT, "include", "ffcz.h")]


ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in deps() if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    extra = os.environ.get("FFCZ_NVCC_EXTRA", "").split()   # e.g. -DFFCZ_W32=4
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-split-compile=0", "-shared", "-Xcompiler", "-fPIC",
           "-cudart", "static", "-I", os.path.join(ROOT, "include"), *extra, *SRC, "-o", LIB + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
