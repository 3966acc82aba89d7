"""Build the in-tree shared library ``libopm_bsr.so`` for sm_103a with nvcc.

The library is the product: CUDA kernels plus the host analysis and the C ABI
declared in ``include/opm_bsr.h``.  It links the shared CUDA runtime so that
it shares one runtime with PyTorch when both are loaded.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libopm_bsr.so")
SOURCES = ["solver.cu", "symbolic.cpp", "noalloc.cu", "autotune.cpp"]
HEADERS = ["kernels.cuh", "sweeps.cuh", "factor.cuh", "gmres.cuh", "iterative.cuh", "opm_internal.h"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "opm_bsr.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc())), "lib64")
    if not os.path.isdir(cuda_lib):
        cuda_lib = "/usr/local/cuda/lib64"
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc(), "-O3", "-std=c++17", ARCH, "-lineinfo", "--threads", "3",
           "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
           "-Xlinker", f"-rpath,{cuda_lib}", "-o", tmp]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += [os.path.join(CSRC, f) for f in SOURCES]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
