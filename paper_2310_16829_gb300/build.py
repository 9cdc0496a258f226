"""In-tree build of the CUDA library ``_build/liblma.so`` for sm_103a.

Two translation units compiled in parallel (nvcc for the kernels, the host
C++ compiler for the C-ABI), linked with the static CUDA runtime so that the
library also loads on machines without a driver (for the export checks).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liblma.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home() -> str:
    home = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if home and os.path.exists(os.path.join(home, "bin", "nvcc")):
        return home
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def build(verbose: bool = False, extra_nvcc=()) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    cxx = os.environ.get("CXX", "g++")
    inc = os.path.join(cuda, "include")
    k_obj = os.path.join(OUT_DIR, "lma_kernels.o")
    h_obj = os.path.join(OUT_DIR, "lma_host.o")
    cmds = [
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
         "-Xptxas", "-v" if verbose else "-O3", *extra_nvcc,
         "-c", os.path.join(CSRC, "lma_kernels.cu"), "-o", k_obj],
        [cxx, "-O2", "-fPIC", "-std=c++17", "-ffp-contract=off", "-Wall", "-Wno-unused-function",
         f"-I{inc}", "-c", os.path.join(CSRC, "lma_host.cpp"), "-o", h_obj],
    ]
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for c in cmds]
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out)
        if p.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(c)}")
    link = [nvcc, ARCH, "-shared", "-cudart", "static", k_obj, h_obj, "-o", LIB]
    p = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if p.returncode != 0:
        sys.stdout.write(p.stdout)
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
