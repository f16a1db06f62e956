"""Build libhpsi.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked with cuBLAS / cuSOLVER (used only for
the Davidson subspace algebra).  The result lands next to this file; ``binding.load()`` opens it.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhpsi.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["api.cu", "local_kernels.cu", "local_fast.cu", "nonlocal_fp64.cu", "nonlocal_tc.cu", "davidson.cu", "cg.cu", "eigh.cu", "subspace_gemm.cu", "noalloc.cu", "gamma.cu", "scf.cu", "fock.cu", "plan.cpp"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libhpsi")


def cuda_home() -> str:
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))


def _compile(src: str, extra: list) -> tuple:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
           "-I", os.path.join(HERE, "..", "include"), "-c", os.path.join(CSRC, src), "-o", obj] + extra
    if src.endswith(".cpp"):
        cmd[cmd.index("-c"):cmd.index("-c")] = ["-x", "c++"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, obj, r.returncode, r.stdout + r.stderr


def build(verbose: bool = False, extra: list | None = None) -> str:
    """Compile every source and link libhpsi.so; returns its path.  Raises on any error."""
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra or [])
    with ThreadPoolExecutor(max_workers=min(8, len(SOURCES))) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    bad = [r for r in results if r[2] != 0]
    for src, _, rc, out in results:
        if verbose or rc != 0:
            sys.stderr.write(f"--- {src} (rc={rc})\n{out}")
    if bad:
        raise RuntimeError("libhpsi build failed: " + ", ".join(b[0] for b in bad))
    lib64 = os.path.join(cuda_home(), "lib64")
    tmp = LIB + ".tmp"
    cmd = [nvcc(), ARCH, "-shared", "-o", tmp] + [r[1] for r in results] + [
        "-L", lib64, "-lcublas", "-lcusolver", "-lcudart", "-Xlinker", "-rpath=" + lib64]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("libhpsi link failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
