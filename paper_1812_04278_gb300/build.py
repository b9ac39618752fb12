"""Build step of libw5ct.so: nvcc for sm_103a, one object per translation
unit compiled in parallel, linked in-tree next to this file."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJDIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libw5ct.so")
SOURCES = ["w5ct_adjoint64z.cu", "w5ct_adjoint64js.cu", "w5ct_adjoint32z.cu", "w5ct_adjoint32js.cu",
           "w5ct_api.cu", "w5ct_sweep32.cu", "w5ct_sweep64.cu", "w5ct_sweep64dw.cu", "w5ct_fused32.cu",
           "w5ct_fused64.cu",
           "w5ct_noalloc.cu"]
HEADERS = ["w5ct_physics.cuh", "w5ct_kernels.cuh", "w5ct_internal.h", "w5ct_adjoint.cuh",
           "w5ct_fused.cuh"]

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE]
# The float sweep (FP32-bulk arithmetic) uses the hardware approximate
# reciprocal / square root and flushes subnormals; every double operation
# and every other translation unit stays IEEE.
FAST_FLOAT = ["-ftz=true", "-prec-div=false", "-prec-sqrt=false"]
TU_FLAGS = {"w5ct_sweep32.cu": FAST_FLOAT, "w5ct_adjoint32z.cu": FAST_FLOAT, "w5ct_adjoint32js.cu": FAST_FLOAT,
            "w5ct_fused32.cu": FAST_FLOAT}


def _newest_input() -> float:
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "w5ct.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libw5ct.so if it is missing or older than its sources."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    os.makedirs(OBJDIR, exist_ok=True)

    def compile_one(src: str) -> str:
        obj = os.path.join(OBJDIR, src.replace(".cu", ".o"))
        cmd = [NVCC, *ARCH, *CFLAGS, *TU_FLAGS.get(src, []), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp.%d" % os.getpid()
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
