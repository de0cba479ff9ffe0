"""Build the CUDA library in-tree with nvcc for sm_103a (GB300)."""
from __future__ import annotations

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm.so")
SOURCES = ["lbm.cu", "lbm_noalloc.cu", "lbm_batch.cu"]
HEADERS = ["lbm_device.cuh", "lbm_kernels.cuh", "lbm_pair.cuh", "lbm_tma.cuh", "lbm_handle.h", "lbm_quad.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu into _build/liblbm.so (static cudart, -lineinfo)."""
    os.makedirs(BUILD, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "lbm.h")]
    if not force and not _stale(LIB, deps):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    # approximate FP32 division and square root (2 ulp): the relaxation time and
    # velocity tolerate it, and IEEE-exact forms cost ~4x the instructions
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-prec-div=false", "-prec-sqrt=false",
             "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]
    if verbose:
        flags.append("-Xptxas=-v")
    objs = [os.path.join(BUILD, os.path.splitext(os.path.basename(s))[0] + f".{os.getpid()}.o") for s in srcs]
    # one nvcc per translation unit, in parallel
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(srcs)) as pool:
        jobs = [pool.submit(subprocess.run, [nvcc(), *flags, "-c", "-o", o, src], check=True)
                for src, o in zip(srcs, objs)]
        for j in jobs:
            j.result()
    subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], check=True)
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
