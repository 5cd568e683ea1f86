"""Build libim.so for sm_103a in-tree (nvcc, one object per source, in parallel)."""
from __future__ import annotations

import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libim.so")
HEADERS = [os.path.join(CSRC, "internal.cuh"),
           os.path.join(os.path.dirname(HERE), "include", "im.h")]
SOURCES = ["scan.cu", "sample.cu", "index.cu", "cover.cu", "lazy.cu", "api.cu", "noalloc.cu", "imm.cu", "opim.cu", "batch.cu", "server.cu", "spread.cu", "tune.cu"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if _stale(obj, [path] + HEADERS):
        tmp = f"{obj}.{os.getpid()}.tmp"
        subprocess.run([NVCC, *FLAGS, "-c", path, "-o", tmp], check=True)
        os.replace(tmp, obj)
    return obj


def build_library(verbose: bool = False) -> str:
    """Compile the CUDA sources that changed and link libim.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    if _stale(LIB, objs):
        tmp = f"{LIB}.{os.getpid()}.tmp"
        subprocess.run([NVCC, "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                        "-Xcompiler", "-fPIC", *objs, "-o", tmp], check=True)
        os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build_library(verbose=True)
