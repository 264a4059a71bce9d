"""Build the CUDA library ``_build/libcc_gb300.so`` in-tree with nvcc (sm_103a).

Each translation unit compiles in parallel; the link step uses nvcc so the
CUDA runtime is linked statically (the library needs no torch at run time).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcc_gb300.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
CU_FLAGS = ARCH + ["-lineinfo", "--expt-relaxed-constexpr"] + COMMON

SOURCES = ["kernels.cu", "fused.cu", "combine.cu", "noalloc.cu", "exec.cpp", "graph.cpp", "plan.cpp", "arena.cpp",
           "api.cpp", "serve.cpp", "estimate.cpp"]
HEADERS = ["kernels.cuh", "gather.cuh", "wideint.cuh", "runtime.h", "plan.h"]


def _obj(src: str) -> str:
    return os.path.join(BUILD, src + ".o")


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src: str, verbose: bool) -> str:
    path = os.path.join(CSRC, src)
    out = _obj(src)
    deps = [path] + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "cc.h")]
    if not _stale(out, deps):
        return out
    if src.endswith(".cu"):
        cmd = [NVCC] + CU_FLAGS + ["-c", path, "-o", out]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
    else:
        cmd = [NVCC, "-x", "c++"] + COMMON + ["-c", path, "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force:
        for s in SOURCES:
            if os.path.exists(_obj(s)):
                os.remove(_obj(s))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
