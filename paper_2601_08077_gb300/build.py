"""Build libdf (CUDA, sm_103a) and the host input generator, in-tree.

``build_all()`` compiles every CUDA translation unit under ``csrc/`` with
``nvcc -gencode arch=compute_103a,code=sm_103a`` in parallel and links them
into ``_build/libdf.so``; it also compiles the C integral generator used by
``inputs``.  Nothing is installed outside the package directory.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libdf.so")
CU_SOURCES = ["split.cu", "slicegemm.cu", "coulomb.cu", "df_api.cu", "noalloc.cu", "batch.cu", "mlp.cu", "cderi.cu", "crt.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_home() -> str:
    return os.path.dirname(os.path.dirname(nvcc()))


def _compile(src: str, verbose: bool) -> str:
    obj = os.path.join(OUT, os.path.splitext(os.path.basename(src))[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c",
           os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h"))]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "df.h"))
    if not force and not _stale(LIB, deps):
        return LIB
    with cf.ThreadPoolExecutor(max_workers=len(CU_SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), CU_SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    lib64 = os.path.join(_cuda_home(), "lib64")
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-L" + lib64, "-Xlinker", "-rpath=" + lib64, "-lcublas", "-lcusolver"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


def build_all(force: bool = False, verbose: bool = False) -> None:
    from . import inputs
    inputs.build_generator_library(force=force)
    build_library(force=force, verbose=verbose)


if __name__ == "__main__":
    build_all(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
