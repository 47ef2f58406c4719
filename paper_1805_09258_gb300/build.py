"""Build libvrc.so (the CUDA library) in place with nvcc for sm_103a.

Each translation unit is compiled in parallel to an object file, then linked into
one shared library next to this file.  Rebuilds only when a source is newer than
the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libvrc.so")
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["scene.cu", "records.cu", "query.cu", "noalloc.cu", "mlp.cu", "render.cu", "flat.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# The record, 2D-record, query and render kernels use the hardware's approximate division,
# reciprocal and square root and flush denormals to zero.  Measured: primary pre-pass -17 %,
# record kernel -9 %, 2D records -27 %, queries -8 %, rendering -16 %, at the same distance
# from the FP64 oracles (errors of a few units in the last place sit far inside the 1e-4 /
# 1e-3 tolerances and the near-tie budgets; region membership compares squared distances,
# which these flags do not touch).
_APPROX = ["-prec-div=false", "-prec-sqrt=false", "-ftz=true"]
SOURCE_FLAGS = {"records.cu": _APPROX, "flat.cu": _APPROX, "query.cu": _APPROX, "render.cu": _APPROX}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _flags(verbose: bool):
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in os.listdir(CSRC)] + [os.path.join(INCLUDE, "vrc.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]

    def one(src):
        obj = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        cmd = [nvcc()] + _flags(verbose) + SOURCE_FLAGS.get(src, []) + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(one, srcs))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared"] + ARCH + [o for o, _ in results] + ["-o", tmp, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
