"""Builds libgs2.so (all CUDA sources of csrc/) for sm_103a, in-tree.

    python -m paper_2501_13975_b300.build [--force] [--ptxas-verbose]

Each translation unit is compiled to an object under _build/ (in parallel, one
nvcc per source), then the objects are linked into the shared library.  An
object is rebuilt when its source, any csrc header or include/gs2.h is newer.

The environment variable GS2_TILE=8 builds the 8x8-tile variant (for
measurement; use --force when switching, the default is 16).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libgs2.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OBJDIR = os.path.join(os.path.dirname(HERE), "_build", "gs2")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
if os.environ.get("GS2_TILE"):
    FLAGS.append("-DGS2_TILE=" + str(int(os.environ["GS2_TILE"])))


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _obj(src: str) -> str:
    return os.path.join(OBJDIR, os.path.basename(src)[:-3] + ".o")


def _newest(paths) -> float:
    return max((os.path.getmtime(p) for p in paths), default=0.0)


def _compile(src: str, verbose: bool) -> str:
    obj = _obj(src)
    cmd = [NVCC, *ARCH, *FLAGS, "-c", "-o", obj + ".tmp", src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    hdr = _newest(_headers())
    if not (force or verbose) and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(hdr, _newest(sources())):
        return LIB   # up to date (also where only the library, not _build/, was copied)
    os.makedirs(OBJDIR, exist_ok=True)
    todo = [s for s in sources()
            if force or verbose or not os.path.exists(_obj(s))
            or os.path.getmtime(_obj(s)) < max(os.path.getmtime(s), hdr)]
    if todo:
        with ThreadPoolExecutor(max_workers=max(1, min(len(todo), os.cpu_count() or 1))) as ex:
            list(ex.map(lambda s: _compile(s, verbose), todo))
    objs = [_obj(s) for s in sources()]
    subprocess.check_call([NVCC, *ARCH, "-shared", "-o", LIB + ".tmp", *objs])
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--ptxas-verbose" in sys.argv)
    print(LIB)
