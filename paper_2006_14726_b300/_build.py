"""Compile the CUDA sources into the in-tree shared library ``libwrs.so`` (sm_103a only).

    python paper_2006_14726_b300/_build.py [--force] [--ptxas-v]

Run it by path: importing the package would load the library being rebuilt.  nvcc
cross-compiles without a GPU; the library travels with the source tree.  Each source is
compiled to its own object in ``_build/`` (in parallel; a source is recompiled when it, a
header or the flags changed), then the objects are linked.
"""
from __future__ import annotations

import concurrent.futures
import hashlib
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libwrs.so")
OBJ_DIR = os.path.join(PKG, "_build")
SOURCES = ["api.cu", "unproject.cu", "raycast.cu", "lbvh.cu", "trace.cu", "point_splat.cu", "codec.cu", "peak.cu"]
HEADERS = [os.path.join(CSRC, "common.cuh"), os.path.join(CSRC, "codec.cuh"), os.path.join(INCLUDE, "wrs.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [*ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _obj(src: str, flags) -> str:
    tag = hashlib.sha1(" ".join(flags).encode()).hexdigest()[:8]
    return os.path.join(OBJ_DIR, f"{os.path.splitext(src)[0]}.{tag}.o")


def _newer(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def stale() -> bool:
    return _newer(LIB, [os.path.join(CSRC, s) for s in SOURCES] + HEADERS)


def build(force: bool = False, verbose: bool = False, extra=(), out: str = LIB) -> str:
    if not force and out == LIB and not extra and not stale():
        return LIB
    os.makedirs(OBJ_DIR, exist_ok=True)
    flags = [*NVCC_FLAGS, *extra, "-I", INCLUDE, "-I", CSRC]
    jobs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = _obj(s, flags)
        if force or _newer(obj, [src, *HEADERS]):
            jobs.append([_nvcc(), *flags, "-c", src, "-o", obj + f".tmp{os.getpid()}"])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        subprocess.check_call(cmd)
        os.replace(cmd[-1], cmd[-1].rsplit(".tmp", 1)[0])

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for f in [ex.submit(run, j) for j in jobs]:
            f.result()
    tmp = out + f".tmp{os.getpid()}"
    link = [_nvcc(), *ARCH, "-shared", "-Xcompiler", "-fPIC",
            *[_obj(s, flags) for s in SOURCES], "-o", tmp]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.check_call(link)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra=["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else [])
    print(LIB)
