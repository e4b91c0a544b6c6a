"""Builds libqrmc.so in-tree with nvcc for sm_103a (B300).

Each CUDA source is compiled to an object in parallel (objects under
_build/, which is not part of the repository), then linked into
paper_2407_21084_b300/libqrmc.so.

Usage: python -m paper_2407_21084_b300.build [--force]
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libqrmc.so")
SOURCES = ["qr_kernels.cu", "qr_fast.cu", "qr_fast_more.cu", "qr_proj_tree.cu", "qr_proj_more.cu", "qr_api.cu",
           "qr_static.cu", "qr_mlp.cu", "qr_batch.cu", "qr_group.cu", "qr_fast_paper.cu",
           "qr_cosine.cu", "qr_peak.cu", "qr_tc_selftest.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _headers():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return out


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _headers() + [os.path.join(CSRC, s) for s in SOURCES])


def _compile(src: str, nvcc: str, verbose: bool) -> str:
    obj = os.path.join(OBJ, src.replace(".cu", ".o"))
    newest = max([os.path.getmtime(os.path.join(CSRC, src))] + [os.path.getmtime(h) for h in _headers()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    cmd = [nvcc, *ARCH, *FLAGS, "-I", INCLUDE, "-c", "-o", obj + ".tmp", os.path.join(CSRC, src)]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    if force:
        for s in SOURCES:
            p = os.path.join(OBJ, s.replace(".cu", ".o"))
            if os.path.exists(p):
                os.remove(p)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc, verbose), SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
