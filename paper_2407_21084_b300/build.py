"""Builds libqrmc.so in-tree with nvcc for sm_103a (B300).

Each CUDA source is compiled to an object in parallel (objects under
_build/, which is not part of the repository), then linked into
paper_2407_21084_b300/libqrmc.so. With --checked the same sources are built
with QR_CHECKED=1 (objects under _build_checked/) into libqrmc_checked.so:
the hot kernels test every computed index against its buffer and report
one that falls outside through the context's status word (the stand-in for
a device memory checker; tests/test_gpu_checked.py runs it).

Usage: python -m paper_2407_21084_b300.build [--force] [--checked]
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
OBJ_CHECKED = os.path.join(ROOT, "_build_checked")
LIB_CHECKED = os.path.join(HERE, "libqrmc_checked.so")
SOURCES = ["qr_kernels.cu", "qr_fast.cu", "qr_fast_more.cu", "qr_proj_tree.cu", "qr_proj_more.cu", "qr_api.cu",
           "qr_static.cu", "qr_mlp.cu", "qr_batch.cu", "qr_group.cu", "qr_fast_paper.cu",
           "qr_cosine.cu", "qr_peak.cu", "qr_tc_selftest.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _headers():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return out


def stale(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in _headers() + [os.path.join(CSRC, s) for s in SOURCES])


def _compile(src: str, nvcc: str, verbose: bool, checked: bool = False) -> str:
    obj = os.path.join(OBJ_CHECKED if checked else OBJ, src.replace(".cu", ".o"))
    newest = max([os.path.getmtime(os.path.join(CSRC, src))] + [os.path.getmtime(h) for h in _headers()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    extra = ["-DQR_CHECKED=1"] if checked else []
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-I", INCLUDE, "-c", "-o", obj + ".tmp", os.path.join(CSRC, src)]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    lib, obj_dir = (LIB_CHECKED, OBJ_CHECKED) if checked else (LIB, OBJ)
    if not force and not stale(checked):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(obj_dir, exist_ok=True)
    if force:
        for s in SOURCES:
            p = os.path.join(obj_dir, s.replace(".cu", ".o"))
            if os.path.exists(p):
                os.remove(p)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, nvcc, verbose, checked), SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv)
