"""Build liboat.so (the sm_103a projector / backprojector and its C ABI) in-tree.

Each translation unit is compiled by nvcc in parallel into ``_build/`` and linked into
``paper_1304_2017_gb300/liboat.so``.  Host code is compiled without floating-point
contraction so that the FP64 lattice tables follow IEEE arithmetic in the written order.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "liboat.so")
ROOT = os.path.dirname(PKG)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["abi.cpp", "plan.cpp", "forward.cu", "adjoint.cu", "recon.cu", "unet.cu", "conv_tc.cu", "probe.cu", "fbp.cu", "eir.cu", "sph.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA extension cannot be built")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
                   "-I", os.path.join(ROOT, "include"), "-I", SRC]


def _compile(src: str) -> str:
    obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
    path = os.path.join(SRC, src)
    deps = [path, os.path.join(SRC, "oat_internal.h"), os.path.join(SRC, "brick.cuh"), os.path.join(ROOT, "include", "oat.h"),
            os.path.join(ROOT, "include", "oat_recon.h"), os.path.join(ROOT, "include", "oat_unet.h"), os.path.join(ROOT, "include", "oat_probe.h")]
    if os.path.exists(obj) and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
        return obj
    subprocess.check_call([nvcc()] + _flags() + ["-c", path, "-o", obj])
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(_compile, SOURCES))
    if os.path.exists(LIB) and all(os.path.getmtime(LIB) >= os.path.getmtime(o) for o in objs):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-ldl", "-lrt", "-lpthread"])
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
