"""Build the CUDA library `librt_b300.so` in-tree for sm_103a (B300).

The library is plain C ABI (include/rt.h) linked against the shared CUDA
runtime, so it shares one runtime with PyTorch in the same process.
"""
from __future__ import annotations

import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "librt_b300.so")
SOURCES = [os.path.join(CSRC, "rt_api.cu"), os.path.join(CSRC, "rt_noalloc.cu"), os.path.join(CSRC, "nn_kernels.cu"),
           os.path.join(CSRC, "conv_tc.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + \
    [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a",
         "-Xcompiler", "-fPIC", "-shared", "-cudart", "shared",
         "-Xlinker", "-rpath,/usr/local/cuda/lib64", "-I", INCLUDE]


# The bounds-checking variant of the tracer (RT_CHECK_BOUNDS=1): every gather,
# tally and box index in the transport kernel is checked, and a failed check
# sets a status bit (RT_E_BOUNDS) instead of trapping. Test-only; it holds the
# rt_* entry points (not the denoiser's nn_* ones).
CHECKED_LIB = os.path.join(PKG, "librt_b300_checked.so")
CHECKED_SOURCES = [os.path.join(CSRC, "rt_api.cu"), os.path.join(CSRC, "rt_noalloc.cu")]


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in DEPS)


def _compile(lib, sources, extra, verbose):
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC, *FLAGS, *extra, "-o", tmp, *sources]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(tmp, lib)


def build(force: bool = False, verbose: bool = False) -> str:
    if force or needs_build(LIB):
        _compile(LIB, SOURCES, [], verbose)
    return LIB


def build_checked(force: bool = False, verbose: bool = False) -> str:
    """The bounds-checking variant of the tracer library; returns its path."""
    if force or needs_build(CHECKED_LIB):
        _compile(CHECKED_LIB, CHECKED_SOURCES, ["-DRT_CHECK_BOUNDS=1"], verbose)
    return CHECKED_LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
    print(build_checked(force=True))
