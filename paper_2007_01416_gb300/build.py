"""Builds libacat.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel into ``_build/`` and linked
against the shared CUDA runtime, so that the library and PyTorch share one
runtime and one primary context. Rebuilds only what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libacat.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["step1d.cu", "batch1d.cu", "step2d.cu", "adjoint1d.cu", "api.cu", "peak.cu", "weights.cpp",
           "noalloc.cu"]
HEADERS = [os.path.join(CSRC, "acat_internal.h"), os.path.join(CSRC, "device_common.cuh"),
           os.path.join(CSRC, "phys1d.cuh"), os.path.join(CSRC, "step1d_core.cuh"),
           os.path.join(ROOT, "include", "acat.h")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libacat")


def _compile(src: str, force: bool, extra: list[str], build_dir: str = BUILD) -> str:
    path = os.path.join(CSRC, src)
    obj = os.path.join(build_dir, src + ".o")
    deps = [path] + HEADERS
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= max(map(os.path.getmtime, deps)):
        return obj
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-c", path, "-o", obj + ".tmp", *extra]
    if src.endswith(".cu"):
        cmd += ["--expt-relaxed-constexpr"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


# Library variants: the product library, and a bounds-checked build of the same
# sources (-DACAT_BOUNDS_CHECK: every checked index records ACAT_STATUS_BOUNDS
# and skips its access instead of faulting) used by the tests.
VARIANTS = {"": (BUILD, LIB, []),
            "bounds": (os.path.join(HERE, "_build_bounds"), os.path.join(HERE, "libacat_bounds.so"),
                       ["-DACAT_BOUNDS_CHECK"])}


def build(force: bool = False, extra: list[str] | None = None, variant: str = "") -> str:
    build_dir, lib, vflags = VARIANTS[variant]
    os.makedirs(build_dir, exist_ok=True)
    extra = list(extra or []) + vflags
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, extra, build_dir), SOURCES))
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < max(map(os.path.getmtime, objs)):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", *objs, "-o", tmp]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stderr}")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
