"""Builds the CUDA library ``lib/liblisa_psd.so`` in-tree with nvcc for sm_103a.

Each translation unit under ``csrc/`` is compiled in parallel (``-gencode
arch=compute_103a,code=sm_103a``, no other architecture) and linked into one shared library
with a plain C ABI (``include/lisa_psd.h``); the CUDA runtime is linked statically.

``build(debug=True)`` builds the bounds-checked variant ``lib/liblisa_psd_debug.so`` (the same
sources with ``-DLISA_DEBUG_BOUNDS``: every checked tile, bin, knot, record, slot and list index is
tested and clamped, violations are recorded; ``include/lisa_debug.h``) in its own object folder.
It is built on demand, not by the default build."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIB_DIR, "liblisa_psd.so")
LIB_DEBUG = os.path.join(LIB_DIR, "liblisa_psd_debug.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
              "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblisa_psd.so")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps() + [__file__])


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Compiles (if needed) and returns the path of ``liblisa_psd.so`` (``debug``: of the
    bounds-checked ``liblisa_psd_debug.so``)."""
    lib = LIB_DEBUG if debug else LIB
    obj_dir = BUILD_DEBUG if debug else BUILD
    flags = [*extra_flags, "-DLISA_DEBUG_BOUNDS"] if debug else list(extra_flags)
    if not force and up_to_date(debug):
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
