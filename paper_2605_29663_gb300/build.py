"""Build step of the CUDA library: nvcc for sm_103a, in-tree, no cmake.

Compiles every translation unit under ``csrc/`` in parallel into
``_build/`` and links ``_lib/libexact_mppi.so``.  Rebuilds only when a
source, a header or the flags changed.  ``build(debug=True)`` makes the
debug variant ``_lib/libexact_mppi_debug.so`` (``-DEXACT_DEBUG_CHECKS``:
device-side index checks that record EXACT_ECAPACITY in the error word and
skip the access) from ``_build_debug/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
LIB_DIR = os.path.join(PKG, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "libexact_mppi.so")
LIB_PATH_DEBUG = os.path.join(LIB_DIR, "libexact_mppi_debug.so")
BUILD_DIR_DEBUG = os.path.join(PKG, "_build_debug")

SOURCES = ["runtime.cu", "sdf_batch.cu", "mppi.cu", "batched.cu", "noalloc.cu", "mlp.cu", "features.cu", "hybrid.cu", "mppi_predicted.cu", "mppi_dense.cu", "mppi_points.cu", "batched_uniform_small.cu", "batched_uniform_large.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--ptxas-options=-O3", f"-I{INCLUDE}", f"-I{CSRC}"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _fingerprint() -> str:
    h = hashlib.sha256()
    h.update(" ".join(ARCH + FLAGS + SOURCES).encode())
    for d in (CSRC, INCLUDE):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                with open(os.path.join(d, name), "rb") as f:
                    h.update(name.encode())
                    h.update(f.read())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> str:
    """Compile (if needed) and return the path of libexact_mppi.so (or of the
    debug variant)."""
    build_dir = BUILD_DIR_DEBUG if debug else BUILD_DIR
    lib_path = LIB_PATH_DEBUG if debug else LIB_PATH
    extra_flags = tuple(extra_flags) + (("-DEXACT_DEBUG_CHECKS",) if debug else ())
    os.makedirs(build_dir, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    fp = _fingerprint() + "|" + " ".join(extra_flags)
    stamp = os.path.join(build_dir, "stamp")
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read() == fp:
                return lib_path
    nvcc = _nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra_flags, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as f:
        f.write(fp)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose=True))
