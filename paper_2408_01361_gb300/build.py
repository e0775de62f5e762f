"""Build the CUDA library libkharma_gb300.so in place (sm_103a only).

Each translation unit is compiled by its own nvcc process (in parallel), then
linked with the CUDA runtime into a plain shared library that exports the C
ABI of include/kharma_gb300.h.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkharma_gb300.so")
# the bounds-checked variant (-DKH_BOUNDS_CHECK): every instrumented kernel
# checks its work item's cells against the allocation and counts and skips a
# violation instead of touching memory out of bounds
BUILD_BOUNDS = os.path.join(HERE, "_build_bounds")
LIB_BOUNDS = os.path.join(HERE, "libkharma_gb300_bounds.so")
SOURCES = ["kh_kernels.cu", "kh_api.cu", "kh_noalloc.cu", "kh_mesh.cu", "kh_adjoint.cu", "kh_flux_tma.cu",
           "kh_update_tma.cu"]
HEADERS = ["kh_internal.h", "kh_physics.cuh", "kh_geom_math.h", "kh_zone.cuh", "kh_ctx.h", "kh_dual.cuh", "kh_df64.cuh",
           "kh_mixed.cuh", "kh_face_vjp.cuh", "kh_pair.cuh", "kh_tma.cuh", "kh_update_tile.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _flags(verbose: bool, bounds: bool = False):
    f = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", CSRC, "-I", os.path.join(ROOT, "include")]
    f += ARCH
    if verbose:
        f += ["-Xptxas", "-v"]
    if bounds:
        f += ["-DKH_BOUNDS_CHECK"]
    return f


def build(force: bool = False, verbose: bool = False, bounds: bool = False) -> str:
    lib_path, build_dir = (LIB_BOUNDS, BUILD_BOUNDS) if bounds else (LIB, BUILD)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "kharma_gb300.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= newest and not verbose:
        return lib_path
    os.makedirs(build_dir, exist_ok=True)
    objs = [os.path.join(build_dir, s.replace(".cu", ".o")) for s in SOURCES]

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(verbose, bounds)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, zip(SOURCES, objs)))
    for cmd, r in results:
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
    tmp = lib_path + ".tmp"
    link = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("link failed: " + " ".join(link))
    os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv))
