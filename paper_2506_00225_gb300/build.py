"""Build the native rasterizer library ``libgs.so`` in-tree for sm_103a.

Each CUDA translation unit is compiled separately (in parallel) with
``nvcc -gencode arch=compute_103a,code=sm_103a -lineinfo -O3``, then linked
into one shared library with the CUDA runtime linked statically.  The
projection unit is compiled with ``-fmad=false`` so that its arithmetic is
evaluated one rounding per operation; the blend, semantic, candidate and
adjoint passes are compiled with ``-ftz=true`` (single-instruction exponential and
reciprocal).  Flushing denormals changes no contributor decision: a
denormal exponential gives alpha far below 1/255 either way, and the
transmittance never falls below the 1e-4 stop.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "_lib", "libgs.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = {
    "project.cu": ["-fmad=false"],
    "sort.cu": [],
    "render_fwd.cu": ["-ftz=true"],
    "render_bwd.cu": ["-ftz=true"],
    "candidates.cu": ["-ftz=true"],
    "loss.cu": [],
    "mapping_loss.cu": [],
    "render_objective.cu": [],
    "render_dense.cu": ["-ftz=true"],
    "explore.cu": [],
    "topk.cu": [],
    "voxel.cu": ["-fmad=false"],
    "api.cu": [],
    "noalloc.cu": [],
    "stats.cu": ["-ftz=true"],
}
HEADERS = ["gs_internal.cuh", "render_common.cuh", "objective_math.cuh"]


def nvcc() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _newest_dep() -> float:
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INC, "gs.h"), __file__]
    return max(os.path.getmtime(d) for d in deps)


def _compile(src: str, extra: list[str], verbose: bool) -> str:
    obj = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
    srcp = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(srcp), _newest_dep()):
        return obj
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC,
           *extra, "-c", srcp, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force:
        for f in os.listdir(OUT_DIR):
            os.remove(os.path.join(OUT_DIR, f))
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda kv: _compile(kv[0], kv[1], verbose), SOURCES.items()))
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs):
        return LIB
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", *objs, "-o", LIB + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
