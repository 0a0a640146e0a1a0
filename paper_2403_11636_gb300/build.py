"""In-tree build of libfc (CUDA, sm_103a) with nvcc.

Each translation unit is compiled in parallel to an object file under
``_build/`` and linked into ``libfc.so`` next to this file.  The geometry
unit is compiled with ``--fmad=false`` so that its sums follow the operation
order of the quadrature definition; the host code of the adaptive-grid unit
(its constrained assembly) with ``-ffp-contract=off`` for the same reason,
while its device kernels keep fused multiply-adds.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["fc_geom.cu", "fc_assemble.cu", "fc_mg.cu", "fc_patch.cu", "fc_api.cu", "fc_noalloc.cu", "fc_batch.cu",
           "fc_probe.cu", "fc_q2.cu", "fc_amr.cu"]
EXTRA = {"fc_geom.cu": ["--fmad=false"], "fc_amr.cu": ["-Xcompiler", "-ffp-contract=off"]}


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, "fc_internal.cuh"), os.path.join(INCLUDE, "fc.h")]
    nvcc = _nvcc()

    def compile_one(src):
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        if force or _stale(obj, [path] + headers):
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE, *EXTRA.get(src, []), "-c", path, "-o", obj]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
