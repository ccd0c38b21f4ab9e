"""Compile liblsm.so (CUDA kernels + C ABI) in-tree for sm_103a with nvcc.

Translation units are compiled in parallel into ``_build/`` and linked into
``liblsm.so`` next to this file. Nothing is installed anywhere else.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblsm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = ["kernels.cu", "batch.cu", "tile2d.cu", "strip2d.cu", "tile3d.cu", "static_scratch.cu", "csr_fix.cu", "fields.cu", "nn.cu", "conv_tc.cu", "build.cpp", "checkpoint.cpp", "api.cpp"]
HEADERS = ["lsm_internal.h", "dfloat.cuh", "tile_body.cuh", "strip_body.cuh", "nn_internal.h", "nvtx_range.h"]


def _nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblsm")


def _sources():
    return [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.exists(d) and os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    inc = os.path.join(os.path.dirname(HERE), "include")
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(inc, q) for q in os.listdir(inc)]
    procs, objs = [], []
    for src in _sources():
        path = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if not force and not _stale(obj, [path, __file__] + hdrs):
            continue
        cmd = [nvcc, "-c", path, "-o", obj, "-O3", "-std=c++17", "-lineinfo", "-I", inc,
               "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        cmd += ARCH
        if src.endswith(".cu"):
            cmd += ["--expt-relaxed-constexpr"]
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if verbose or pr.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
        if pr.returncode != 0:
            errors.append(src)
    if errors:
        raise RuntimeError("nvcc failed for: " + ", ".join(errors))
    if force or procs or not os.path.exists(LIB):
        tmp = LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call([nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
