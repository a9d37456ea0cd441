"""Builds libsgeo.so in-tree with nvcc for sm_103a (GB300).

Sources under csrc/ are compiled in parallel into objects, then linked into
paper_2603_15780_gb300/_build/libsgeo.so against the shared CUDA runtime (so the
library and PyTorch share one runtime and one primary context).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsgeo.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["exp_map.cu", "exp_map64.cu", "exp_map_steps.cu", "backward.cu", "mesh_update.cu", "mesh_build.cpp"]
# The host mesh builder and the device vertex update evaluate the same FP64 expressions; both are
# compiled without multiply-add contraction so that they round identically.
PER_FILE = {"mesh_build.cpp": ["-Xcompiler", "-ffp-contract=off"], "mesh_update.cu": ["--fmad=false"]}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsgeo.so")


def _cuda_lib_dir(nv: str) -> str:
    return os.path.join(os.path.dirname(os.path.dirname(nv)), "lib64")


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    deps = srcs + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "sgeo.h"))
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo"] + ARCH + list(extra_flags or [])
    procs = []
    objs = []
    for s in srcs:
        o = os.path.join(OUT_DIR, os.path.basename(s) + ".o")
        objs.append(o)
        cmd = [nv, "-c", s, "-o", o] + common + PER_FILE.get(os.path.basename(s), [])
        if s.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            sys.stderr.write(out.decode(errors="replace"))
            raise RuntimeError("nvcc failed: " + " ".join(cmd))
        if verbose and out:
            sys.stderr.write(out.decode(errors="replace"))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nv, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared",
                                                       "-Xlinker", "-rpath," + _cuda_lib_dir(nv)]
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
