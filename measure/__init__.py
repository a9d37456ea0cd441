"""Measurement-only helpers of the benchmark: the 32-byte record gather probe and the reduction
probe.

``probe.cu`` is built into its own library, ``measure/_build/libsgeo_probe.so`` (nvcc, sm_103a,
in-tree), separate from the exponential-map library: it measures the memory ceilings a record
walk can reach on the device (L2 streaming reads, independent and dependent 32-byte gathers) so
that the benchmark can state the walk kernels' rates against them, and the rate of random
floating-point reductions into a gradient accumulator (in L2, or in a thread-block cluster's
distributed shared memory).  No part of the exponential map calls it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libsgeo_probe.so")
SRC = os.path.join(HERE, "probe.cu")

PROBE_STREAM, PROBE_RANDOM, PROBE_CHAIN, PROBE_LD256 = 0, 1, 2, 4
PROBE_RED8, PROBE_RED16, PROBE_RED_DSM = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    from paper_2603_15780_gb300 import build as pkg_build
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    nv = pkg_build.nvcc()
    cmd = [nv, "-shared", "-o", tmp, SRC, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo"] + \
        pkg_build.ARCH + ["-cudart", "shared", "-Xlinker", "-rpath," + pkg_build._cuda_lib_dir(nv)]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        sys.stderr.write(r.stdout.decode(errors="replace"))
        raise RuntimeError("nvcc failed: " + " ".join(cmd))
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.sg_probe_gather.argtypes = [C.c_int32, C.c_int64, C.c_int32, C.c_int32, C.c_int32,
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.sg_probe_gather.restype = C.c_int
        L.sg_probe_reduce.argtypes = [C.c_int32, C.c_int64, C.c_int32, C.c_int32,
                                      C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.sg_probe_reduce.restype = C.c_int
        _lib = L
    return _lib


def probe_gather(mode: int, table_bytes: int, blocks_per_sm: int, threads: int, loads: int) -> float:
    """GB/s of one timed launch reading a table of 32-byte records: PROBE_STREAM (coalesced
    16-byte loads sweeping the table `loads` times), PROBE_RANDOM (`loads` independent record
    gathers per thread, four in flight) or PROBE_CHAIN (`loads` dependent gathers per thread along
    one random cycle through the table), optionally | PROBE_LD256 (one 256-bit load per record).
    The table (the largest power-of-two count of records within table_bytes) is read once
    untimed first, so a table that fits stays in L2.  Synchronous on the legacy default stream;
    allocates and frees its own device memory."""
    sec, nb = C.c_double(), C.c_double()
    rc = lib().sg_probe_gather(mode, table_bytes, blocks_per_sm, threads, loads, C.byref(sec), C.byref(nb))
    if rc != 0:
        raise RuntimeError(f"sg_probe_gather failed with status {rc}")
    return nb.value / sec.value / 1e9


def probe_reduce(mode: int, table_bytes: int, iters: int, cluster: int = 0) -> float:
    """Random reductions per second (in G/s) into an accumulator table of table_bytes: PROBE_RED8
    (8-byte reductions into L2), PROBE_RED16 (16-byte reductions into L2) or PROBE_RED_DSM (the
    table spread over the shared memory of clusters of `cluster` CTAs, one CTA of 896 threads per
    SM, each reduction two 4-byte remote shared-memory reductions).  `iters` reductions per thread,
    one untimed and one timed launch.  Synchronous on the legacy default stream; allocates and frees
    its own device memory."""
    sec, ops = C.c_double(), C.c_double()
    rc = lib().sg_probe_reduce(mode, table_bytes, cluster, iters, C.byref(sec), C.byref(ops))
    if rc != 0:
        raise RuntimeError(f"sg_probe_reduce failed with status {rc}")
    return ops.value / sec.value / 1e9
