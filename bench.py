#!/usr/bin/env python3
"""Benchmark of the batched straightest-geodesic exponential map on GB300.

One step = one pass of the whole path over one batch resident in HBM:
  sg_exp_map (start-face sort + persistent walk, FP64-escalated classification)
  sg_exp_map_backward EP  (grad_v)
  sg_exp_map_backward GFD (grad_v, grad_p, grad_bary) with grad_V (vertex positions)
on the noisy icosphere s6 workload (81,920 faces, 1,048,576 queries, L ~ U[0.1, 1]).

Prints one JSON line (metric: geodesics/s fwd+bwd; face-crossings/s and the roofline of
the dominant kernel alongside).  `--impl reference` times the FP64 CPU oracle on the
host cores instead (bounded sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "face-crossings/sec and geodesics/sec fwd+bwd at 1M queries; frac of L2/HBM peak"
WORKLOAD_INDEX = 2
EPS = 1e-4
L2_FLUSH_BYTES = 512 << 20     # > 129 MB L2
# where the nvidia-smi clock samples of the timed region are written
CLOCKS_DIR = os.environ.get("SG_BENCH_CLOCKS_DIR", "/tmp")
RECORD_BYTES = 32


def ncu_traffic(kernel: str, key: str = "dram_bytes_per_launch"):
    """DRAM bytes (or, with key="lts_requests_per_launch", L2 requests) per launch of `kernel` from
    the committed ncu capture, or None when the kernel's sources changed since that capture
    (profiles/ncu_traffic.json)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(kernel)
    if not rec:
        return None
    files = {"k_bwd_rewalk": ["walk.cuh", "backward.cu"], "k_walk_persistent": ["walk.cuh", "exp_map.cu"]}.get(kernel)
    if files is None:
        return None
    csrc = os.path.join(ROOT, "paper_2603_15780_gb300", "csrc")
    sha = hashlib.sha1(b"".join(open(os.path.join(csrc, f), "rb").read() for f in files)).hexdigest()
    return rec.get(key) if sha == rec["source_sha1"] else None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index: int, path: str):
        self.path = path
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=open(path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0])); mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def gather_ceilings(ncross, ktimes):
    """The walks' record reads against the device's own 32-B gather ceilings, measured after the
    timed region by sg_probe_gather on an L2-resident 16 MiB table (the icosphere's half-edge and
    face records take 10.5 MB): the L2 streaming read rate, independent random record gathers,
    and chains of dependent gathers at each walk kernel's occupancy (one gather in flight per
    thread, as in a walk), each with the walks' two 16-B loads per record and with one 256-bit
    load.  Rates are of record bytes only (32 B per crossing)."""
    import measure as sg
    tb = 16 << 20
    W = sg.PROBE_LD256
    out = {"table_MiB": tb >> 20, "stream_GBps": sg.probe_gather(sg.PROBE_STREAM, tb, 4, 256, 100),
           "random_GBps": {"2x16B": sg.probe_gather(sg.PROBE_RANDOM, tb, 4, 256, 256),
                           "1x32B": sg.probe_gather(sg.PROBE_RANDOM | W, tb, 4, 256, 256)}}
    for k, key, bps, thr in (("k_walk_persistent", "walk", 4, 256), ("k_bwd_rewalk", "rewalk", 7, 128)):
        rec = ncross * RECORD_BYTES / (float(np.mean(ktimes[key])) * 1e-3) / 1e9
        c16 = sg.probe_gather(sg.PROBE_CHAIN, tb, bps, thr, 256)
        c32 = sg.probe_gather(sg.PROBE_CHAIN | W, tb, bps, thr, 256)
        out[k] = {"record_GBps": rec, "chain_GBps": {"2x16B": c16, "1x32B": c32},
                  "frac_of_chain": {"2x16B": rec / c16, "1x32B": rec / c32}}
    # the re-walk's other L2 traffic: random reductions into the grad_V accumulator, 8 B (one
    # crossing) or 16 B (a pair of crossings, the face windows: 48 B per face of the 81,920-face
    # mesh), against the same 983,040-byte per-edge table held in a cluster's shared memory
    wtab, etab = 48 * 81920, 8 * 122880
    out["reduce_G_per_s"] = {"l2_8B": sg.probe_reduce(sg.PROBE_RED8, wtab, 400),
                             "l2_16B": sg.probe_reduce(sg.PROBE_RED16, wtab, 400),
                             "cluster5_dsmem_8B": sg.probe_reduce(sg.PROBE_RED_DSM, etab, 400, cluster=5),
                             "cluster8_dsmem_8B": sg.probe_reduce(sg.PROBE_RED_DSM, etab, 400, cluster=8),
                             "tables": {"l2_bytes": wtab, "dsmem_bytes": etab}}
    return out


def load_workload(scale=1.0):
    import meshgen
    wl = meshgen.workload(WORKLOAD_INDEX, scale=scale)
    X, F = wl.single
    return wl, np.ascontiguousarray(X, np.float32), F


def rank_queries(wl, X, F, rank: int):
    """Weak scaling: rank 0 takes the workload's own queries; rank r > 0 an independent batch
    of the same size and distribution from its own PCG64 stream (seed 1000 + index, r)."""
    if rank == 0:
        return wl.queries
    import meshgen
    rng = np.random.Generator(np.random.PCG64([1000 + WORKLOAD_INDEX, rank]))
    return meshgen.sample_queries(X.astype(np.float64), F, len(wl.queries), rng, 0.1, 1.0, 0)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (all-reduce MAX); identity for one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- oracle arm
def oracle_sample(n_sample: int, threads: int):
    """Time the FP64 oracle (forward + EP + GFD, as it stands) on the first n_sample queries."""
    import oracle
    wl, X32, F = load_workload(n_sample / 1048576)
    q = wl.queries
    om = oracle.Mesh(X32.astype(np.float64), F)
    b = q.bary.astype(np.float32).astype(np.float64)
    v = q.v.astype(np.float32).astype(np.float64)
    g = q.g_pos.astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    out = oracle.exp_map(om, q.face, b, v, threads=threads)
    oracle.ep_backward(om, q.face, b, v, g, threads=threads)
    oracle.gfd_backward(om, q.face, b, v, g, EPS, EPS, threads=threads)
    dt = time.perf_counter() - t0
    return len(q), dt, int(out["ncross"].sum())


def run_reference(args):
    threads = os.cpu_count() or 1
    n = args.ref_sample
    per = []
    for _ in range(max(args.warmup, 0)):
        oracle_sample(min(n, 4096), threads)
    crossings = 0
    for _ in range(args.steps):
        nq, dt, nc = oracle_sample(n, threads)
        per.append(dt)
        crossings = nc
    t = float(np.sum(per))
    value = args.steps * n / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "geodesics/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "icosphere-s6-noisy 81920F 1Mq fwd+EP+GFD+gradV", "global_batch": n,
                       "faces": 81920, "sample": f"first {n} of the 1,048,576 queries per step; the oracle "
                       "computes fwd+EP+GFD (its vertex gradient is checked by finite differences, not timed)"},
            "crossings_per_s": crossings * args.steps / t,
            "cpu_baseline": {"value": value, "unit": "geodesics/s", "cores": threads, "kind": "oracle",
                             "sample": f"first {n} of the 1,048,576 workload queries, fwd+EP+GFD"},
            "e2e": {"value": value, "unit": "geodesics/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- multi-mesh
def run_multimesh(args):
    """64 meshes of uneven size (workload 3): the plain FP32 kernel launched once per mesh on a
    one-mesh object vs one autotuned, graph-captured persistent launch (start-face sort, FP64
    classification) over the batched object; accuracy of both against the FP64 oracle on a
    sample."""
    import torch
    import meshgen
    import oracle
    import paper_2603_15780_gb300 as sg
    from paper_2603_15780_gb300 import autotune
    dev = torch.device("cuda", 0)
    wl = meshgen.workload(3)
    q = wl.queries
    nq = len(q)
    meshes32 = [(np.ascontiguousarray(X, np.float32), F) for X, F in wl.meshes]
    batched = sg.Mesh(meshes32)
    singles = [sg.Mesh(X, F) for X, F in meshes32]
    T = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    face, bary, v, mid = T(q.face, torch.int32), T(q.bary), T(q.v), T(q.mesh_id, torch.int32)
    bounds = np.searchsorted(q.mesh_id, np.arange(65))
    per = [(face[bounds[m]:bounds[m + 1]], bary[bounds[m]:bounds[m + 1]], v[bounds[m]:bounds[m + 1]])
           for m in range(64)]
    plain = sg.default_opts(kernel=sg.KERNEL_PLAIN, fp64_escalate=0, sort=0)
    outs = [sg.exp_map(singles[m], *per[m], opts=plain) for m in range(64)]

    def run_plain():
        for m in range(64):
            sg.exp_map(singles[m], *per[m], opts=plain, out=outs[m])

    if args.no_autotune:
        best, table = sg.default_opts(), []
    else:
        best, table = autotune.tune(batched, face, bary, v, mesh_id=mid, reps=3)
    g = autotune.GraphedExpMap(batched, face, bary, v, mesh_id=mid, opts=best)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ts = []
        for _ in range(args.steps):
            torch.cuda.synchronize()
            flush.zero_()            # evicts L2; the timed work is enqueued behind it (not timed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    clk = Clocks(0, os.path.join(CLOCKS_DIR, "clocks_mm.csv"))
    t_plain = timed(run_plain)
    t_graph = timed(g.replay)
    clocks = clk.stop()
    ncross = int(g.outputs["ncross"].sum().item())
    # accuracy against the oracle on 8 meshes x 500 queries
    rng = np.random.default_rng(7)
    acc = {"plain": [], "graph": []}
    flagged = {"plain": [], "graph": []}
    for m in rng.choice(64, 8, replace=False):
        idx = np.arange(bounds[m], bounds[m + 1])
        idx = rng.choice(idx, min(500, len(idx)), replace=False)
        X, F = meshes32[m]
        om = oracle.Mesh(X.astype(np.float64), F)
        ref = oracle.exp_map(om, q.face[idx], q.bary[idx].astype(np.float32).astype(np.float64),
                             q.v[idx].astype(np.float32).astype(np.float64))
        diag = meshgen.bbox_diag(X)
        for name, pos, st in (("plain", outs[m]["pos"][idx - bounds[m]], outs[m]["status"][idx - bounds[m]]),
                              ("graph", g.outputs["pos"][idx], g.outputs["status"][idx])):
            st = st.cpu().numpy().astype(np.uint32) | ref["status"]
            ok = (st & 4) == 0
            err = np.linalg.norm(pos.cpu().numpy() - ref["pos"], axis=1) / diag
            acc[name].append(err[ok])
            flagged[name].append(1.0 - ok.mean())
    stats = {k: {"max_pos_err_over_diag": float(np.concatenate(v).max()),
                 "p99_pos_err_over_diag": float(np.quantile(np.concatenate(v), 0.99)),
                 "near_vertex_flagged": float(np.mean(flagged[k]))} for k, v in acc.items()}
    cfg = {f[0]: getattr(best, f[0]) for f in best._fields_
           if f[0] in ("kernel", "block", "blocks_per_sm", "sort", "fp64_escalate", "queries_per_thread",
                       "precision")}
    line = {"metric": "geodesics/s, 64 uneven meshes in one launch", "value": nq / (t_graph * 1e-3),
            "unit": "geodesics/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_graph, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 meshes F log-uniform [1e3,5e5] (5.8M faces), q_m = clamp(2F_m,1e3,1e6)",
                       "queries": nq, "faces": int(batched.n_faces), "autotuned": cfg,
                       "l2": "flushed between steps (512 MB write)"},
            "plain_per_mesh": {"ms": t_plain, "geodesics_per_s": nq / (t_plain * 1e-3), "launches": 64},
            "graph_persistent": {"ms": t_graph, "geodesics_per_s": nq / (t_graph * 1e-3),
                                 "crossings_per_s": ncross / (t_graph * 1e-3)},
            "speedup": t_plain / t_graph, "accuracy_vs_oracle": stats,
            "autotune_table": [(c, round(ms, 4)) for c, ms in table], "clocks": clocks}
    print(json.dumps(line), flush=True)
    if args.json_out:
        open(args.json_out, "w").write(json.dumps(line) + "\n")


def run_config(args, index):
    """Forward throughput and accuracy on one of the single-mesh workloads: 0 (icosphere s3, 4096
    queries, 1 carried vector), 1 (torus 262k faces, 4M queries, 2 carried vectors) or 4 (sliver
    heightfield 4.2M faces, 16M queries; also EP / GFD backward and the FP64 and double-float
    walks).  Variants: the library's default (auto: one thread per query below 65,536 queries,
    else the persistent kernel in the automatic query order, FP64 classification), the persistent
    kernel forced, and the plain one-thread-per-query FP32 kernel; accuracy of each against the
    FP64 oracle on a sample of 2000 queries."""
    import torch
    import meshgen
    import oracle
    import paper_2603_15780_gb300 as sg
    dev = torch.device("cuda", 0)
    wl = meshgen.workload(index)
    X, F = wl.single
    q = wl.queries
    nq = len(q)
    nw = {0: 1, 1: 2, 4: 0}[index]
    X32 = np.ascontiguousarray(X, np.float32)
    mesh = sg.Mesh(X32, F)
    T = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    face, bary, v = T(q.face, torch.int32), T(q.bary), T(q.v)
    w = T(q.w[:, :nw]) if nw else None
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    steps = args.steps if index != 4 else min(args.steps, 5)

    def timed(fn, n_steps):
        for _ in range(args.warmup):
            fn()
        ts = []
        for _ in range(n_steps):
            torch.cuda.synchronize()
            flush.zero_()            # evicts L2; the timed work is enqueued behind it (not timed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    variants = {"auto": sg.default_opts(), "persistent": sg.default_opts(kernel=sg.KERNEL_PERSISTENT),
                "fp32": sg.default_opts(kernel=sg.KERNEL_PERSISTENT, precision=32),
                "plain": sg.default_opts(kernel=sg.KERNEL_PLAIN, sort=0, fp64_escalate=0, precision=32)}
    res, outs = {}, {}
    clk = Clocks(0, os.path.join(CLOCKS_DIR, f"clocks_w{index}.csv"))
    for name, o in variants.items():
        out = sg.exp_map(mesh, face, bary, v, w, opts=o, want_hash=True)
        ws = out.pop("_workspace", None)
        t = timed(lambda: sg.exp_map(mesh, face, bary, v, w, opts=o, workspace=ws, out=out), steps)
        nc = int(out["ncross"].sum().item())
        res[name] = {"ms": t, "geodesics_per_s": nq / (t * 1e-3), "crossings_per_s": nc / (t * 1e-3)}
        outs[name] = out
    sub64 = None
    if index == 4:
        # the full-precision walks (FP64, double-float) on the first 1M queries
        n64 = min(nq, 1 << 20)
        sub64 = n64
        for pname, prec in (("auto_1M", 0), ("mixed", 40), ("fp64", 64), ("double_float", 48)):
            o64 = sg.default_opts(precision=prec)
            out = sg.exp_map(mesh, face[:n64], bary[:n64], v[:n64], opts=o64, want_hash=True)
            ws = out.pop("_workspace", None)
            t = timed(lambda: sg.exp_map(mesh, face[:n64], bary[:n64], v[:n64], opts=o64, workspace=ws, out=out), 3)
            nc = int(out["ncross"].sum().item())
            res[pname] = {"ms": t, "queries": n64, "geodesics_per_s": n64 / (t * 1e-3),
                          "crossings_per_s": nc / (t * 1e-3)}
            outs[pname] = out
        # backward at full size (EP, GFD) on the persistent forward's outputs
        po = outs["persistent"]
        g = T(q.g_pos)
        for est in ("ep", "gfd"):
            nb = sg.backward_workspace_size(mesh, est, nq, False)
            bws = torch.empty(nb, dtype=torch.uint8, device=dev)
            fn = lambda: sg.exp_map_backward(mesh, est, face, bary, v, po["face"], po["bary"], po["dir"], po["status"],
                                             g, workspace=bws)
            t = timed(fn, 3)
            res[f"bwd_{est}"] = {"ms": t, "geodesics_per_s": nq / (t * 1e-3)}
    clocks = clk.stop()
    # accuracy against the oracle on 2000 queries
    rng = np.random.default_rng(11)
    idx = np.sort(rng.choice(nq if sub64 is None else sub64, 2000, replace=False))
    om = oracle.Mesh(X32.astype(np.float64), F)
    f64 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    acc = {}
    refs = {}
    for name, o_kw in (("auto", {}), ("persistent", {}), ("fp32", {}), ("plain", {}), ("auto_1M", {}), ("mixed", {}),
                       ("fp64", {"tau_snap": 1e-12}), ("double_float", {"tau_snap": 1e-12})):
        if name not in outs:
            continue
        key = str(o_kw)
        if key not in refs:
            refs[key] = oracle.exp_map(om, q.face[idx], f64(q.bary[idx]), f64(q.v[idx]),
                                       f64(q.w[idx, :nw]) if nw else None, **o_kw)
        ref = refs[key]
        o = outs[name]
        st = o["status"][idx].cpu().numpy().astype(np.uint32)
        fl = ((st | ref["status"]) & 12) != 0
        err = np.linalg.norm(o["pos"][idx].cpu().numpy() - ref["pos"], axis=1) / meshgen.bbox_diag(X)
        same = o["face"][idx].cpu().numpy() == ref["face"]
        acc[name] = {"flagged": float(fl.mean()), "same_end_face_unflagged": float(same[~fl].mean()),
                     "max_pos_err_over_diag_unflagged": float(err[~fl].max()),
                     "median_pos_err_over_diag": float(np.median(err)),
                     "frac_within_1e-5_diag": float((err <= 1e-5).mean()),
                     "mixed_walk_fraction": float(((st & 4096) != 0).mean())}
        if "hash" in o:
            h = o["hash"][idx].cpu().numpy().view(np.uint64)
            acc[name]["same_face_sequence_unflagged"] = float((h == ref["hash"])[~fl].mean())
    name = {0: "icosphere-s3 1280F 4096q 1w", 1: "torus 512x256 262144F 4Mq 2w",
            4: "heightfield 1449^2 4.2MF slivers 16Mq"}[index]
    line = {"metric": "geodesics/s forward (library default)", "value": res["auto"]["geodesics_per_s"],
            "unit": "geodesics/s", "n_gpus": 1, "steps": steps, "warmup": args.warmup,
            "ms_per_step": res["auto"]["ms"], "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": name, "queries": nq, "faces": int(mesh.n_faces), "carried_vectors": nw,
                       "l2": "flushed between steps (512 MB write)"},
            "variants": res, "speedup_vs_plain": res["plain"]["ms"] / res["auto"]["ms"],
            "speedup_vs_double_float_1M": (res["double_float"]["ms"] / res["auto_1M"]["ms"]) if index == 4 else None,
            "accuracy_vs_oracle_2000": acc, "clocks": clocks}
    print(json.dumps(line), flush=True)
    if args.json_out:
        open(args.json_out, "w").write(json.dumps(line) + "\n")


def run_features(args):
    """Throughput of the features beyond the headline step, each on the workload named in its
    entry (CUDA events, L2 flushed between steps, median of the timed steps):
      trace      sg_exp_map_trace on the icosphere-s6 workload (1M queries, 64 path entries)
                 against sg_exp_map on the same queries;
      fp64       the full-precision walks (FP64, double-float, mixed) on the same workload against
                 the FP32 walk;
      hole       hole avoidance on the icosphere s6 with 8% of its faces removed (1M queries)
                 against the stopping walk;
      update     sg_mesh_update_vertices on the icosphere s6 (81,920 faces);
      k_step     exp_map_steps with K = 5 and a linear field on 1M queries, forward and
                 forward + GFD backward through all steps;
      field_steps  the fused K-step of a vertex-sampled field (sg_exp_map_steps, K = 5) against
                 K launches with the field evaluated by torch between them."""
    import torch
    import meshgen
    import paper_2603_15780_gb300 as sg
    dev = torch.device("cuda", 0)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    n_steps = max(3, min(args.steps, 20))

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        ts = []
        for _ in range(n_steps):
            torch.cuda.synchronize()
            flush.zero_()            # evicts L2; the timed work is enqueued behind it (not timed)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    T = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    wl = meshgen.workload(2)
    X, F = wl.single
    q = wl.queries
    nq = len(q)
    X32 = np.ascontiguousarray(X, np.float32)
    mesh = sg.Mesh(X32, F)
    face, bary, v = T(q.face, torch.int32), T(q.bary), T(q.v)
    res = {}
    out = sg.exp_map(mesh, face, bary, v)
    ws = out.pop("_workspace")
    t_fwd = timed(lambda: sg.exp_map(mesh, face, bary, v, workspace=ws, out=out))
    res["exp_map"] = {"ms": t_fwd, "geodesics_per_s": nq / (t_fwd * 1e-3)}
    t_tr = timed(lambda: sg.exp_map_trace(mesh, face, bary, v, path_cap=64, workspace=ws))
    res["trace"] = {"ms": t_tr, "geodesics_per_s": nq / (t_tr * 1e-3), "path_cap": 64,
                    "path_bytes_per_query": 64 * 16, "vs_exp_map": t_tr / t_fwd}
    o64 = sg.default_opts(precision=64)
    out64 = sg.exp_map(mesh, face, bary, v, opts=o64)
    ws64 = out64.pop("_workspace")
    t64 = timed(lambda: sg.exp_map(mesh, face, bary, v, opts=o64, workspace=ws64, out=out64))
    res["fp64"] = {"ms": t64, "geodesics_per_s": nq / (t64 * 1e-3), "vs_fp32": t64 / t_fwd}
    o48 = sg.default_opts(precision=48)
    out48 = sg.exp_map(mesh, face, bary, v, opts=o48)
    ws48 = out48.pop("_workspace")
    t48 = timed(lambda: sg.exp_map(mesh, face, bary, v, opts=o48, workspace=ws48, out=out48))
    res["double_float"] = {"ms": t48, "geodesics_per_s": nq / (t48 * 1e-3), "vs_fp32": t48 / t_fwd,
                           "vs_fp64": t64 / t48}
    o40 = sg.default_opts(precision=40)
    out40 = sg.exp_map(mesh, face, bary, v, opts=o40)
    ws40 = out40.pop("_workspace")
    t40 = timed(lambda: sg.exp_map(mesh, face, bary, v, opts=o40, workspace=ws40, out=out40))
    res["mixed"] = {"ms": t40, "geodesics_per_s": nq / (t40 * 1e-3), "vs_fp32": t40 / t_fwd,
                    "vs_double_float": t48 / t40}
    # update: positions with fresh radial noise
    rng = np.random.default_rng(5)
    Vn = T(X32 * (1.0 + 0.003 * rng.standard_normal((len(X32), 1))).astype(np.float32))
    Vo = T(X32)
    flip = [Vn, Vo]
    k = [0]

    def upd():
        mesh.update_vertices(flip[k[0] & 1])
        k[0] += 1
    t_up = timed(upd)
    mesh.update_vertices(Vo)
    res["update_vertices"] = {"ms": t_up, "faces": int(mesh.n_faces), "faces_per_s": mesh.n_faces / (t_up * 1e-3)}
    # K-step with a linear field
    A = torch.tensor(0.8 * rng.standard_normal((3, 3)), dtype=torch.float32, device=dev)
    t_k = timed(lambda: sg.exp_map_steps(mesh, face, bary, lambda x, kk: x @ A.T, 5, "gfd"))
    Ag = A.clone().requires_grad_(True)
    gK = torch.randn(nq, 3, device=dev)

    def kstep_bwd():
        xK = sg.exp_map_steps(mesh, face, bary, lambda x, kk: x @ Ag.T, 5, "gfd")[0]
        (xK * gK).sum().backward()
    t_kb = timed(kstep_bwd)
    res["k_step"] = {"K": 5, "fwd_ms": t_k, "fwd_bwd_gfd_ms": t_kb, "geodesics_per_s_fwd": 5 * nq / (t_k * 1e-3)}
    # K-step of a vertex-sampled field (u = the vertex values of x -> A x, interpolated in each
    # face): one fused launch (sg_exp_map_steps) against K sg_exp_map launches with the field
    # evaluated by torch between them, forward and forward + GFD backward through all steps
    Fd = torch.tensor(F, dtype=torch.int64, device=dev)
    U = (T(X32) @ A.T).contiguous()
    fs = sg.exp_map_field_steps(mesh, face, bary, U, 5)
    t_fs = timed(lambda: sg.exp_map_field_steps(mesh, face, bary, U, 5))
    Ug = U.clone().requires_grad_(True)
    bg = bary.clone().requires_grad_(True)

    def fused_bwd():
        xK = sg.ExpMapFieldSteps.apply(mesh, face, bg, Ug, 5)[0]
        (xK * gK).sum().backward()
    t_fsb = timed(fused_bwd)

    def loop(Uu, b0, grad=False):
        f, b = face, b0
        for _ in range(5):
            v = 0.2 * (b.clamp(min=0.0)[:, :, None] * Uu[Fd[f.long()]]).sum(1)
            x, f, b, _, _ = sg.ExpMap.apply(mesh, f, b, v, "gfd")
        return x

    def loop_fwd():
        with torch.no_grad():
            loop(U, bary)

    def loop_bwd():
        (loop(Ug, bg) * gK).sum().backward()
    t_lf = timed(loop_fwd)
    t_lb = timed(loop_bwd)
    res["field_steps"] = {"K": 5, "fused_fwd_ms": t_fs, "fused_fwd_bwd_gfd_ms": t_fsb, "loop_fwd_ms": t_lf,
                          "loop_fwd_bwd_gfd_ms": t_lb, "speedup_fwd": t_lf / t_fs, "speedup_fwd_bwd": t_lb / t_fsb,
                          "mixed_or_flagged": float(((fs["status"].cpu().numpy() & 12) != 0).mean())}
    # hole avoidance on the sphere with 8% of its faces removed
    rngh = np.random.default_rng(6)
    Xh, Fh = meshgen.remove_faces(X, F, 0.08, rngh)
    qh = meshgen.sample_queries(Xh, Fh, nq, rngh, 0.1, 1.0, 0)
    mh = sg.Mesh(np.ascontiguousarray(Xh, np.float32), Fh)
    fh, bh, vh = T(qh.face, torch.int32), T(qh.bary), T(qh.v)
    for name, o in (("stop", sg.default_opts()), ("hole", sg.default_opts(boundary_mode=1))):
        oh = sg.exp_map(mh, fh, bh, vh, opts=o)
        wsh = oh.pop("_workspace")
        th = timed(lambda: sg.exp_map(mh, fh, bh, vh, opts=o, workspace=wsh, out=oh))
        st = oh["status"].cpu().numpy()
        nc = float(oh["ncross"].sum().item())
        # the stopping walk ends at the first boundary it meets, hole avoidance walks the whole
        # length: crossings per second compare the two per unit of work
        res[f"holey_sphere_{name}"] = {"ms": th, "geodesics_per_s": nq / (th * 1e-3),
                                       "crossings_per_query": nc / nq, "crossings_per_s": nc / (th * 1e-3),
                                       "boundary_frac": float(((st & 1) != 0).mean()),
                                       "hole_frac": float(((st & 2048) != 0).mean())}
    line = {"metric": "feature throughput (see entries)", "value": res["trace"]["geodesics_per_s"],
            "unit": "geodesics/s", "n_gpus": 1, "steps": n_steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "icosphere-s6-noisy 81920F 1Mq (holey: 8% faces removed)",
                       "l2": "flushed between steps (512 MB write)"},
            "features": res}
    print(json.dumps(line), flush=True)
    if args.json_out:
        open(args.json_out, "w").write(json.dumps(line) + "\n")


# ----------------------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=262144)
    ap.add_argument("--cpu-sample", type=int, default=1048576)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="time the step as eager launches, not a CUDA graph")
    ap.add_argument("--no-probe", action="store_true", help="skip the 32-B gather ceilings measured after the timed steps")
    ap.add_argument("--kernel", type=int, default=None,
                    help="1 plain, 2 persistent; giving --kernel, --sort or --block skips the autotuner")
    ap.add_argument("--sort", type=int, default=None, help="1 on, 0 off, -1 the library's automatic choice")
    ap.add_argument("--block", type=int, default=None)
    ap.add_argument("--fp64", type=int, default=1)
    ap.add_argument("--json-out", default=None)
    ap.add_argument("--no-autotune", action="store_true",
                    help="the library's default launch options instead of the autotuner's pick")
    ap.add_argument("--workload", default="fwdbwd",
                    choices=["fwdbwd", "multimesh", "icosphere-s3", "torus", "heightfield", "features"],
                    help="fwdbwd: the headline step; multimesh: 64 uneven meshes, plain per-mesh launches vs "
                         "one graph-captured persistent launch")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        run_reference(args)
        return

    import torch
    import torch.distributed as dist
    import paper_2603_15780_gb300 as sg
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "features":
        run_features(args)
        return
    if args.workload in ("icosphere-s3", "torus", "heightfield"):
        run_config(args, {"icosphere-s3": 0, "torus": 1, "heightfield": 4}[args.workload])
        return
    if args.workload == "multimesh":
        if rank == 0:
            run_multimesh(args)
        return
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    wl, X32, F = load_workload()
    q = rank_queries(wl, X32, F, rank)
    nq = len(q)
    mesh = sg.Mesh(X32, F)
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a, np.float32), device=dev)
    face = torch.tensor(q.face, device=dev)
    bary, v, g = f32(q.bary), f32(q.v), f32(q.g_pos)
    # The forward's launch options: the autotuner's pick on this batch (kernel shape, block, queries
    # per thread, query order; timed before and outside the timed region), unless options are given.
    tuned = None
    if args.kernel is None and args.sort is None and args.block is None and not args.no_autotune:
        from paper_2603_15780_gb300 import autotune
        best, table = autotune.tune(mesh, face, bary, v, reps=5, fp64_escalate=args.fp64)
        args.kernel, args.sort, args.block = best.kernel, best.sort, best.block
        tuned = {"pick": {k: getattr(best, k) for k in ("kernel", "block", "sort", "queries_per_thread")},
                 "candidates": len(table), "pick_ms": min(t for _, t in table),
                 "default_ms": next((t for c, t in table if c["kernel"] == 2 and c["block"] == 256 and c["sort"] == -1
                                     and c["queries_per_thread"] == 0), None)}
    # the backward's query order: the library's automatic choice unless --sort is given (the
    # autotuner times the forward only)
    bsort = -1 if (tuned is not None or args.sort is None) else args.sort
    args.kernel = 2 if args.kernel is None else args.kernel
    args.sort = -1 if args.sort is None else args.sort
    args.block = 0 if args.block is None else args.block
    qpt = tuned["pick"]["queries_per_thread"] if tuned else 0
    # The query order the forward's options give, as the library decides it: by start face (5
    # sort/scan kernels) when the mesh's records (128 B per face) exceed half of L2, else by walk
    # length (2 kernels), input order for the plain kernel and small batches.  The forward writes
    # the length order into `qorder` (its own queue's, or two more launches after another order)
    # and the GFD backward's re-walk takes the queries in that order (sg_opts.order) instead of
    # sorting them again.
    if args.kernel == 1:
        sort_mode = 0
    elif args.sort >= 0:
        sort_mode = args.sort
    else:
        l2 = torch.cuda.get_device_properties(dev).L2_cache_size
        sort_mode = 0 if nq < 65536 else (1 if 128 * mesh.n_faces > l2 // 2 else 2)
    qorder = torch.empty(nq, dtype=torch.int32, device=dev)
    opts = sg.default_opts(kernel=args.kernel, sort=args.sort, fp64_escalate=args.fp64,
                           block=args.block if args.block > 0 else None, queries_per_thread=qpt)
    opts.order = qorder.data_ptr()   # the workspace is sized with the order buffer in use
    ws = torch.empty(sg.workspace_size(mesh, nq, opts), dtype=torch.uint8, device=dev)
    bopts = sg.default_opts(sort=bsort)
    bws = torch.empty(sg.backward_workspace_size(mesh, "gfd", nq, True), dtype=torch.uint8, device=dev)
    # per-kernel events recorded by the library around its walk kernels (forward walk, GFD re-walk)
    kev = {k: [torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)] for k in ("walk", "rewalk")}
    for pair in kev.values():
        for e in pair:
            e.record()
    import ctypes
    kh = {k: (ctypes.c_void_p * 2)(pair[0].cuda_event, pair[1].cuda_event) for k, pair in kev.items()}
    popts = sg.default_opts(kernel=args.kernel, sort=args.sort, fp64_escalate=args.fp64,
                            block=args.block if args.block > 0 else None, queries_per_thread=qpt)
    popts.prof_events = ctypes.addressof(kh["walk"])
    pbopts = sg.default_opts(sort=bsort)
    pbopts.prof_events = ctypes.addressof(kh["rewalk"])
    out = {"face": torch.empty(nq, dtype=torch.int32, device=dev), "bary": torch.empty(nq, 3, device=dev),
           "pos": torch.empty(nq, 3, device=dev), "dir": torch.empty(nq, 3, device=dev),
           "status": torch.empty(nq, dtype=torch.int32, device=dev),
           "ncross": torch.empty(nq, dtype=torch.int32, device=dev)}
    gV = torch.zeros(mesh.n_vertices, 3, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    # The two backward estimators are independent calls on the forward's outputs: EP runs on a
    # second stream (its own workspace) beside GFD and fills the SMs the GFD kernels leave idle in
    # their tails; the step ends when both are done.
    ep_stream = torch.cuda.Stream(device=dev)
    ews = torch.empty(sg.backward_workspace_size(mesh, "ep", nq, False), dtype=torch.uint8, device=dev)

    def step(ev=None, epev=None):
        stream = torch.cuda.current_stream()  # the capture stream while the step is captured
        if ev is not None:
            ev[0].record(stream)
        sg.exp_map(mesh, face, bary, v, out=out, workspace=ws, opts=popts if ev is not None else opts, order=qorder)
        if ev is not None:
            ev[1].record(stream)
        fdone = torch.cuda.Event()
        fdone.record(stream)
        ep_stream.wait_event(fdone)
        with torch.cuda.stream(ep_stream):
            if epev is not None:
                epev[0].record(ep_stream)
            sg.exp_map_backward(mesh, "ep", face, bary, v, out["face"], out["bary"], out["dir"], out["status"], g,
                                opts=bopts, workspace=ews)
            if epev is not None:
                epev[1].record(ep_stream)
            edone = torch.cuda.Event()
            edone.record(ep_stream)
        if ev is not None:
            ev[2].record(stream)
        gV.zero_()
        if ev is not None:
            ev[3].record(stream)
        r = sg.exp_map_backward(mesh, "gfd", face, bary, v, out["face"], out["bary"], out["dir"], out["status"], g,
                                eps_v=EPS, eps_p=EPS, grad_V=gV, opts=pbopts if ev is not None else bopts,
                                workspace=bws, order=qorder)
        stream.wait_event(edone)
        if ev is not None:
            ev[4].record(stream)
        return r

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ncross = int(out["ncross"].sum().item())
    st = out["status"].cpu().numpy().astype(np.uint32)

    clk = Clocks(local, os.path.join(CLOCKS_DIR, f"clocks_r{rank}.csv"))
    times = np.zeros((args.steps, 4))
    ep_own = np.zeros(args.steps)
    ktimes = {"walk": [], "rewalk": []}
    for k in range(args.steps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        # evict L2 between timed iterations (not timed); the step is enqueued while the flush
        # runs, so its events time the device work and not the host's first launch
        flush.zero_()
        epev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        step(ev, epev)
        torch.cuda.synchronize()
        times[k] = [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3]),
                    ev[3].elapsed_time(ev[4])]
        ep_own[k] = epev[0].elapsed_time(epev[1])
        for kk, pair in kev.items():
            ktimes[kk].append(pair[0].elapsed_time(pair[1]))
    eager_ms = float(times.sum()) / args.steps

    # ---- the timed steps: the step captured once as a CUDA graph and replayed (its launches and
    # memsets leave the host), checked against the eager step's per-query gradients first
    graph = None
    if not args.no_graph:
        cap = torch.cuda.Stream(device=dev)
        cap.wait_stream(stream)
        with torch.cuda.stream(cap):
            for _ in range(2):
                step()
        stream.wait_stream(cap)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=cap):
            r_graph = step()
        eager_r = step()
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        for key in ("grad_v", "grad_p", "grad_bary", "status"):
            if not torch.equal(r_graph[key], eager_r[key]):
                raise RuntimeError(f"graph replay differs from the eager step in {key}")
        gms = np.zeros(args.steps)
        for k in range(args.steps):
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            flush.zero_()  # evicts L2 (not timed); the replay is enqueued behind it
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            torch.cuda.synchronize()
            gms[k] = e0.elapsed_time(e1)
    clocks = clk.stop()
    total_ms = max_over_ranks(float(gms.sum() if graph is not None else times.sum()), world, dev)
    if world > 1:
        dist.barrier()
    ms_step = total_ms / args.steps
    value = world * nq / (ms_step * 1e-3)
    fwd_ms, ep_ms, gfd_ms = times[:, 0].mean(), float(ep_own.mean()), times[:, 3].mean()

    # ---- end to end through the public API with host buffers (pinned), copies timed.  The steps
    # run as a serving loop runs them: step k+1's inputs go up on a copy stream while step k
    # computes, and step k's results come down on another while step k+1 computes (two buffer
    # slots, each with its step captured as a CUDA graph reading the slot's device buffers).  One
    # pair of events spans all timed steps, so every step's copies lie inside the timed region,
    # and so does the L2 flush that precedes every step's compute.
    e2e = None
    if not args.no_e2e:
        hb = {k: torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for k, a in
              {"face": q.face, "bary": q.bary.astype(np.float32), "v": q.v.astype(np.float32),
               "g": q.g_pos.astype(np.float32)}.items()}
        host_out = [{"grad_v": torch.empty(nq, 3).pin_memory(), "grad_p": torch.empty(nq, 3).pin_memory(),
                     "pos": torch.empty(nq, 3).pin_memory()} for _ in range(2)]
        h2d = sum(t.numel() * t.element_size() for t in hb.values())
        d2h = sum(t.numel() * t.element_size() for t in host_out[0].values())
        up, down = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
        dev_in = [{k: torch.empty_like(t, device=dev) for k, t in hb.items()} for _ in range(2)]
        free = [torch.cuda.Event(), torch.cuda.Event()]     # slot's inputs no longer read
        for ev in free:
            ev.record(stream)
        outs_done = [torch.cuda.Event(), torch.cuda.Event()]  # slot's results copied to the host
        for ev in outs_done:
            ev.record(stream)

        def compute(di):
            cs = torch.cuda.current_stream()
            o = sg.exp_map(mesh, di["face"], di["bary"], di["v"], workspace=ws, opts=opts, order=qorder)
            fdone = torch.cuda.Event()
            fdone.record(cs)
            ep_stream.wait_event(fdone)
            with torch.cuda.stream(ep_stream):
                sg.exp_map_backward(mesh, "ep", di["face"], di["bary"], di["v"], o["face"], o["bary"], o["dir"],
                                    o["status"], di["g"], opts=bopts, workspace=ews)
                edone = torch.cuda.Event()
                edone.record(ep_stream)
                if not torch.cuda.is_current_stream_capturing():
                    for t in (o["face"], o["bary"], o["dir"], o["status"]):
                        t.record_stream(ep_stream)
            gV.zero_()
            r = sg.exp_map_backward(mesh, "gfd", di["face"], di["bary"], di["v"], o["face"], o["bary"], o["dir"],
                                    o["status"], di["g"], eps_v=EPS, eps_p=EPS, grad_V=gV, opts=bopts,
                                    workspace=bws, order=qorder)
            cs.wait_event(edone)
            return o, r

        # with graphs, one captured step per buffer slot (its inputs are the slot's device buffers)
        graphs, static = None, None
        if not args.no_graph:
            for sl in range(2):
                for name, t in hb.items():
                    dev_in[sl][name].copy_(t)
            cap = torch.cuda.Stream(device=dev)
            cap.wait_stream(stream)
            with torch.cuda.stream(cap):
                compute(dev_in[0])
            stream.wait_stream(cap)
            torch.cuda.synchronize()
            graphs, static = [], []
            for sl in range(2):
                gr = torch.cuda.CUDAGraph()
                with torch.cuda.graph(gr, stream=cap):
                    static.append(compute(dev_in[sl]))
                graphs.append(gr)
            torch.cuda.synchronize()

        def e2e_step(k):
            sl = k & 1
            di, ho = dev_in[sl], host_out[sl]
            up.wait_event(free[sl])
            with torch.cuda.stream(up):
                for name, t in hb.items():
                    di[name].copy_(t, non_blocking=True)
                ready = torch.cuda.Event()
                ready.record(up)
            flush.zero_()
            stream.wait_event(ready)
            if graphs is not None:
                stream.wait_event(outs_done[sl])  # the slot's last results are on the host
                graphs[sl].replay()
                o, r = static[sl]
            else:
                o, r = compute(di)
            free[sl].record(stream)
            done = torch.cuda.Event()
            done.record(stream)
            down.wait_event(done)
            down.wait_event(outs_done[sl])
            with torch.cuda.stream(down):
                for name, t in (("pos", o["pos"]), ("grad_v", r["grad_v"]), ("grad_p", r["grad_p"])):
                    ho[name].copy_(t, non_blocking=True)
                    if graphs is None:
                        t.record_stream(down)
                outs_done[sl].record(down)

        for k in range(2):  # untimed: both slots warm
            e2e_step(k)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        up.wait_event(e0)
        for k in range(args.steps):
            e2e_step(k)
        stream.wait_stream(down)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e = {"value": args.steps * nq / (e0.elapsed_time(e1) * 1e-3), "unit": "geodesics/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "pipelined": "step k+1 uploads and step k-1 downloads overlap step k; L2 flush inside",
               "launch": "eager" if graphs is None else "one captured CUDA graph per buffer slot"}

    launches_per_step = 10 + {0: 2, 1: 7, 2: 2}[sort_mode]

    # ---- roofline of the dominant kernel (algorithmic bytes per launch / measured launch time)
    # Algorithmic bytes as the measurement plan defines them: the 32-B record of every face a walk
    # enters, plus each query's own input and output.  Forward walk, per query: inputs (face,
    # bary, v: 28 B), the start and end frame gathers (48 B each), the outputs (face, bary, pos,
    # dir, status, ncross: 48 B).  GFD re-walk with the vertex gradient, per query: inputs (28 B),
    # start face record, frame, vertex ids and vertices (128 B), the forward end state and upstream
    # gradient with the end frame (64 B), the end face record (32 B), start/end vertex atomics
    # (6 x 16 B), the end-face frame and ids (48 B), status (4 B): 400 B.  The re-walk's 8-B edge
    # atomic per crossing (the vertex gradient's accumulation) is reported as a separate term.
    peak_hbm, peak_kind = peaks()
    walk_bytes = ncross * RECORD_BYTES + nq * (28 + 2 * 48 + 48)
    rewalk_bytes = ncross * RECORD_BYTES + nq * 400
    rewalk_atomic_bytes = ncross * 8
    kern = {("k_walk_persistent" if args.kernel == 2 else "k_walk_plain"): (walk_bytes, float(np.mean(ktimes["walk"]))),
            "k_bwd_rewalk": (rewalk_bytes, float(np.mean(ktimes["rewalk"])))}
    dom = max(kern, key=lambda k: kern[k][1])
    achieved = kern[dom][0] / (kern[dom][1] * 1e-3) / 1e9
    l2_gather = None if args.no_probe else gather_ceilings(ncross, ktimes)
    # The icosphere's records (10.5 MB) stay in L2, so the walks are bound by L2 gathers, not HBM:
    # the ceiling is the device's measured rate of independent 32-B record gathers from an
    # L2-resident table, one 256-bit load per record (the walks' load).  HBM-normalised figures
    # (the measured HBM copy bandwidth) are kept beside it.
    hbm_norm = {"achieved": achieved, "peak": peak_hbm, "unit": "GB/s", "frac": achieved / peak_hbm,
                "peak_kind": peak_kind}
    if l2_gather is not None:
        l2_peak = l2_gather["random_GBps"]["1x32B"]
        roofline = {"bound": "l2", "kernel": dom, "achieved": achieved, "peak": l2_peak, "unit": "GB/s",
                    "frac": achieved / l2_peak,
                    "peak_kind": "measured in this run: independent 32-B record gathers from an L2-resident "
                                 "16 MiB table, one 256-bit load each (l2_gather.random_GBps.1x32B)",
                    "hbm_normalised": hbm_norm}
    else:
        roofline = dict(hbm_norm, bound="hbm", kernel=dom)
    roofline.update({"traffic": ncu_traffic(dom), "algorithmic_bytes_per_launch": int(kern[dom][0]),
                     "launch_ms": kern[dom][1], "crossings_per_launch": int(ncross), "queries_per_launch": nq})
    # The same kernel counted in L2 requests (ncu's lts__t_requests of the committed capture, null
    # once the kernel changed): record reads, edge reductions and query I/O, each a request, against
    # the request rate of the gather probe (one request per 32-B gather).
    nreq = ncu_traffic(dom, "lts_requests_per_launch")
    if nreq is not None and l2_gather is not None:
        peak_req = l2_gather["random_GBps"]["1x32B"] * 1e9 / 32
        ach_req = nreq / (kern[dom][1] * 1e-3)
        roofline["l2_requests"] = {"per_launch": int(nreq), "achieved_per_s": ach_req, "peak_per_s": peak_req,
                                   "frac": ach_req / peak_req,
                                   "source": "ncu lts__t_requests.sum of the committed capture; peak: the gather "
                                             "probe's 32-B gathers per second"}
    if dom == "k_bwd_rewalk":
        roofline["atomic_bytes_per_launch"] = int(rewalk_atomic_bytes)
    kernels = {k: {"ms": t, "algorithmic_GBps": b / (t * 1e-3) / 1e9, "frac_of_hbm": b / (t * 1e-3) / 1e9 / peak_hbm}
               for k, (b, t) in kern.items()}
    if l2_gather is not None:
        for k in kernels:
            kernels[k]["frac_of_l2_gather"] = kernels[k]["algorithmic_GBps"] / l2_gather["random_GBps"]["1x32B"]

    line = {"metric": METRIC, "value": value, "unit": "geodesics/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "icosphere-s6-noisy 81920F 1Mq fwd+EP+GFD+gradV", "global_batch": world * nq,
                       "faces": int(len(F)), "queries_per_gpu": nq, "l2": "flushed between steps (512 MB write)",
                       "kernel": "persistent" if args.kernel == 2 else "plain",
                       "autotuned": tuned,
                       "query_order": {0: "input", 1: "start face", 2: "walk length"}[sort_mode],
                       "bwd_query_order": "walk length, written by the forward (sg_opts.order)",
                       "fp64_classification": bool(args.fp64),
                       "launch": "eager" if graph is None else "CUDA graph of the step, captured once and replayed"},
            "crossings_per_s": world * ncross / (float(np.mean(ktimes["walk"])) * 1e-3),
            "fwd_geodesics_per_s": world * nq / (fwd_ms * 1e-3),
            "phase_ms": {"fwd": fwd_ms, "ep_bwd": ep_ms, "gfd_bwd_gradV": gfd_ms, "eager_step": eager_ms,
                         "note": "eager launches with per-phase events; ep_bwd runs on a second stream beside "
                                 "gfd_bwd_gradV (its own interval)"},
            "crossings_per_query": ncross / nq,
            "flag_fraction": {"near_vertex": float(((st & 4) != 0).mean()), "near_edge": float(((st & 8) != 0).mean()),
                              "fp64": float(((st & 32) != 0).mean())},
            "gpu_launches": args.steps * launches_per_step,
            "roofline": roofline, "kernels": kernels, "clocks": clocks, "e2e": e2e}
    if l2_gather is not None:
        line["l2_gather"] = l2_gather
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        n, dt, _ = oracle_sample(args.cpu_sample, threads)
        line["cpu_baseline"] = {"value": n / dt, "unit": "geodesics/s", "cores": threads, "kind": "oracle",
                                "sample": f"first {n} of the 1,048,576 queries, fwd+EP+GFD, {dt:.1f} s"}
        n1, dt1, _ = oracle_sample(min(args.cpu_sample, 65536), 1)
        line["cpu_baseline"]["one_core"] = {"value": n1 / dt1, "unit": "geodesics/s", "cores": 1,
                                            "sample": f"first {n1} queries, fwd+EP+GFD, {dt1:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
        if args.json_out:
            open(args.json_out, "w").write(json.dumps(line) + "\n")
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
