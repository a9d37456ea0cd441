"""Launch-configuration autotuner and CUDA-graph capture for sg_exp_map.

`tune(mesh, face, bary, v, ...)` times candidate launch configurations of the forward
walk on the caller's own batch (CUDA events on the current stream, median of `reps`) and
returns the fastest `Opts`: kernel shape (plain or persistent), threads per block, queries
per thread and the query order.  Queries per thread is the plain kernel's grid-stride count
(1 = the paper's one thread per query) and, for the persistent kernel, the average number of
queries each thread takes from the queue (it sets the grid: blocks per SM = nq / (qpt x SMs x
block), capped by the occupancy limit; 0 = as many resident blocks as fit).  Results are
cached per (mesh, batch size bucket, carried vectors).

`GraphedExpMap` captures one sg_exp_map call (static input/output/workspace buffers) into a
torch.cuda.CUDAGraph so a fixed-shape batch -- e.g. many meshes of uneven size in one
persistent launch -- replays with a single graph launch.
"""
from __future__ import annotations

import itertools
import math

from . import KERNEL_PERSISTENT, KERNEL_PLAIN, Mesh, SgError, default_opts, exp_map, workspace_size

_cache: dict = {}


def candidates(fp64_escalate: int = 1):
    """The search space: the plain kernel at 3 block sizes x {1, 2, 4} queries per thread; the
    persistent kernel at 2 block sizes x {all resident, 32, 8} queries per thread x query order
    {the library's automatic choice, start face, input order}."""
    out = []
    for block, qpt in itertools.product((64, 128, 256), (1, 2, 4)):
        out.append(dict(kernel=KERNEL_PLAIN, block=block, sort=0, fp64_escalate=0, queries_per_thread=qpt))
    for block, qpt, sort in itertools.product((128, 256), (0, 32, 8), (-1, 1, 0)):
        out.append(dict(kernel=KERNEL_PERSISTENT, block=block, sort=sort, fp64_escalate=fp64_escalate,
                        queries_per_thread=qpt))
    return out


def _time(fn, reps):
    import torch
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts.sort()
    return ts[len(ts) // 2]


def tune(mesh: Mesh, face, bary, v, w=None, mesh_id=None, *, reps: int = 5, fp64_escalate: int = 1,
         space=None, key=None, verbose: bool = False):
    """Return (best Opts, table of (config, ms)).  Inputs are torch CUDA tensors."""
    import torch
    nq = face.numel()
    nw = 0 if w is None else w.shape[1]
    k = key if key is not None else (id(mesh), int(math.log2(max(nq, 1))), nw, fp64_escalate)
    if k in _cache:
        return _cache[k]
    out = exp_map(mesh, face, bary, v, w, mesh_id=mesh_id)  # also allocates outputs once
    out.pop("_workspace", None)
    table = []
    for cfg in (space or candidates(fp64_escalate)):
        o = default_opts(**cfg)
        ws = torch.empty(max(workspace_size(mesh, nq, o), 1), dtype=torch.uint8, device=face.device)
        try:
            fn = lambda: exp_map(mesh, face, bary, v, w, mesh_id=mesh_id, opts=o, workspace=ws, out=out)
            fn()
            torch.cuda.synchronize()
            ms = _time(fn, reps)
        except SgError:
            continue
        table.append((cfg, ms))
        if verbose:
            print(f"  {cfg} {ms:.3f} ms")
    best_cfg, _ = min(table, key=lambda t: t[1])
    best = default_opts(**best_cfg)
    _cache[k] = (best, table)
    return best, table


class GraphedExpMap:
    """One sg_exp_map call captured in a CUDA graph over static buffers.

        g = GraphedExpMap(mesh, face, bary, v, mesh_id=mesh_id, opts=opts)
        g.inputs["v"].copy_(new_v); g.replay(); g.outputs["pos"]
    """

    def __init__(self, mesh: Mesh, face, bary, v, w=None, mesh_id=None, opts=None):
        import torch
        self.mesh = mesh
        self.inputs = {"face": face.clone(), "bary": bary.clone(), "v": v.clone(),
                       "w": None if w is None else w.clone(),
                       "mesh_id": None if mesh_id is None else mesh_id.clone()}
        nq = face.numel()
        self.opts = opts if opts is not None else default_opts()
        self.workspace = torch.empty(max(workspace_size(mesh, nq, self.opts), 1), dtype=torch.uint8,
                                     device=face.device)
        self.outputs = exp_map(mesh, **self._args())
        self.outputs.pop("_workspace", None)
        torch.cuda.synchronize()
        self.stream = torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(self.stream):
            exp_map(mesh, **self._args(), out=self.outputs)   # warm-up on the capture stream
            torch.cuda.synchronize()
            with torch.cuda.graph(self.graph, stream=self.stream):
                exp_map(mesh, **self._args(), out=self.outputs, stream=self.stream)
        torch.cuda.current_stream().wait_stream(self.stream)

    def _args(self):
        i = self.inputs
        return dict(face=i["face"], bary=i["bary"], v=i["v"], w=i["w"], mesh_id=i["mesh_id"], opts=self.opts,
                    workspace=self.workspace)

    def replay(self):
        self.graph.replay()
        return self.outputs
