"""Launch-configuration autotuner and CUDA-graph capture for sg_exp_map.

`tune(mesh, face, bary, v, ...)` times candidate launch configurations of the forward
walk on the caller's own batch (CUDA events on the current stream, median of `reps`) and
returns the fastest `Opts`: kernel shape (plain one-thread-per-query or persistent),
threads per block, persistent residency (blocks per SM, which sets how many queries each
thread takes from the queue) and the start-face sort.  Results are cached per
(mesh, batch size bucket, carried vectors).

`GraphedExpMap` captures one sg_exp_map call (static input/output/workspace buffers) into a
torch.cuda.CUDAGraph so a fixed-shape batch -- e.g. many meshes of uneven size in one
persistent launch -- replays with a single graph launch.
"""
from __future__ import annotations

import itertools
import math

from . import (KERNEL_PERSISTENT, KERNEL_PLAIN, Mesh, SgError, default_opts, exp_map, workspace_size)

_cache: dict = {}


def candidates(fp64_escalate: int = 1):
    """The search space: plain kernel at 3 block sizes; persistent kernel at 3 block sizes x
    residency {auto, 2, 1 blocks/SM} x sort {on, off}."""
    out = []
    for block in (64, 128, 256):
        out.append(dict(kernel=KERNEL_PLAIN, block=block, sort=0, fp64_escalate=0, blocks_per_sm=0))
    for block, per, sort in itertools.product((64, 128, 256), (0, 2, 1), (1, 0)):
        out.append(dict(kernel=KERNEL_PERSISTENT, block=block, sort=sort, fp64_escalate=fp64_escalate,
                        blocks_per_sm=per))
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
        ws = None
        if o.kernel != KERNEL_PLAIN:
            ws = torch.empty(workspace_size(mesh, nq, o), dtype=torch.uint8, device=face.device)
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
