"""Helpers shared by the GPU parity tests: run the CUDA library and the FP64 oracle on the
same float32 inputs and compare them element by element.

Tolerances (stated once, used by every forward parity test):
  end point     |pos_gpu - pos_oracle| <= 1e-5 * bbox diagonal (the target accuracy of the
                FP32 walk against the FP64 oracle)
  face, hash,   bit-exact on every query that neither side flags NEAR_VERTEX / NEAR_EDGE
  ncross        (a flagged query passed within tau_near * l_ref of a vertex, or ended that
                close to an edge, where FP32 and FP64 may legitimately pick different faces)
  direction,    |.|_inf <= 2e-4 (unit vectors); the FP32 direction error grows like
  carried w     sqrt(#crossings) * 1e-7 rad times curvature amplification along the path
"""
from __future__ import annotations

import numpy as np

import oracle

FLAGS = oracle.NEAR_VERTEX | oracle.NEAR_EDGE


def as_f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def run_gpu(mesh, q, nw, mesh_id=None, length=None, **kw):
    import paper_2603_15780_gb300 as sg
    import torch
    w = as_f32(q.w[:, :nw]) if nw else None
    out = sg.exp_map(mesh, q.face, as_f32(q.bary), as_f32(q.v), w, length=length, mesh_id=mesh_id,
                     want_hash=True, **kw)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items() if k != "_workspace" and v is not None}
    res["status"] = res["status"].astype(np.uint32)
    res["hash"] = res["hash"].view(np.uint64)
    return res


def run_oracle(X32, F, q, nw, length=None, **kw):
    om = oracle.Mesh(np.asarray(X32, np.float64), F)
    w = as_f32(q.w[:, :nw]).astype(np.float64) if nw else None
    ref = oracle.exp_map(om, q.face, as_f32(q.bary).astype(np.float64), as_f32(q.v).astype(np.float64), w,
                         length=None if length is None else np.asarray(length, np.float32).astype(np.float64),
                         **kw)
    return ref, om


def compare(gpu, ref, diag, nw, *, max_flagged=0.05, pos_tol=1e-5, dir_tol=2e-4, what=""):
    st_g, st_o = gpu["status"], ref["status"]
    flagged = ((st_g | st_o) & FLAGS) != 0
    ok = ~flagged
    frac = flagged.mean()
    assert frac <= max_flagged, f"{what}: flagged fraction {frac:.4f}"
    # discrete results: bit-exact on unflagged queries
    bad = np.nonzero(ok & (gpu["face"] != ref["face"]))[0]
    assert len(bad) == 0, f"{what}: end face differs on {len(bad)} unflagged queries, e.g. {bad[:5]}"
    bad = np.nonzero(ok & (gpu["hash"] != ref["hash"]))[0]
    assert len(bad) == 0, f"{what}: face sequence differs on {len(bad)} unflagged queries, e.g. {bad[:5]}"
    bad = np.nonzero(ok & (gpu["ncross"] != ref["ncross"]))[0]
    assert len(bad) == 0, f"{what}: crossing count differs on {len(bad)} queries"
    keep_bits = oracle.BOUNDARY | oracle.VERTEX_HIT | oracle.INVALID | oracle.MAX_STEPS
    bad = np.nonzero(ok & ((st_g & keep_bits) != (st_o & keep_bits)))[0]
    assert len(bad) == 0, f"{what}: status differs on {len(bad)} queries, e.g. {bad[:5]} {st_g[bad[:5]]} {st_o[bad[:5]]}"
    # continuous results: end point within 1e-5 of the bbox diagonal, also on NEAR_EDGE-only
    # queries (the point is the same whichever face it is reported in)
    near_v = ((st_g | st_o) & oracle.NEAR_VERTEX) != 0
    cmp_pos = ~near_v
    dpos = np.linalg.norm(gpu["pos"] - ref["pos"], axis=1)
    assert dpos[cmp_pos].max() <= pos_tol * diag, f"{what}: max pos err {dpos[cmp_pos].max():.3e} (diag {diag:.3f})"
    ddir = np.abs(gpu["dir"] - ref["dir"])[ok].max() if ok.any() else 0.0
    assert ddir <= dir_tol, f"{what}: max dir err {ddir:.3e}"
    if nw:
        dw = np.abs(gpu["w"] - ref["w"])[ok].max()
        assert dw <= dir_tol, f"{what}: max carried-vector err {dw:.3e}"
    return {"flagged": float(frac), "max_pos_err": float(dpos[cmp_pos].max()), "max_dir_err": float(ddir),
            "mean_pos_err": float(dpos[cmp_pos].mean())}


def check_flag_semantics(gpu, ref, lref, tau_near=1e-4):
    """Queries whose oracle margin is far above the flag radius must not be flagged by the
    GPU; queries far below it must be flagged (or snapped) by the GPU -- checked where the
    GPU's own state error (bounded by its end-point error) is below a tenth of the band."""
    m = ref["margin"]
    st_g = gpu["status"]
    clear = m > 10 * tau_near
    assert not np.any(clear & ((st_g & oracle.NEAR_VERTEX) != 0) & ((ref["status"] & oracle.VERTEX_HIT) == 0))
    accurate = np.linalg.norm(gpu["pos"] - ref["pos"], axis=1) < 0.1 * tau_near * lref
    close = (m < 0.1 * tau_near) & accurate & ((ref["status"] & (oracle.VERTEX_HIT | oracle.INVALID)) == 0)
    assert np.all((st_g[close] & (oracle.NEAR_VERTEX | oracle.VERTEX_HIT)) != 0)
