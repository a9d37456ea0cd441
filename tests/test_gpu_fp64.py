"""GPU parity of the full-precision walk (sg_opts.precision = 64) against the FP64 oracle.

On the sliver heightfield of workload 4 (~1.4k crossings per walk) the FP32 walk's accumulated
state error (~1e-6 of l_ref) exceeds the near-vertex band, so FP32 and FP64 pass some vertices
on different sides.  The FP64 walk keeps its error near 1e-13, so with a near-vertex band of
1e-8 l_ref on both sides its face sequences must equal the oracle's on every unflagged query.
"""
import numpy as np
import pytest

import meshgen
import oracle
from tests import parity

pytestmark = pytest.mark.gpu


def sg():
    import paper_2603_15780_gb300 as m
    return m


def test_fp64_walk_on_the_sliver_heightfield():
    wl = meshgen.workload(4, scale=20000 / 16777216)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    q = wl.queries
    tau = 1e-8
    g64 = parity.run_gpu(mesh, q, 0, precision=64, tau_near=tau)
    g32 = parity.run_gpu(mesh, q, 0, tau_near=tau)
    ref, _ = parity.run_oracle(X32, F, q, 0, tau_near=tau)
    diag = meshgen.bbox_diag(X)
    flag64 = ((g64["status"] | ref["status"]) & parity.FLAGS) != 0
    flag32 = ((g32["status"] | ref["status"]) & parity.FLAGS) != 0
    assert flag64.mean() < 0.01
    same64 = (g64["hash"] == ref["hash"]) & (g64["face"] == ref["face"]) & (g64["ncross"] == ref["ncross"])
    same32 = (g32["hash"] == ref["hash"]) & (g32["face"] == ref["face"])
    print("fp64 same", same64[~flag64].mean(), "fp32 same", same32[~flag32].mean(),
          "mean ncross", ref["ncross"].mean())
    assert same64[~flag64].all()
    assert np.array_equal(g64["status"][~flag64] & ~np.uint32(32), ref["status"][~flag64])
    err = np.linalg.norm(g64["pos"] - ref["pos"], axis=1)[~flag64] / diag
    assert err.max() <= 1e-6, err.max()
    # the FP32 walk diverges on many of these walks; the FP64 walk on none
    assert (~same32[~flag32]).sum() > 100


def test_fp64_walk_workload0_parity_with_carried_vectors():
    wl = meshgen.workload(0)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    g = parity.run_gpu(mesh, wl.queries, 1, precision=64)
    ref, _ = parity.run_oracle(X32, F, wl.queries, 1)
    parity.compare(g, ref, meshgen.bbox_diag(X), 1, what="fp64 workload 0", pos_tol=1e-6, dir_tol=1e-5)


def test_fp64_geometry_follows_vertex_updates():
    rng = np.random.default_rng(91)
    XA, F = meshgen.icosphere(4, 0.004, rng)
    XB, _ = meshgen.icosphere(4, 0.004, rng)
    q = meshgen.sample_queries(XB, F, 5000, rng, 0.0, 2.0, 1)
    mesh = sg().Mesh(parity.as_f32(XA), F)
    parity.run_gpu(mesh, q, 1, precision=64)            # builds the FP64 geometry of A
    mesh.update_vertices(parity.as_f32(XB))
    moved = parity.run_gpu(mesh, q, 1, precision=64)
    fresh = parity.run_gpu(sg().Mesh(parity.as_f32(XB), F), q, 1, precision=64)
    for k in ("face", "status", "hash", "ncross"):
        assert np.array_equal(moved[k], fresh[k]), k
    for k in ("bary", "pos", "dir", "w"):
        assert np.abs(moved[k] - fresh[k]).max() <= 1e-6, k


def test_fp64_rejected_where_unsupported():
    wl = meshgen.workload(0, scale=0.05)
    X, F = wl.single
    mesh = sg().Mesh(parity.as_f32(X), F)
    q = wl.queries
    f32 = parity.as_f32
    with pytest.raises(sg().SgError):
        sg().exp_map(mesh, q.face, f32(q.bary), f32(q.v), kernel=1, precision=64)
    with pytest.raises(sg().SgError):
        sg().exp_map_trace(mesh, q.face, f32(q.bary), f32(q.v), precision=64)
    out = sg().exp_map(mesh, q.face, f32(q.bary), f32(q.v))
    with pytest.raises(sg().SgError):
        sg().exp_map_backward(mesh, "ep", q.face, f32(q.bary), f32(q.v), out["face"], out["bary"], out["dir"],
                              out["status"], f32(q.g_pos), opts=sg().default_opts(precision=64))
