"""GPU parity of the full-precision walks against the FP64 oracle: the FP64 walk
(sg_opts.precision = 64) and the double-float walk (precision = 48: each crossing in pairs of
FP32 numbers, about 48 significant bits, the rare events in FP64).

On the sliver heightfield of workload 4 (~1.4k crossings per walk) the FP32 walk's accumulated
state error (~1e-6 of l_ref) exceeds the near-vertex band, so FP32 and FP64 pass some vertices
on different sides.  The FP64 walk keeps its error near 1e-13 and the double-float walk near
1e-12, so with a near-vertex band of 1e-8 l_ref on both sides their face sequences must equal
the oracle's on every unflagged query.
"""
import numpy as np
import pytest

import meshgen
from tests import parity

pytestmark = pytest.mark.gpu


def sg():
    import paper_2603_15780_gb300 as m
    return m


PRECISIONS = pytest.mark.parametrize("prec", [64, 48], ids=["fp64", "double-float"])
# with the mixed walk (FP32 positions and orientation tests, double-float direction)
ALL_WIDE = pytest.mark.parametrize("prec", [64, 48, 40], ids=["fp64", "double-float", "mixed"])


@PRECISIONS
def test_fp64_walk_on_the_sliver_heightfield(prec):
    wl = meshgen.workload(4, scale=20000 / 16777216)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    q = wl.queries
    tau = 1e-8
    g64 = parity.run_gpu(mesh, q, 0, precision=prec, tau_near=tau)
    g32 = parity.run_gpu(mesh, q, 0, tau_near=tau, precision=32)
    ref, _ = parity.run_oracle(X32, F, q, 0, tau_near=tau)
    diag = meshgen.bbox_diag(X)
    flag64 = ((g64["status"] | ref["status"]) & parity.FLAGS) != 0
    flag32 = ((g32["status"] | ref["status"]) & parity.FLAGS) != 0
    assert flag64.mean() < 0.01
    same64 = (g64["hash"] == ref["hash"]) & (g64["face"] == ref["face"]) & (g64["ncross"] == ref["ncross"])
    same32 = (g32["hash"] == ref["hash"]) & (g32["face"] == ref["face"])
    err = np.linalg.norm(g64["pos"] - ref["pos"], axis=1)[~flag64] / diag
    print(f"precision {prec} same", same64[~flag64].mean(), "fp32 same", same32[~flag32].mean(),
          "mean ncross", ref["ncross"].mean(), "max pos err / diag", err.max(), "flagged", flag64.mean())
    assert same64[~flag64].all()
    assert np.array_equal(g64["status"][~flag64] & ~np.uint32(32), ref["status"][~flag64])
    assert err.max() <= 1e-6, err.max()
    # the FP32 walk diverges on many of these walks; the FP64 walk on none
    assert (~same32[~flag32]).sum() > 100


@ALL_WIDE
def test_fp64_walk_workload0_parity_with_carried_vectors(prec):
    wl = meshgen.workload(0)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    g = parity.run_gpu(mesh, wl.queries, 1, precision=prec)
    ref, _ = parity.run_oracle(X32, F, wl.queries, 1)
    parity.compare(g, ref, meshgen.bbox_diag(X), 1, what=f"precision {prec} workload 0", pos_tol=1e-6, dir_tol=1e-5)


def test_double_float_walk_matches_the_fp64_walk():
    """The double-float walk and the FP64 walk take the same decisions wherever neither passes
    within the near band of a vertex: equal faces, face sequences and statuses, end points equal
    to float32 rounding.  Torus of workload 1 (2 carried vectors) and a flat grid (Exp = p + v)."""
    rng = np.random.default_rng(17)
    wl = meshgen.workload(1, scale=50000 / 4194304)
    cases = [(wl.single, wl.queries, 2)]
    Xf, Ff = meshgen.flat_grid(33, rng, jitter=0.3)
    cases.append(((Xf, Ff), meshgen.sample_queries(Xf, Ff, 20000, rng, 0.0, 0.4, 1), 1))
    for (X, F), q, nw in cases:
        mesh = sg().Mesh(parity.as_f32(X), F)
        tau = 1e-7
        a = parity.run_gpu(mesh, q, nw, precision=48, tau_near=tau)
        b = parity.run_gpu(mesh, q, nw, precision=64, tau_near=tau)
        flag = ((a["status"] | b["status"]) & parity.FLAGS) != 0
        assert flag.mean() < 0.01
        for k in ("face", "hash", "ncross", "status"):
            assert np.array_equal(a[k][~flag], b[k][~flag]), k
        diag = meshgen.bbox_diag(X)
        assert np.abs(a["pos"] - b["pos"])[~flag].max() <= 1e-6 * diag
        for k in ("dir", "w"):
            assert np.abs(a[k] - b[k])[~flag].max() <= 1e-6, k


def test_double_float_walk_on_a_multi_mesh_batch():
    """Mesh-tagged queries over a CSR batch of a sphere, a torus and a heightfield: the
    double-float walk against the oracle mesh by mesh."""
    rng = np.random.default_rng(23)
    meshes = [meshgen.icosphere(3, 0.003, rng), meshgen.torus(48, 24, 1.0, 0.4, 0.002, rng),
              meshgen.heightfield(24, rng)[:2]]
    qs = [meshgen.sample_queries(X, F, 1500, rng, 0.0, 1.0, 1) for X, F in meshes]
    mesh = sg().Mesh([(parity.as_f32(X), F) for X, F in meshes])
    q = meshgen.Queries(*(np.concatenate([getattr(x, n) for x in qs]) for n in ("face", "bary", "v", "w", "g_pos")))
    mid = np.repeat(np.arange(3, dtype=np.int32), 1500)
    g = parity.run_gpu(mesh, q, 1, mesh_id=mid, precision=48)
    for m, (X, F) in enumerate(meshes):
        sl = slice(1500 * m, 1500 * (m + 1))
        ref, _ = parity.run_oracle(parity.as_f32(X), F, q.take(np.arange(1500 * m, 1500 * (m + 1))), 1)
        parity.compare({k: v[sl] for k, v in g.items()}, ref, meshgen.bbox_diag(X), 1,
                       what=f"double-float mesh {m}", pos_tol=1e-6, dir_tol=1e-5)


@ALL_WIDE
def test_fp64_geometry_follows_vertex_updates(prec):
    rng = np.random.default_rng(91)
    XA, F = meshgen.icosphere(4, 0.004, rng)
    XB, _ = meshgen.icosphere(4, 0.004, rng)
    q = meshgen.sample_queries(XB, F, 5000, rng, 0.0, 2.0, 1)
    mesh = sg().Mesh(parity.as_f32(XA), F)
    parity.run_gpu(mesh, q, 1, precision=prec)          # builds the geometry of A
    mesh.update_vertices(parity.as_f32(XB))
    moved = parity.run_gpu(mesh, q, 1, precision=prec)
    fresh = parity.run_gpu(sg().Mesh(parity.as_f32(XB), F), q, 1, precision=prec)
    for k in ("face", "status", "hash", "ncross"):
        assert np.array_equal(moved[k], fresh[k]), k
    for k in ("bary", "pos", "dir", "w"):
        assert np.abs(moved[k] - fresh[k]).max() <= 1e-6, k


@ALL_WIDE
def test_fp64_rejected_where_unsupported(prec):
    wl = meshgen.workload(0, scale=0.05)
    X, F = wl.single
    mesh = sg().Mesh(parity.as_f32(X), F)
    q = wl.queries
    f32 = parity.as_f32
    with pytest.raises(sg().SgError):
        sg().exp_map(mesh, q.face, f32(q.bary), f32(q.v), kernel=1, precision=prec)
    with pytest.raises(sg().SgError):
        sg().exp_map_trace(mesh, q.face, f32(q.bary), f32(q.v), precision=prec)
    out = sg().exp_map(mesh, q.face, f32(q.bary), f32(q.v))
    with pytest.raises(sg().SgError):
        sg().exp_map_backward(mesh, "ep", q.face, f32(q.bary), f32(q.v), out["face"], out["bary"], out["dir"],
                              out["status"], f32(q.g_pos), opts=sg().default_opts(precision=prec))
