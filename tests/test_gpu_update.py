"""GPU tests of sg_mesh_update_vertices: moving the vertices of an existing mesh re-derives its
geometry on the device so that it walks like a mesh created from the new positions.

Sec. 4: the records hold functions of the vertex positions (face shapes, frames, theta) and of
F (adjacency); the update rewrites the former only.  Checks: equality with a freshly created
mesh (single and batched, closed and with boundary), parity with the FP64 oracle on the moved
mesh, rejection of a degenerate move and recovery, and a descent step along grad_V.
"""
import numpy as np
import pytest

import meshgen
import oracle
from tests import parity

pytestmark = pytest.mark.gpu

OUT_KEYS = ("face", "bary", "pos", "dir", "w", "status", "hash", "ncross")


def sg():
    import paper_2603_15780_gb300 as m
    return m


def _same_outputs(a, b, min_exact=0.999):
    """Updated vs fresh mesh on identical queries.  The walk reads identical records except where
    a theta or l_ref sum rounded differently (FP64 atomics in another order), so integer outputs
    must match everywhere and float outputs bit for bit on almost all queries."""
    for k in ("face", "status", "hash", "ncross"):
        assert np.array_equal(a[k], b[k]), k
    for k in ("bary", "pos", "dir", "w"):
        if k not in a:
            continue
        eq = np.all(a[k].reshape(len(a["face"]), -1) == b[k].reshape(len(b["face"]), -1), axis=1)
        assert eq.mean() >= min_exact, (k, eq.mean())
        assert np.abs(a[k] - b[k]).max() <= 1e-6, k


def test_update_matches_fresh_mesh_and_oracle():
    rng = np.random.default_rng(41)
    XA, F = meshgen.icosphere(4, 0.004, rng)
    XB, _ = meshgen.icosphere(4, 0.004, rng)   # same faces, other radial noise
    XA32, XB32 = parity.as_f32(XA), parity.as_f32(XB)
    q = meshgen.sample_queries(XB, F, 20000, rng, 0.0, 2.0, 1)
    mesh = sg().Mesh(XA32, F)
    before = parity.run_gpu(mesh, q, 1)
    mesh.update_vertices(XB32)
    moved = parity.run_gpu(mesh, q, 1)
    fresh_mesh = sg().Mesh(XB32, F)
    fresh = parity.run_gpu(fresh_mesh, q, 1)
    _same_outputs(moved, fresh)
    assert not np.array_equal(before["pos"], moved["pos"])   # the geometry did change
    info, finfo = mesh.info(), fresh_mesh.info()
    assert info.n_degenerate == 0
    assert abs(info.l_ref_mean - finfo.l_ref_mean) <= 1e-12 * finfo.l_ref_mean
    ref, om = parity.run_oracle(XB32, F, q, 1)
    parity.compare(moved, ref, meshgen.bbox_diag(XB), 1, what="updated icosphere")
    # a second update back to A restores the first results
    mesh.update_vertices(XA32)
    _same_outputs(parity.run_gpu(mesh, q, 1), before)


def test_update_batched_with_boundary():
    """Batched meshes, one with a boundary (boundary flags are topological and must survive)."""
    rng = np.random.default_rng(42)
    X0, F0 = meshgen.icosphere(3, 0.003, rng)
    X1, F1, _ = meshgen.heightfield(40, rng)
    X0b, _ = meshgen.icosphere(3, 0.003, rng)
    X1b = X1.copy()
    X1b[:, 2] *= 1.7
    X1b[:, :2] += rng.normal(scale=0.002, size=(len(X1), 2))
    mk = lambda a, b: sg().Mesh([(parity.as_f32(a), F0), (parity.as_f32(b), F1)])
    mesh = mk(X0, X1)
    Vb = np.concatenate([parity.as_f32(X0b), parity.as_f32(X1b)])
    mesh.update_vertices(Vb)
    fresh = mk(X0b, X1b)
    qa = meshgen.sample_queries(X0b, F0, 4000, rng, 0.0, 1.5, 2)
    qb = meshgen.sample_queries(X1b, F1, 4000, rng, 0.0, 1.0, 2)
    q = meshgen.Queries(np.concatenate([qa.face, qb.face]), np.concatenate([qa.bary, qb.bary]),
                        np.concatenate([qa.v, qb.v]), np.concatenate([qa.w, qb.w]),
                        np.concatenate([qa.g_pos, qb.g_pos]))
    mid = np.repeat(np.arange(2, dtype=np.int32), 4000)
    a = parity.run_gpu(mesh, q, 2, mesh_id=mid)
    b = parity.run_gpu(fresh, q, 2, mesh_id=mid)
    _same_outputs(a, b)
    assert ((a["status"][4000:] & oracle.BOUNDARY) != 0).mean() > 0.05


def test_degenerate_move_rejects_queries_then_recovers():
    rng = np.random.default_rng(43)
    X, F = meshgen.icosphere(3, 0.003, rng)
    X32 = parity.as_f32(X)
    mesh = sg().Mesh([(X32, F), (X32, F)])
    q = meshgen.sample_queries(X, F, 3000, rng, 0.0, 1.0, 0)
    q2 = meshgen.Queries(np.concatenate([q.face, q.face]), np.concatenate([q.bary, q.bary]),
                         np.concatenate([q.v, q.v]), None, np.concatenate([q.g_pos, q.g_pos]))
    mid = np.repeat(np.arange(2, dtype=np.int32), 3000)
    base = parity.run_gpu(mesh, q2, 0, mesh_id=mid)
    for bad_value in ("collapse", "nan"):
        V = np.concatenate([X32, X32])
        a, b = F[0, 0], F[0, 1]
        if bad_value == "collapse":
            V[len(X32) + a] = V[len(X32) + b]        # face 0 of mesh 1 loses its area
        else:
            V[len(X32) + a, 1] = np.nan
        mesh.update_vertices(V)
        assert mesh.info().n_degenerate >= 1
        r = parity.run_gpu(mesh, q2, 0, mesh_id=mid)
        assert np.all((r["status"][3000:] & oracle.INVALID) != 0)
        for k in ("face", "pos", "status", "hash"):
            assert np.array_equal(r[k][:3000], base[k][:3000]), k     # mesh 0 untouched
        mesh.update_vertices(np.concatenate([X32, X32]))
        assert mesh.info().n_degenerate == 0
        _same_outputs(parity.run_gpu(mesh, q2, 0, mesh_id=mid), base)


def test_descent_step_along_grad_V():
    """One optimisation step X <- X - eta * grad_V on the device (update_vertices) lowers
    sum_q g_q . Exp_q(X) by eta |grad_V|^2 to first order, on queries whose face sequence is
    unchanged by the step."""
    import torch
    S = sg()
    rng = np.random.default_rng(44)
    X, F = meshgen.icosphere(4, 0.01, rng)
    X32 = parity.as_f32(X)
    q = meshgen.sample_queries(X, F, 4000, rng, 0.1, 1.0, 0)
    f32 = parity.as_f32
    mesh = S.Mesh(X32, F)
    out = S.exp_map(mesh, q.face, f32(q.bary), f32(q.v), want_hash=True)
    g = torch.tensor(f32(q.g_pos), device="cuda")
    r = S.exp_map_backward(mesh, "ep", q.face, f32(q.bary), f32(q.v), out["face"], out["bary"], out["dir"],
                           out["status"], g, want_grad_V=True)
    gV = r["grad_V"].double()
    eta = 1e-4 / float(gV.abs().max())
    Xd = torch.tensor(X32, device="cuda", dtype=torch.float64)
    Xn = (Xd - eta * gV).float()
    mesh.update_vertices(Xn)
    out2 = S.exp_map(mesh, q.face, f32(q.bary), f32(q.v), want_hash=True)
    keep = (out2["hash"] == out["hash"]) & ((out["status"] & (oracle.BOUNDARY | oracle.VERTEX_HIT)) == 0)
    assert keep.float().mean() > 0.9
    # redo the gradient on the kept queries only, so that both sides see the same loss
    gk = g * keep[:, None]
    mesh.update_vertices(torch.tensor(X32, device="cuda"))
    rk = S.exp_map_backward(mesh, "ep", q.face, f32(q.bary), f32(q.v), out["face"], out["bary"], out["dir"],
                            out["status"], gk, want_grad_V=True)
    gk_V = rk["grad_V"].double()
    dX = Xn.double() - Xd               # the step actually taken (after float rounding)
    pred = float((gk_V * dX).sum())
    actual = float(((out2["pos"].double() - out["pos"].double()) * gk.double()).sum())
    assert pred < 0
    assert abs(actual - pred) <= 0.05 * abs(pred), (actual, pred)


def test_mesh_from_device_arrays_equals_host_build():
    """sg_mesh_create with V and F in device memory (detected, copied to the host) builds the
    same records as from host arrays: identical walks."""
    import torch
    rng = np.random.default_rng(45)
    X, F = meshgen.icosphere(3, 0.004, rng)
    X32 = parity.as_f32(X)
    q = meshgen.sample_queries(X, F, 3000, rng, 0.0, 1.5, 1)
    host = parity.run_gpu(sg().Mesh(X32, F), q, 1)
    dev = parity.run_gpu(sg().Mesh(torch.tensor(X32, device="cuda"), torch.tensor(F, device="cuda")), q, 1)
    for k in OUT_KEYS:
        assert np.array_equal(host[k], dev[k]), k
