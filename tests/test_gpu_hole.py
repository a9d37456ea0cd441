"""GPU parity of hole avoidance (sg_opts.boundary_mode = 1) against the FP64 oracle.

Sec. 4: instead of stopping at the boundary, the walk traces along it and resumes with the last
straightest direction as soon as a face receives it.  The oracle's reading of the face choice is
pinned to closed forms on a square with a square hole (tests/test_oracle_pins.py); here the CUDA
walk is compared with the oracle query by query, with the bars of tests/parity.py.
"""
import numpy as np
import pytest

import meshgen
import oracle
from tests import parity
from tests.test_oracle_pins import _locate, _square_with_hole

pytestmark = pytest.mark.gpu


def sg():
    import paper_2603_15780_gb300 as m
    return m


def test_square_with_hole_closed_form_and_oracle():
    X, F = _square_with_hole()
    X32 = parity.as_f32(X)
    rng = np.random.default_rng(81)
    n = 4000
    a = rng.uniform(0.1, 1.0, n)
    d = np.stack([np.cos(a), np.sin(a), np.zeros(n)], 1)
    p = np.stack([np.full(n, 0.2), rng.uniform(0.42, 0.58, n), np.zeros(n)], 1)
    face, bary = _locate(X, F, p)
    q = meshgen.Queries(face, bary, 0.5 * d, np.zeros((n, 0, 3)), np.zeros((n, 3)))
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, q, 0, boundary_mode=1)
    ref, _ = parity.run_oracle(X32, F, q, 0, boundary_mode=1)
    parity.compare(gpu, ref, meshgen.bbox_diag(X), 0, what="square with hole")
    qy = p[:, 1] + 0.2 * np.tan(a)
    into = qy < 0.6
    ok = ((gpu["status"] | ref["status"]) & parity.FLAGS) == 0
    assert np.all(((gpu["status"] & oracle.HOLE) != 0)[ok] == into[ok])
    qq = np.stack([np.full(n, 0.4), qy, np.zeros(n)], 1)
    rem = 0.5 - np.linalg.norm(qq - p, axis=1) - (0.6 - qy)
    expect = np.where(into[:, None], np.array([0.4, 0.6, 0.0]) + rem[:, None] * d, p + 0.5 * d)
    assert np.abs(gpu["pos"] - expect)[ok].max() < 2e-6
    # the default mode still stops there
    stop = parity.run_gpu(mesh, q, 0)
    assert np.all(((stop["status"] & oracle.BOUNDARY) != 0)[ok] == into[ok])


@pytest.fixture(scope="module")
def holey_sphere():
    rng = np.random.default_rng(82)
    X, F = meshgen.icosphere(4, 0.003, rng)
    X, F = meshgen.remove_faces(X, F, 0.08, rng)
    X32 = parity.as_f32(X)
    q = meshgen.sample_queries(X, F, 6000, rng, 0.1, 3.0, 1)
    return X32, F, q, sg().Mesh(X32, F)


def test_sphere_with_holes_parity(holey_sphere):
    X32, F, q, mesh = holey_sphere
    gpu = parity.run_gpu(mesh, q, 1, boundary_mode=1)
    ref, _ = parity.run_oracle(X32, F, q, 1, boundary_mode=1)
    r = parity.compare(gpu, ref, meshgen.bbox_diag(X32), 1, what="sphere with holes", max_flagged=0.08)
    hole = (gpu["status"] & oracle.HOLE) != 0
    assert hole.mean() > 0.2
    assert not np.any(gpu["status"] & oracle.BOUNDARY)
    # walks that never touch the boundary equal the default mode's, bit for bit
    stop = parity.run_gpu(mesh, q, 1)
    same = (stop["status"] & oracle.BOUNDARY) == 0
    for k in ("face", "pos", "dir", "w", "hash", "ncross"):
        assert np.array_equal(stop[k][same], gpu[k][same]), k


def test_closed_mesh_is_unchanged_by_hole_mode():
    wl = meshgen.workload(0)
    X, F = wl.single
    mesh = sg().Mesh(parity.as_f32(X), F)
    a = parity.run_gpu(mesh, wl.queries, 1)
    b = parity.run_gpu(mesh, wl.queries, 1, boundary_mode=1)
    for k in ("face", "bary", "pos", "dir", "w", "status", "hash", "ncross"):
        assert np.array_equal(a[k], b[k]), k


def test_hole_mode_backward(holey_sphere):
    """EP (closed form in the start and end frames) and GFD under hole avoidance against the
    oracle's, and grad_V marks the queries that slid along the boundary as not differentiable.
    A walk that slid takes literal GFD walks, which difference two independent FP32 walks: such a
    column carries the FP32 end-point error (~1e-6 of the bbox over these walks) divided by eps,
    so GFD is compared at eps = 1e-3 with a bar of 5e-3 at the 98th percentile."""
    import torch
    X32, F, q, mesh = holey_sphere
    f32 = parity.as_f32
    n = 3000
    qs = q.take(np.arange(n))
    out = sg().exp_map(mesh, qs.face, f32(qs.bary), f32(qs.v), boundary_mode=1)
    om = oracle.Mesh(X32.astype(np.float64), F)
    b, v, g = (f32(x).astype(np.float64) for x in (qs.bary, qs.v, qs.g_pos))
    fst = out["status"].cpu().numpy().astype(np.uint32)
    for est in ("ep", "gfd"):
        r = sg().exp_map_backward(mesh, est, qs.face, f32(qs.bary), f32(qs.v), out["face"], out["bary"], out["dir"],
                                  out["status"], f32(qs.g_pos), want_grad_V=True, eps_v=1e-3, eps_p=1e-3,
                                  opts=sg().default_opts(boundary_mode=1))
        torch.cuda.synchronize()
        gv = r["grad_v"].cpu().numpy()
        if est == "ep":
            ref = oracle.ep_backward(om, qs.face, b, v, g, boundary_mode=1)
        else:
            ref = oracle.gfd_backward(om, qs.face, b, v, g, eps_v=1e-3, eps_p=1e-3, boundary_mode=1)
        ok = ((fst | ref["flags"]) & (parity.FLAGS | oracle.INVALID)) == 0
        if est == "gfd":
            # a GFD column is a finite difference: where a perturbation changes how the walk
            # meets the boundary it jumps on both sides, so compare where both are moderate
            ok &= (r["status"].cpu().numpy() & oracle.NEAR_VERTEX) == 0
        assert ok.mean() > 0.8
        err = np.linalg.norm(gv - ref["grad_v"], axis=1) / (np.linalg.norm(ref["grad_v"], axis=1) + 1e-3)
        bar = 1e-3 if est == "ep" else 5e-3
        assert np.quantile(err[ok], 0.98) < bar, (est, np.quantile(err[ok], 0.98))
        assert np.median(err[ok]) < 0.1 * bar, (est, np.median(err[ok]))
        st = r["status"].cpu().numpy()
        hole = (fst & oracle.HOLE) != 0
        assert np.all((st[hole] & 1024) != 0)   # SG_ST_NO_GRADV


def test_hole_mode_rejected_where_unsupported():
    wl = meshgen.workload(0, scale=0.05)
    X, F = wl.single
    mesh = sg().Mesh(parity.as_f32(X), F)
    q = wl.queries
    with pytest.raises(sg().SgError):
        sg().exp_map(mesh, q.face, parity.as_f32(q.bary), parity.as_f32(q.v), kernel=1, boundary_mode=1)
    with pytest.raises(sg().SgError):
        sg().exp_map_trace(mesh, q.face, parity.as_f32(q.bary), parity.as_f32(q.v), boundary_mode=1)
