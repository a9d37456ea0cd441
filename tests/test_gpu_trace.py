"""GPU parity of geodesic tracing (sg_exp_map_trace) against the FP64 oracle's traced paths.

Straightest geodesics trace the geodesic as a by-product of the exponential map (Sec. 1,
Sec. 4): the ordered faces the walk enters and the point where it enters each, followed by the
end point, form the geodesic's polyline.  Bars (tests/parity.py): face sequences bit-exact on
queries neither side flags, points within 1e-5 of the bbox diagonal.
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


def run_trace(mesh, q, cap, mesh_id=None, **kw):
    import torch
    f32 = parity.as_f32
    out = sg().exp_map_trace(mesh, q.face, f32(q.bary), f32(q.v), mesh_id=mesh_id, path_cap=cap, want_hash=True, **kw)
    torch.cuda.synchronize()
    r = {k: v.cpu().numpy() for k, v in out.items()}
    r["status"] = r["status"].astype(np.uint32)
    r["hash"] = r["hash"].view(np.uint64)
    return r


def check_against_oracle(tr, ref, diag, cap, what, min_ok=0.95, pt_tol=1e-5, pt_quantile=1.0, pt_max=1e-5):
    """Face sequences bit-exact on unflagged queries; entry points within pt_tol * diag at the
    given quantile of all points and within pt_max * diag everywhere."""
    ok = ((tr["status"] | ref["status"]) & parity.FLAGS) == 0
    assert ok.mean() > min_ok, what
    assert np.array_equal(tr["path_len"][ok], ref["path_len"][ok]), what
    errs = []
    for i in np.nonzero(ok)[0]:
        n = min(int(tr["path_len"][i]), cap)
        assert np.array_equal(tr["path_face"][i, :n], ref["path"][i, :n]), (what, i)
        if n:
            errs.append(np.abs(tr["path_pt"][i, :n] - ref["path_pt"][i, :n]).max(1))
    errs = np.concatenate(errs) / diag
    assert np.quantile(errs, pt_quantile) <= pt_tol, (what, np.quantile(errs, pt_quantile))
    assert errs.max() <= pt_max, (what, errs.max())
    return len(errs)


def test_trace_matches_oracle_paths_and_exp_map():
    rng = np.random.default_rng(51)
    X, F = meshgen.icosphere(4, 0.004, rng)
    X32 = parity.as_f32(X)
    q = meshgen.sample_queries(X, F, 3000, rng, 0.0, 2.0, 0)
    q.v[:20] = 0.0   # zero-length queries enter no face
    mesh = sg().Mesh(X32, F)
    cap = 160
    for kw in (dict(), dict(sort=0), dict(kernel=1)):
        tr = run_trace(mesh, q, cap, **kw)
        ref, _ = parity.run_oracle(X32, F, q, 0, path_cap=cap)
        assert np.all(tr["path_len"][:20] == 0)
        n_pt = check_against_oracle(tr, ref, meshgen.bbox_diag(X), cap, str(kw))
        assert n_pt > 3000 * 10
        # the end outputs are those of sg_exp_map, and the hash hashes the traced faces
        ex = parity.run_gpu(mesh, q, 0, **kw)
        for k in ("face", "status", "hash", "ncross"):
            assert np.array_equal(tr[k], ex[k]), k
        for k in ("bary", "pos", "dir"):
            assert np.abs(tr[k] - ex[k]).max() <= 1e-6, k
        short = np.nonzero(tr["path_len"] <= cap)[0]
        for i in short[:400]:
            n = tr["path_len"][i]
            if n:
                assert oracle.fnv_hash(tr["path_face"][i, :n]) == tr["hash"][i]


def test_traced_polyline_length_and_truncation():
    rng = np.random.default_rng(52)
    X, F = meshgen.torus(128, 64, noise=0.002, rng=rng)
    q = meshgen.sample_queries(X, F, 4000, rng, 0.1, 2.0, 0)
    mesh = sg().Mesh(parity.as_f32(X), F)
    full = run_trace(mesh, q, 400)
    L = np.linalg.norm(parity.as_f32(q.v).astype(np.float64), axis=1)
    m = (full["path_len"] <= 400) & ((full["status"] & (oracle.BOUNDARY | oracle.INVALID)) == 0)
    assert m.mean() > 0.99
    for i in np.nonzero(m)[0][:500]:
        n = full["path_len"][i]
        poly = np.concatenate([full["path_pt"][i, :n], full["pos"][i][None]]).astype(np.float64)
        length = np.linalg.norm(np.diff(poly, axis=0), axis=1).sum()
        assert abs(length - L[i]) <= 2e-5 * max(L[i], 1.0), (i, length, L[i])
    # a small cap keeps the first entries and still reports the full count (entries past the
    # path length are not written, so only the written prefix is compared)
    small = run_trace(mesh, q, 4)
    assert np.array_equal(small["path_len"], full["path_len"])
    for i in range(len(q.face)):
        n = min(int(full["path_len"][i]), 4)
        assert np.array_equal(small["path_face"][i, :n], full["path_face"][i, :n])
        assert np.array_equal(small["path_pt"][i, :n], full["path_pt"][i, :n])
    # a cap that is not a multiple of 4 takes the one-entry-at-a-time store path
    odd = run_trace(mesh, q, 13)
    assert np.array_equal(odd["path_len"], full["path_len"])
    for i in range(len(q.face)):
        n = min(int(full["path_len"][i]), 13)
        assert np.array_equal(odd["path_face"][i, :n], full["path_face"][i, :n])
        assert np.array_equal(odd["path_pt"][i, :n], full["path_pt"][i, :n])
    # cap 0: no path storage at all, counts only
    none = run_trace(mesh, q, 0)
    assert np.array_equal(none["path_len"], full["path_len"])


def test_trace_vertex_hits_and_boundary():
    """Cone apex hits (the entry point is the apex itself) and a heightfield with boundary
    stops, against the oracle run with the GPU's snap radius."""
    n = 9
    X, F = meshgen.cone_fan(n, 1.5 * np.pi)
    rng = np.random.default_rng(53)
    X32 = parity.as_f32(X)
    apex = X32[0].astype(np.float64)
    # rays aimed at the apex (vertex 0, the origin) from random points of the fan's faces
    face, bary, v = [], [], []
    for _ in range(400):
        f0 = int(rng.integers(n))
        u = X32[F[f0][1]].astype(np.float64); w = X32[F[f0][2]].astype(np.float64)
        b1, b2 = rng.uniform(0.05, 0.5), rng.uniform(0.05, 0.4)
        p = b1 * u + b2 * w
        rho = np.linalg.norm(p)
        face.append(f0); bary.append([1 - b1 - b2, b1, b2]); v.append(-p / rho * (rho + rng.uniform(0.05, 0.3)))
    q = meshgen.Queries(np.array(face, np.int32), np.array(bary), np.array(v), np.zeros((400, 0, 3)),
                        np.zeros((400, 3)))
    mesh = sg().Mesh(X32, F)
    tr = run_trace(mesh, q, 16)
    ref, _ = parity.run_oracle(X32, F, q, 0, path_cap=16, tau_snap=1e-6)
    hit = (tr["status"] & oracle.VERTEX_HIT) != 0
    assert hit.mean() > 0.9
    check_against_oracle(tr, ref, meshgen.bbox_diag(X), 16, "cone", min_ok=0.6)
    apex_row = np.zeros(400, bool)
    for i in np.nonzero(hit)[0]:
        n = min(tr["path_len"][i], 16)
        apex_row[i] = np.any(np.abs(tr["path_pt"][i, 1:n] - apex).max(axis=1) <= 1e-5)
    assert apex_row[hit].mean() > 0.9
    Xh, Fh, _ = meshgen.heightfield(48, rng)
    qh = meshgen.sample_queries(Xh, Fh, 3000, rng, 0.0, 1.2, 0)
    mh = sg().Mesh(parity.as_f32(Xh), Fh)
    trh = run_trace(mh, qh, 256)
    refh, _ = parity.run_oracle(parity.as_f32(Xh), Fh, qh, 0, path_cap=256)
    assert ((trh["status"] & oracle.BOUNDARY) != 0).mean() > 0.1
    # long grazing walks over the waves amplify the FP32 direction error (as for the end points
    # of the heightfield workload): 99.5% of the entry points within the bar, all within 1e-4
    check_against_oracle(trh, refh, meshgen.bbox_diag(Xh), 256, "heightfield", pt_quantile=0.995, pt_max=1e-4)


def test_trace_multi_mesh_local_ids():
    rng = np.random.default_rng(54)
    meshes = [meshgen.icosphere(3, 0.003, rng), meshgen.torus(48, 24, noise=0.002, rng=rng)]
    qs = [meshgen.sample_queries(X, F, 1500, rng, 0.0, 1.5, 0) for X, F in meshes]
    mesh = sg().Mesh([(parity.as_f32(X), F) for X, F in meshes])
    q = meshgen.Queries(np.concatenate([a.face for a in qs]), np.concatenate([a.bary for a in qs]),
                        np.concatenate([a.v for a in qs]), np.zeros((3000, 0, 3)), np.zeros((3000, 3)))
    mid = np.repeat(np.arange(2, dtype=np.int32), 1500)
    tr = run_trace(mesh, q, 128, mesh_id=mid)
    for k, (X, F) in enumerate(meshes):
        sl = slice(1500 * k, 1500 * (k + 1))
        sub = {key: val[sl] for key, val in tr.items()}
        ref, _ = parity.run_oracle(parity.as_f32(X), F, qs[k], 0, path_cap=128)
        check_against_oracle(sub, ref, meshgen.bbox_diag(X), 128, f"mesh {k}")
