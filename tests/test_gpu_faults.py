"""Bad inputs made on the host come back as error codes or per-query INVALID status, on every
walk variant, and never stop a batch: NaN and infinite barycentrics, vectors and lengths, faces
and mesh ids out of range, NaN or collapsed vertices at mesh creation, and a non-manifold face
list.  Every loop on the device is bounded (MAX_STEPS, the fan guard), so none of these can hang.
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


def _bad_batch():
    rng = np.random.default_rng(101)
    X, F = meshgen.icosphere(3, 0.003, rng)
    q = meshgen.sample_queries(X, F, 256, rng, 0.1, 1.5, 1)
    q.bary[0] = [np.nan, 0.5, 0.5]
    q.bary[1] = [np.inf, 0.0, 0.0]
    q.v[2] = [np.nan, 0.0, 0.0]
    q.v[3] = [np.inf, 1.0, 0.0]
    q.face[4] = -1
    q.face[5] = len(F)
    q.bary[6] = [-0.5, 0.75, 0.75]
    return X, F, q, np.arange(7)


VARIANTS = [dict(), dict(kernel=1), dict(sort=0), dict(sort=2), dict(boundary_mode=1), dict(precision=64),
            dict(precision=48), dict(precision=40), dict(precision=32)]


@pytest.mark.parametrize("kw", VARIANTS, ids=["persistent", "plain", "unsorted", "length-order", "hole", "fp64", "double-float",
                                             "mixed", "fp32"])
def test_bad_queries_are_invalid_and_the_rest_walk(kw):
    X, F, q, bad = _bad_batch()
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, q, 1, **kw)
    assert np.all(gpu["status"][bad] & oracle.INVALID)
    good = np.setdiff1d(np.arange(len(q)), bad)
    assert not np.any(gpu["status"][good] & oracle.INVALID)
    assert np.isfinite(gpu["pos"][good]).all()
    ref, _ = parity.run_oracle(X32, F, q.take(good), 1)
    sub = {k: v[good] for k, v in gpu.items()}
    parity.compare(sub, ref, meshgen.bbox_diag(X), 1, what=str(kw))


def test_bad_lengths_and_mesh_ids():
    import torch
    rng = np.random.default_rng(102)
    meshes = [meshgen.icosphere(2, 0.0, rng), meshgen.icosphere(3, 0.0, rng)]
    mesh = sg().Mesh([(parity.as_f32(X), F) for X, F in meshes])
    q = meshgen.sample_queries(*meshes[0], 64, rng, 0.1, 1.0, 0)
    mid = np.zeros(64, np.int32)
    mid[0], mid[1] = -1, 2
    L = np.full(64, 0.5, np.float32)
    L[2], L[3] = -1.0, np.nan
    for sort in (0, 1, 2):   # invalid mesh ids and lengths take the last bucket of the length order
        out = sg().exp_map(mesh, q.face, parity.as_f32(q.bary), parity.as_f32(q.v), length=L, mesh_id=mid,
                           sort=sort)
        st = out["status"].cpu().numpy()
        assert np.all(st[:4] & oracle.INVALID)
        assert not np.any(st[4:] & oracle.INVALID)


def test_backward_of_invalid_queries_is_zero():
    import torch
    X, F, q, bad = _bad_batch()
    mesh = sg().Mesh(parity.as_f32(X), F)
    f32 = parity.as_f32
    out = sg().exp_map(mesh, q.face, f32(q.bary), f32(q.v))
    for est in ("ep", "gfd"):
        r = sg().exp_map_backward(mesh, est, q.face, f32(q.bary), f32(q.v), out["face"], out["bary"], out["dir"],
                                  out["status"], f32(q.g_pos), want_grad_V=True)
        torch.cuda.synchronize()
        gv = r["grad_v"].cpu().numpy()
        assert np.all(gv[bad] == 0.0)
        assert np.isfinite(gv).all() and torch.isfinite(r["grad_V"]).all()


def test_bad_meshes_are_rejected_at_creation():
    X, F = meshgen.icosphere(2)
    X32 = parity.as_f32(X)
    Xn = X32.copy()
    Xn[3, 1] = np.nan
    with pytest.raises(sg().SgError, match="degenerate"):
        sg().Mesh(Xn, F)
    Xc = X32.copy()
    Xc[F[0, 0]] = Xc[F[0, 1]]             # a face with zero area
    with pytest.raises(sg().SgError, match="degenerate"):
        sg().Mesh(Xc, F)
    Fb = F.copy()
    Fb[0, 0] = len(X)                      # index out of range
    with pytest.raises(sg().SgError):
        sg().Mesh(X32, Fb)
    Fn = np.concatenate([F, F[:1, [0, 2, 1]], F[:1]])   # an edge with three faces
    with pytest.raises(sg().SgError):
        sg().Mesh(X32, Fn)


def test_snap_radius_beyond_the_near_band_is_rejected():
    # the hot step tests the snap radius only inside the near band, so a snap radius larger than
    # tau_near is an invalid option on every entry point that walks
    X, F, q, _ = _bad_batch()
    mesh = sg().Mesh(parity.as_f32(X), F)
    f32 = parity.as_f32
    with pytest.raises(sg().SgError, match="status 1"):
        sg().exp_map(mesh, q.face, f32(q.bary), f32(q.v), tau_near=1e-4, tau_snap=1e-3)
    out = sg().exp_map(mesh, q.face, f32(q.bary), f32(q.v), tau_near=1e-4, tau_snap=1e-4)  # equal: allowed
    with pytest.raises(sg().SgError, match="status 1"):
        sg().exp_map_backward(mesh, "gfd", q.face, f32(q.bary), f32(q.v), out["face"], out["bary"], out["dir"],
                              out["status"], f32(q.g_pos), opts=sg().default_opts(tau_near=1e-5, tau_snap=1e-4))
