"""The order in which the persistent kernels take queries (sg_opts.sort: input order, by start
face, or by walk length, longest first) changes nothing but speed: every query's walk is the
same arithmetic in any order, so the forward outputs and the backward's per-query gradients are
bit-identical across orders, and the vertex gradient (atomic sums in a different order) agrees
to float rounding.  The batch is above the size where the automatic choice orders queries."""
import numpy as np
import pytest

import meshgen
from tests import parity

pytestmark = pytest.mark.gpu


def _batch(n, rng):
    a = meshgen.icosphere(4, 0.003, rng)
    b = meshgen.torus(64, 32, 1.0, 0.4, 0.002, rng)
    qa = meshgen.sample_queries(*a, n // 2, rng, 0.0, 1.5, 1)
    qb = meshgen.sample_queries(*b, n - n // 2, rng, 0.0, 1.5, 1)
    q = meshgen.Queries(np.concatenate([qa.face, qb.face]), np.concatenate([qa.bary, qb.bary]),
                        np.concatenate([qa.v, qb.v]), np.concatenate([qa.w, qb.w]),
                        np.concatenate([qa.g_pos, qb.g_pos]))
    mid = np.repeat(np.arange(2, dtype=np.int32), [n // 2, n - n // 2])
    perm = rng.permutation(n)
    q = meshgen.Queries(q.face[perm], q.bary[perm], q.v[perm], q.w[perm], q.g_pos[perm])
    return [a, b], q, mid[perm]


def test_forward_and_backward_are_independent_of_the_query_order():
    import torch
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(141)
    n = 100_000
    meshes, q, mid = _batch(n, rng)
    mesh = sg.Mesh([(parity.as_f32(X), F) for X, F in meshes])
    f32 = parity.as_f32
    dev = "cuda"
    face = torch.tensor(q.face, device=dev)
    bary = torch.tensor(f32(q.bary), device=dev)
    v = torch.tensor(f32(q.v), device=dev)
    w = torch.tensor(f32(q.w[:, :1]), device=dev)
    g = torch.tensor(f32(q.g_pos), device=dev)
    m = torch.tensor(mid, device=dev)
    length = torch.tensor(f32(np.linalg.norm(q.v, axis=1) * rng.uniform(0.5, 1.5, n)), device=dev)
    length[:50] = 0.0
    res = {}
    for sort in (0, 1, 2, -1):
        o = sg.default_opts(sort=sort)
        fw = sg.exp_map(mesh, face, bary, v, w, mesh_id=m, want_hash=True, opts=o)
        fl = sg.exp_map(mesh, face, bary, v, w, length=length, mesh_id=m, want_hash=True, opts=o)
        bw = sg.exp_map_backward(mesh, "gfd", face, bary, v, fw["face"], fw["bary"], fw["dir"], fw["status"], g,
                                 mesh_id=m, want_grad_V=True, opts=o)
        torch.cuda.synchronize()
        res[sort] = (fw, fl, bw)
    base = res[0]
    for sort in (1, 2, -1):
        for a, b in zip(base[:2], res[sort][:2]):
            for k in ("face", "bary", "pos", "dir", "w", "status", "ncross", "hash"):
                assert torch.equal(a[k], b[k]), f"sort {sort}: forward {k} differs"
        for k in ("grad_v", "grad_p", "grad_bary", "status"):
            assert torch.equal(base[2][k], res[sort][2][k]), f"sort {sort}: backward {k} differs"
        gV0, gV1 = base[2]["grad_V"], res[sort][2]["grad_V"]
        assert float((gV0 - gV1).abs().max()) <= 1e-5 * float(gV0.abs().max())


def test_backward_reuses_the_forward_order():
    """sg_opts.order: the forward writes the walk-length order of the queries (longest first) into
    the buffer, whatever order its own kernel took them in, and the backward's re-walk takes the
    queries in that order instead of sorting them again.  Same gradients as the backward's own
    order."""
    import torch
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(142)
    n = 100_000
    meshes, q, mid = _batch(n, rng)
    mesh = sg.Mesh([(parity.as_f32(X), F) for X, F in meshes])
    f32 = parity.as_f32
    dev = "cuda"
    face = torch.tensor(q.face, device=dev)
    bary = torch.tensor(f32(q.bary), device=dev)
    v = torch.tensor(f32(q.v), device=dev)
    g = torch.tensor(f32(q.g_pos), device=dev)
    midt = torch.tensor(mid, device=dev)
    # the length key: an eighth of an octave of |v| / l_ref per bucket (the meshes' mean edge lengths)
    lref = np.array([np.linalg.norm(X[F[:, [1, 2, 0]]] - X[F], axis=2).mean() for X, F in meshes])
    L = np.linalg.norm(f32(q.v).astype(np.float64), axis=1)
    key = np.floor(8 * np.log2(L / lref[mid]))
    ref = None
    for kw in (dict(), dict(sort=0), dict(sort=1), dict(kernel=1, sort=0, precision=32)):
        order = torch.full((n,), -7, dtype=torch.int32, device=dev)
        out = sg.exp_map(mesh, face, bary, v, mesh_id=midt, order=order, **kw)
        o = order.cpu().numpy()
        assert np.array_equal(np.sort(o), np.arange(n)), kw             # a permutation of the queries
        # longest first: bucket keys non-increasing along the order (one bucket of slack for the
        # float32 rounding of the key on the device)
        assert np.all(np.diff(key[o]) <= 1.0), kw
        assert key[o[: n // 10]].mean() > key[o[-n // 10:]].mean() + 8, kw
        if kw.get("kernel") == 1:
            continue  # the plain kernel: another launch shape, results compared elsewhere
        if ref is None:
            ref = out
        else:  # the persistent kernel gives the same results in every query order
            assert torch.equal(out["face"], ref["face"]) and torch.equal(out["pos"], ref["pos"]), kw
    order = torch.empty(n, dtype=torch.int32, device=dev)
    out = sg.exp_map(mesh, face, bary, v, mesh_id=midt, order=order)
    for est in ("gfd", "ep"):
        args = (mesh, est, face, bary, v, out["face"], out["bary"], out["dir"], out["status"], g)
        a = sg.exp_map_backward(*args, mesh_id=midt, want_grad_V=True)
        b = sg.exp_map_backward(*args, mesh_id=midt, want_grad_V=True, order=order)
        torch.cuda.synchronize()
        for k in ("grad_v", "grad_p", "grad_bary", "status"):
            assert torch.equal(a[k], b[k]), (est, k)
        gva, gvb = a["grad_V"].cpu().numpy(), b["grad_V"].cpu().numpy()
        scale = np.abs(gva).max()
        assert np.abs(gva - gvb).max() <= 1e-5 * scale, (est, np.abs(gva - gvb).max(), scale)
