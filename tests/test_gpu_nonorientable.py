"""GPU parity on non-orientable meshes (Moebius strip, Klein bottle): adjacency flip bits,
carried vectors through orientation reversals, and the EP gradient with the transported
frame (App. 'Main differences with SotA implementation')."""
import numpy as np
import pytest

import meshgen
import oracle
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["klein", "mobius"])
def test_non_orientable_parity(which):
    import torch
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(42)
    if which == "klein":
        X, F = meshgen.klein_bottle(96, 48)
        q = meshgen.sample_queries(X, F, 20000, rng, 1.0, 8.0, 2)
    else:
        X, F = meshgen.mobius(120, 17, 1.0, 0.4)
        q = meshgen.sample_queries(X, F, 20000, rng, 0.2, 1.5, 2)
    X32 = parity.as_f32(X)
    mesh = sg.Mesh(X32, F)
    gpu = parity.run_gpu(mesh, q, 2)
    ref, om = parity.run_oracle(X32, F, q, 2)
    r = parity.compare(gpu, ref, meshgen.bbox_diag(X), 2, what=which, max_flagged=0.05)
    flipped = (gpu["status"] & sg.ST_FLIPPED) != 0
    assert 0.02 < flipped.mean() < 0.9, flipped.mean()    # the seam is actually crossed
    # EP with the transported end frame
    out = sg.exp_map(mesh, q.face, parity.as_f32(q.bary), parity.as_f32(q.v))
    rb = sg.exp_map_backward(mesh, "ep", q.face, parity.as_f32(q.bary), parity.as_f32(q.v), out["face"],
                             out["bary"], out["dir"], out["status"], parity.as_f32(q.g_pos))
    torch.cuda.synchronize()
    ep = oracle.ep_backward(om, q.face, parity.as_f32(q.bary).astype(np.float64),
                            parity.as_f32(q.v).astype(np.float64), parity.as_f32(q.g_pos).astype(np.float64))
    st = out["status"].cpu().numpy().astype(np.uint32) | ep["flags"]
    ok = (st & (parity.FLAGS | oracle.BOUNDARY)) == 0
    gv = rb["grad_v"].cpu().numpy()
    rel = np.linalg.norm(gv - ep["grad_v"], axis=1) / np.maximum(np.linalg.norm(ep["grad_v"], axis=1), 1e-12)
    assert rel[ok].max() < 1e-3
    print(which, r, "flipped", flipped.mean())


def test_vertex_gradient_on_klein_bottle_matches_central_differences():
    """grad_V across orientation-reversing edges: <grad_V, dX> vs FP64 central differences of
    sum_q g_q . Exp_q(X) on queries whose face sequence is unchanged at X +- h dX."""
    import torch
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(43)
    X, F = meshgen.klein_bottle(48, 24)
    X32 = parity.as_f32(X)
    Xd = X32.astype(np.float64)
    q = meshgen.sample_queries(X, F, 1500, rng, 1.0, 6.0, 0)
    b = parity.as_f32(q.bary).astype(np.float64)
    v = parity.as_f32(q.v).astype(np.float64)
    g = parity.as_f32(q.g_pos).astype(np.float64)
    mesh = sg.Mesh(X32, F)
    base = oracle.exp_map(oracle.Mesh(Xd, F), q.face, b, v)
    out = sg.exp_map(mesh, q.face, parity.as_f32(q.bary), parity.as_f32(q.v))
    flipped = (out["status"].cpu().numpy() & sg.ST_FLIPPED) != 0
    assert flipped.mean() > 0.1   # enough walks end across an odd number of flipped edges
    h = 1e-5
    for trial in range(2):
        dX = rng.normal(size=X.shape)
        op = oracle.exp_map(oracle.Mesh(Xd + h * dX, F), q.face, b, v)
        on = oracle.exp_map(oracle.Mesh(Xd - h * dX, F), q.face, b, v)
        keep = (op["hash"] == base["hash"]) & (on["hash"] == base["hash"])
        keep &= (base["status"] & (oracle.BOUNDARY | oracle.VERTEX_HIT | parity.FLAGS)) == 0
        assert keep.mean() > 0.7
        fd = (np.einsum("ij,ij->i", op["pos"], g) - np.einsum("ij,ij->i", on["pos"], g)) / (2 * h)
        gm = (g * keep[:, None]).astype(np.float32)
        r = sg.exp_map_backward(mesh, "ep", q.face, parity.as_f32(q.bary), parity.as_f32(q.v), out["face"],
                                out["bary"], out["dir"], out["status"], gm, want_grad_V=True)
        torch.cuda.synchronize()
        lhs = float(np.sum(r["grad_V"].cpu().numpy().astype(np.float64) * dX))
        rhs = float(np.sum(fd[keep]))
        assert abs(lhs - rhs) <= 1e-3 * float(np.sum(np.abs(fd[keep]))), (lhs, rhs)
