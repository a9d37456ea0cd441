"""GPU parity of sg_transport_back, the adjoint (inverse) parallel transport used by the
paper's Mesh-LBFGS (App. "Additional Details on Mesh-LBFGS and GCVT"), against the oracle's
adjoint, written from its definition with a carried start basis: on orientable meshes, on a
Klein bottle (orientation flips), for zero-length and invalid queries, and after hole
avoidance.  The GPU side also satisfies <Pi a, u> = <a, Pi* u> and Pi* Pi = the projection."""
import numpy as np
import pytest

import meshgen
import oracle
from tests import parity

pytestmark = pytest.mark.gpu


def _run(mesh, q, u, **kw):
    import torch
    import paper_2603_15780_gb300 as sg
    f32 = parity.as_f32
    face = torch.tensor(q.face, device="cuda")
    bary = torch.tensor(f32(q.bary), device="cuda")
    v = torch.tensor(f32(q.v), device="cuda")
    end = sg.exp_map(mesh, face, bary, v, **kw)
    opts = sg.default_opts(**kw) if kw else None
    back = sg.transport_back(mesh, face, bary, v, end, torch.tensor(f32(u), device="cuda"), opts=opts)
    torch.cuda.synchronize()
    return back.cpu().numpy().astype(np.float64), {k: t.cpu().numpy() for k, t in end.items()}


@pytest.mark.parametrize("which", ["icosphere", "torus", "klein"])
def test_transport_back_matches_the_oracle(which):
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(131)
    if which == "icosphere":
        X, F = meshgen.icosphere(4, 0.003, rng)
        q = meshgen.sample_queries(X, F, 6000, rng, 0.1, 2.0, 0)
    elif which == "torus":
        X, F = meshgen.torus(96, 48, 1.0, 0.4, 0.002, rng)
        q = meshgen.sample_queries(X, F, 6000, rng, 0.0, 2.0, 0)
    else:
        X, F = meshgen.klein_bottle(64, 32)
        q = meshgen.sample_queries(X, F, 6000, rng, 0.5, 4.0, 0)
    X32 = parity.as_f32(X)
    mesh = sg.Mesh(X32, F)
    u = parity.as_f32(rng.normal(size=(len(q.face), 3, 3)))
    back, end = _run(mesh, q, u)
    om = oracle.Mesh(X32.astype(np.float64), F)
    ref, fw = oracle.transport_back(om, q.face, parity.as_f32(q.bary).astype(np.float64),
                                    parity.as_f32(q.v).astype(np.float64), u.astype(np.float64))
    st = end["status"].astype(np.uint32) | fw["status"]
    ok = (st & parity.FLAGS) == 0
    assert ok.mean() > 0.9
    assert np.array_equal(end["face"][ok], fw["face"][ok])
    scale = np.linalg.norm(u, axis=2).max()
    err = np.abs(back - ref)[ok].max()
    assert err <= 2e-4 * scale, f"{which}: max err {err:.3e}"
    if which == "klein":
        assert ((end["status"] & 512) != 0)[ok].mean() > 0.05   # SG_ST_FLIPPED exercised


def test_transport_back_is_adjoint_and_inverse_of_the_forward_transport():
    import torch
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(132)
    X, F = meshgen.torus(96, 48, 1.0, 0.4, 0.002, rng)
    q = meshgen.sample_queries(X, F, 8000, rng, 0.0, 2.0, 2)
    X32 = parity.as_f32(X)
    mesh = sg.Mesh(X32, F)
    f32 = parity.as_f32
    face = torch.tensor(q.face, device="cuda")
    bary = torch.tensor(f32(q.bary), device="cuda")
    v = torch.tensor(f32(q.v), device="cuda")
    w = torch.tensor(f32(q.w), device="cuda")
    end = sg.exp_map(mesh, face, bary, v, w)
    rt = sg.transport_back(mesh, face, bary, v, end, end["w"])
    u = torch.tensor(f32(rng.normal(size=(len(q.face), 2, 3))), device="cuda")
    bu = sg.transport_back(mesh, face, bary, v, end, u)
    torch.cuda.synchronize()
    x0, x1, x2 = (torch.tensor(X32[F[q.face, k]], device="cuda") for k in range(3))
    n = torch.nn.functional.normalize(torch.cross(x1 - x0, x2 - x0, dim=1), dim=1)[:, None, :]
    wp = w - (w * n).sum(2, keepdim=True) * n
    assert float((rt - wp).abs().max()) < 1e-5
    # <Pi w, u> = <w, Pi* u> (u's normal part at the end is dropped on both sides)
    e0, e1, e2 = (torch.tensor(X32[F[end["face"].cpu().numpy(), k]], device="cuda") for k in range(3))
    nend = torch.nn.functional.normalize(torch.cross(e1 - e0, e2 - e0, dim=1), dim=1)[:, None, :]
    up = u - (u * nend).sum(2, keepdim=True) * nend
    lhs = (end["w"] * up).sum(2)
    rhs = (wp * bu).sum(2)
    assert float((lhs - rhs).abs().max()) < 2e-5


def test_transport_back_zero_length_invalid_and_explicit_zero_length():
    """A zero vector v walks an empty path: forward carries w unchanged and the inverse
    returns u projected onto the start face (the oracle's convention for both); invalid
    queries give zeros."""
    import torch
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(133)
    X, F = meshgen.icosphere(3, 0.003, rng)
    X32 = parity.as_f32(X)
    mesh = sg.Mesh(X32, F)
    n = 256
    q = meshgen.sample_queries(X, F, n, rng, 0.1, 1.0, 1)
    v = q.v.copy()
    v[: n // 2] = 0.0
    face = q.face.copy()
    face[-8:] = len(F) + 5             # invalid
    qq = meshgen.Queries(face, q.bary, v, q.w, q.g_pos)
    f32 = parity.as_f32
    gpu = sg.exp_map(mesh, torch.tensor(face, device="cuda"), torch.tensor(f32(q.bary), device="cuda"),
                     torch.tensor(f32(v), device="cuda"), torch.tensor(f32(q.w), device="cuda"))
    u = f32(rng.normal(size=(n, 3)))
    back = sg.transport_back(mesh, torch.tensor(face, device="cuda"), torch.tensor(f32(q.bary), device="cuda"),
                             torch.tensor(f32(v), device="cuda"), gpu, torch.tensor(u, device="cuda"))
    torch.cuda.synchronize()
    om = oracle.Mesh(X32.astype(np.float64), F)
    ref, _ = parity.run_oracle(X32, F, qq, 1)
    z = np.arange(n // 2)
    assert np.abs(gpu["w"].cpu().numpy()[z] - ref["w"][z]).max() < 1e-6
    rb, _ = oracle.transport_back(om, face[z], f32(q.bary[z]).astype(np.float64), np.zeros((len(z), 3)),
                                  u[z].astype(np.float64))
    assert np.abs(back.cpu().numpy()[z] - rb).max() < 1e-6
    assert np.all(back.cpu().numpy()[-8:] == 0.0)
    assert np.all((gpu["status"].cpu().numpy()[-8:] & oracle.INVALID) != 0)


def test_transport_back_after_hole_avoidance_inverts_the_forward():
    """Hole avoidance keeps each carried vector's angle to the direction, so the inverse is
    still the transposed rotation: transporting the carried vectors back returns them."""
    import torch
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(134)
    X, F = meshgen.remove_faces(*meshgen.icosphere(4, 0.003, rng), 0.06, rng)
    X32 = parity.as_f32(X)
    mesh = sg.Mesh(X32, F)
    q = meshgen.sample_queries(X, F, 4000, rng, 0.1, 2.0, 1)
    f32 = parity.as_f32
    face = torch.tensor(q.face, device="cuda")
    bary = torch.tensor(f32(q.bary), device="cuda")
    v = torch.tensor(f32(q.v), device="cuda")
    w = torch.tensor(f32(q.w[:, :1]), device="cuda")
    o = sg.default_opts(boundary_mode=1)
    end = sg.exp_map(mesh, face, bary, v, w, opts=o)
    rt = sg.transport_back(mesh, face, bary, v, end, end["w"], opts=o)
    torch.cuda.synchronize()
    st = end["status"].cpu().numpy()
    assert ((st & oracle.HOLE) != 0).mean() > 0.2
    x0, x1, x2 = (torch.tensor(X32[F[q.face, k]], device="cuda") for k in range(3))
    n = torch.nn.functional.normalize(torch.cross(x1 - x0, x2 - x0, dim=1), dim=1)[:, None, :]
    wp = w - (w * n).sum(2, keepdim=True) * n
    assert float((rt - wp).abs().max()) < 1e-5
