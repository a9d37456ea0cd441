"""GPU tests of the upstream gradients beyond the end point (sg_exp_map_backward g_bary, g_dir,
g_w) and of the K-step exponential map built on them (Sec. 5, Eq. fmobj).

  g_w    parallel transport is a rotation of the tangent planes for a fixed face sequence
         (Sec. 4 "Parallel Transport"), so grad_w = R^T g_w exactly: checked against the FP64
         oracle's transport of a probe vector.
  g_dir  d' = R v/|v| with R held fixed: exact on a flat mesh, and equal to the oracle's
         transported frame (the rotation of Eq. proxy_func) on a sphere.
  g_bary the tangent equivalent of a barycentric gradient: identical to passing that tangent as
         g_pos for grad_v / grad_p, and grad_V against FP64 central differences of sum gb . b'.
  K-step positions against the oracle chained K times, gradients in the field's parameters
         against FP64 central differences of that chain.
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


def fwd(mesh, q, nw=0):
    f32 = parity.as_f32
    w = f32(q.w[:, :nw]) if nw else None
    return sg().exp_map(mesh, q.face, f32(q.bary), f32(q.v), w, want_hash=True)


def bwd(mesh, q, out, est="ep", g_pos=None, **kw):
    import torch
    f32 = parity.as_f32
    nq = len(q.face)
    gp = torch.zeros(nq, 3, device="cuda") if g_pos is None else g_pos
    r = sg().exp_map_backward(mesh, est, q.face, f32(q.bary), f32(q.v), out["face"], out["bary"], out["dir"],
                              out["status"], gp, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in r.items()}


@pytest.fixture(scope="module")
def sphere():
    rng = np.random.default_rng(61)
    X, F = meshgen.icosphere(4, 0.004, rng)
    X32 = parity.as_f32(X)
    q = meshgen.sample_queries(X, F, 3000, rng, 0.1, 1.5, 2)
    return X32, F, q, sg().Mesh(X32, F), oracle.Mesh(X32.astype(np.float64), F)


def test_grad_w_is_the_transpose_of_transport(sphere):
    import torch
    X32, F, q, mesh, om = sphere
    out = fwd(mesh, q, 2)
    rng = np.random.default_rng(62)
    g_w = rng.normal(size=(len(q.face), 2, 3))
    r = bwd(mesh, q, out, g_w=torch.tensor(g_w, dtype=torch.float32, device="cuda"))
    # probe: a random tangent vector at the start, transported by the oracle
    e1, e2 = meshgen._tangent_frame(X32.astype(np.float64), F, q.face)
    a = rng.normal(size=(len(q.face), 2))
    dw = a[:, :1] * e1 + a[:, 1:] * e2
    ref = oracle.exp_map(om, q.face, parity.as_f32(q.bary).astype(np.float64), parity.as_f32(q.v).astype(np.float64),
                         np.stack([dw, dw], 1))
    ok = ((ref["status"] | out["status"].cpu().numpy().astype(np.uint32)) & (parity.FLAGS | oracle.INVALID)) == 0
    assert ok.mean() > 0.95
    lhs = np.einsum("qkc,qc->qk", r["grad_w"], dw)
    rhs = np.einsum("qkc,qkc->qk", g_w, ref["w"])
    scale = np.linalg.norm(g_w, axis=2) * np.linalg.norm(dw, axis=1)[:, None]
    assert np.abs(lhs - rhs)[ok].max() <= 2e-4 * scale[ok].max()


def test_grad_dir_flat_closed_form_and_sphere_rotation(sphere):
    import torch
    # flat: d' = v/|v|, so grad_v = (I - d d^T) g_dir / |v| exactly (tangential part)
    rng = np.random.default_rng(63)
    Xf, Ff = meshgen.flat_grid(31, rng, jitter=0.2)
    qf = meshgen.sample_queries(Xf, Ff, 2000, rng, 0.05, 0.3, 0)
    mf = sg().Mesh(parity.as_f32(Xf), Ff)
    out = fwd(mf, qf)
    g = rng.normal(size=(2000, 3))
    r = bwd(mf, qf, out, g_dir=torch.tensor(g, dtype=torch.float32, device="cuda"))
    v = parity.as_f32(qf.v).astype(np.float64)
    v[:, 2] = 0.0
    L = np.linalg.norm(v, axis=1, keepdims=True)
    d = v / L
    gt = g.copy(); gt[:, 2] = 0.0
    expect = (gt - np.sum(gt * d, 1, keepdims=True) * d) / L
    ok = (out["status"].cpu().numpy() & oracle.BOUNDARY) == 0
    assert np.abs(r["grad_v"] - expect)[ok].max() <= 2e-4 * np.abs(expect[ok]).max()
    # sphere: the component across d0 is (g . Pi(n x v^)) / |v|, with Pi the transport
    X32, F, q, mesh, om = sphere
    out = fwd(mesh, q)
    g = rng.normal(size=(len(q.face), 3))
    r = bwd(mesh, q, out, g_dir=torch.tensor(g, dtype=torch.float32, device="cuda"))
    b = parity.as_f32(q.bary).astype(np.float64)
    v = parity.as_f32(q.v).astype(np.float64)
    n = np.cross(X32[F[q.face, 1]] - X32[F[q.face, 0]], X32[F[q.face, 2]] - X32[F[q.face, 0]]).astype(np.float64)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    vp = v - np.sum(v * n, 1, keepdims=True) * n
    Lv = np.linalg.norm(vp, axis=1, keepdims=True)
    perp = np.cross(n, vp / Lv)
    ref = oracle.exp_map(om, q.face, b, v, perp[:, None, :])
    expect = np.sum(g * ref["w"][:, 0], 1, keepdims=True) * perp / Lv
    ok = ((ref["status"] | out["status"].cpu().numpy().astype(np.uint32)) & (parity.FLAGS | oracle.INVALID)) == 0
    err = np.linalg.norm(r["grad_v"] - expect, axis=1)
    assert err[ok].max() <= 1e-3 * np.linalg.norm(expect, axis=1)[ok].max()


@pytest.mark.parametrize("est", ["ep", "gfd"])
def test_grad_bary_equals_its_tangent_as_g_pos(sphere, est):
    import torch
    X32, F, q, mesh, om = sphere
    out = fwd(mesh, q)
    rng = np.random.default_rng(64)
    ef = out["face"].cpu().numpy()
    Xe = X32[F[ef]].astype(np.float64)                       # [nq, 3 corners, 3]
    n = np.cross(Xe[:, 1] - Xe[:, 0], Xe[:, 2] - Xe[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    gt = rng.normal(size=(len(ef), 3))
    gt -= np.sum(gt * n, 1, keepdims=True) * n               # tangent to the end face
    gb = np.einsum("qkc,qc->qk", Xe, gt) + rng.normal(size=(len(ef), 1))   # any simplex gauge
    T = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda")
    ra = bwd(mesh, q, out, est, g_pos=T(gt))
    rb = bwd(mesh, q, out, est, g_bary=T(gb))
    for k in ("grad_v", "grad_p"):
        scale = np.abs(ra[k]).max() + 1e-30
        assert np.abs(ra[k] - rb[k]).max() <= 2e-3 * scale, k


def test_grad_V_of_end_barycentrics_matches_central_differences():
    import torch
    rng = np.random.default_rng(65)
    X, F = meshgen.icosphere(4, 0.01, rng)
    X32 = parity.as_f32(X)
    Xd = X32.astype(np.float64)
    q = meshgen.sample_queries(X, F, 1500, rng, 0.1, 1.0, 0)
    b = parity.as_f32(q.bary).astype(np.float64)
    v = parity.as_f32(q.v).astype(np.float64)
    gb = rng.normal(size=(1500, 3))
    mesh = sg().Mesh(X32, F)
    base = oracle.exp_map(oracle.Mesh(Xd, F), q.face, b, v)
    h = 1e-5
    out = fwd(mesh, q)
    for trial in range(2):
        dX = rng.normal(size=X.shape)
        op = oracle.exp_map(oracle.Mesh(Xd + h * dX, F), q.face, b, v)
        on = oracle.exp_map(oracle.Mesh(Xd - h * dX, F), q.face, b, v)
        keep = (op["hash"] == base["hash"]) & (on["hash"] == base["hash"])
        keep &= (base["status"] & (oracle.BOUNDARY | oracle.VERTEX_HIT | parity.FLAGS)) == 0
        assert keep.mean() > 0.8
        fd = (np.einsum("ij,ij->i", op["bary"], gb) - np.einsum("ij,ij->i", on["bary"], gb)) / (2 * h)
        gbm = torch.tensor(gb * keep[:, None], dtype=torch.float32, device="cuda")
        r = bwd(mesh, q, out, "ep", g_bary=gbm, want_grad_V=True)
        lhs = float(np.sum(r["grad_V"] * dX))
        rhs = float(np.sum(fd[keep]))
        scale = float(np.linalg.norm(fd[keep]))
        print("grad_V through g_bary: err / |fd| =", abs(lhs - rhs) / scale)
        assert abs(lhs - rhs) <= 1e-3 * scale, (lhs, rhs, scale)


def _oracle_chain(om, X, F, face, bary, A, K):
    x = (bary[:, :, None] * X[F[face]]).sum(1)
    hashes, st = [], 0
    for _ in range(K):
        out = oracle.exp_map(om, face, bary, (x @ A.T) / K)
        face, bary, x = out["face"], out["bary"], out["pos"]
        hashes.append(out["hash"])
        st = st | out["status"]
    return x, np.stack(hashes, 1), st


def test_k_step_exp_positions_and_field_gradient():
    import torch
    S = sg()
    rng = np.random.default_rng(66)
    X, F = meshgen.icosphere(4, 0.004, rng)
    X32 = parity.as_f32(X)
    Xd = X32.astype(np.float64)
    om = oracle.Mesh(Xd, F)
    q = meshgen.sample_queries(X, F, 1200, rng, 0.0, 1.0, 0)
    b = parity.as_f32(q.bary).astype(np.float64)
    A = 0.8 * rng.normal(size=(3, 3))
    K = 5
    mesh = S.Mesh(X32, F)
    At = torch.tensor(A, dtype=torch.float32, device="cuda", requires_grad=True)
    bt = torch.tensor(parity.as_f32(q.bary), device="cuda")
    # GFD is a finite difference with step eps: where an intermediate end point lies within eps of
    # an edge of its face, the eps-chords from it cross that edge and bend with the dihedral angle
    # there, an O(eps) difference from the derivative that the chain carries on (at eps = 1e-4 one
    # query in 200 here, 2e-2 relative on it; at 1e-5, 2e-4).  The chain rule through the K steps
    # is checked at eps = 1e-5, below the chords' bend.
    eps = 1e-5
    xK, fK, bK, st, steps = S.exp_map_steps(mesh, q.face, bt, lambda x, k: x @ At.T, K, "gfd", eps=eps,
                                            return_steps=True)
    xo, ho, so = _oracle_chain(om, Xd, F, q.face, b, A, K)
    ok = (((st.cpu().numpy().astype(np.uint32)) | so) & (parity.FLAGS | oracle.INVALID | oracle.BOUNDARY)) == 0
    assert ok.mean() > 0.9
    diag = meshgen.bbox_diag(X)
    assert np.abs(xK.detach().cpu().numpy() - xo)[ok].max() <= 1e-5 * diag
    # gradient of sum g . x_K in A against FP64 central differences of the oracle chain,
    # over queries whose face sequences do not change under the perturbations
    g = rng.normal(size=(1200, 3))
    h = 1e-6
    keep = ok.copy()
    # GFD is a finite difference with step eps = 1e-4: where a perturbed ray of some step swept a
    # vertex (SG_ST_GFD_SPLIT) it differs from the derivative, so those queries are left out
    for stp in steps:
        r = S.exp_map_backward(mesh, "gfd", stp["face"], stp["bary"], stp["v"], stp["end_face"], stp["end_bary"],
                               stp["end_dir"], stp["status"], torch.zeros(1200, 3, device="cuda"), eps_v=eps, eps_p=eps)
        keep &= (r["status"].cpu().numpy() & 256) == 0
    fd = np.zeros((3, 3, 1200))
    for i in range(3):
        for j in range(3):
            E = np.zeros((3, 3)); E[i, j] = h
            xp, hp, _ = _oracle_chain(om, Xd, F, q.face, b, A + E, K)
            xn, hn, _ = _oracle_chain(om, Xd, F, q.face, b, A - E, K)
            keep &= np.all(hp == ho, 1) & np.all(hn == ho, 1)
            fd[i, j] = np.einsum("qc,qc->q", xp - xn, g) / (2 * h)
    assert keep.mean() > 0.8
    loss = (xK * torch.tensor(g * keep[:, None], dtype=torch.float32, device="cuda")).sum()
    loss.backward()
    lhs = At.grad.cpu().numpy().astype(np.float64)
    rhs = fd[:, :, keep].sum(-1)
    print("K-step field gradient: max |gpu - fd| / max |fd| =", np.abs(lhs - rhs).max() / np.abs(rhs).max())
    assert np.abs(lhs - rhs).max() <= 1e-3 * np.abs(rhs).max(), (lhs, rhs)
