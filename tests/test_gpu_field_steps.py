"""GPU parity of the fused K-step exponential map of a vertex-sampled vector field
(sg_exp_map_steps, Sec. 5 Eq. "fmobj": x_{k+1} = Exp_{x_k}(h u(x_k)) with u interpolated from
vertex values) and of its backward (sg_exp_map_steps_backward), against an oracle chain of K FP64
walks that evaluates the same field at each intermediate point.

Bars: each step's face sequence bit-exact on queries that no side flags at any step; the end point
within 1e-5 of the bbox diagonal; the gradients in the field and in the start barycentrics within
1e-3 of FP64 central differences of the oracle chain (norm of the per-query difference quotients as
the scale), on queries whose face sequences the perturbations leave unchanged.
"""
import numpy as np
import pytest

import meshgen
import oracle
from tests import parity

pytestmark = pytest.mark.gpu

K = 5


def sg():
    import paper_2603_15780_gb300 as m
    return m


def _setup(nq=2000, seed=71):
    rng = np.random.default_rng(seed)
    X, F = meshgen.icosphere(4, 0.004, rng)
    X32 = parity.as_f32(X)
    q = meshgen.sample_queries(X, F, nq, rng, 0.0, 1.0, 0)
    U = (0.8 * rng.normal(size=X.shape)).astype(np.float32)
    return rng, X32, F, q, U


def oracle_chain(om, X, F, face, bary, U, K, h):
    """K oracle walks, each from the previous end (face, barycentrics), with the vector h sum_j
    max(b_j, 0) U[F[f, j]] (the field interpolated at the step's start)."""
    hashes, st = [], np.zeros(len(face), np.uint32)
    for _ in range(K):
        c = np.maximum(bary, 0.0)
        v = h * np.einsum("qj,qjc->qc", c, U[F[face]])
        out = oracle.exp_map(om, face, bary, v)
        face, bary = out["face"], out["bary"]
        hashes.append(out["hash"])
        st = st | out["status"]
    return out["pos"], np.stack(hashes, 1), st


def test_each_step_matches_the_oracle():
    """Every step of the fused chain against the oracle walk from that step's recorded start (face,
    barycentrics, vector): face sequences bit-exact on unflagged steps, end points within 1e-5 of
    the bbox diagonal, and each step starting exactly where the previous one ended.  The field is
    random at every vertex, the roughest case: the chain itself amplifies a start difference about
    fivefold per step there, which is why each step is checked from its own recorded start."""
    import torch
    S = sg()
    rng, X32, F, q, U = _setup()
    Xd = X32.astype(np.float64)
    om = oracle.Mesh(Xd, F)
    mesh = S.Mesh(X32, F)
    out = S.exp_map_field_steps(mesh, q.face, parity.as_f32(q.bary), U, K, want_hash=True)
    torch.cuda.synchronize()
    diag = meshgen.bbox_diag(X32)
    rec = {k: out[k].cpu().numpy() for k in ("step_face", "step_bary", "step_v", "step_status", "step_hash")}
    for k in range(K):
        ref = oracle.exp_map(om, rec["step_face"][k], rec["step_bary"][k].astype(np.float64),
                             rec["step_v"][k].astype(np.float64))
        st = rec["step_status"][k].astype(np.uint32)
        ok = ((st | ref["status"]) & parity.FLAGS) == 0
        assert ok.mean() > 0.97, (k, ok.mean())
        assert np.array_equal(rec["step_hash"][k].view(np.uint64)[ok], ref["hash"][ok]), k
        assert np.array_equal(rec["step_face"][k + 1][ok], ref["face"][ok]), k
        pk = (rec["step_bary"][k + 1].astype(np.float64)[:, :, None] * Xd[F[rec["step_face"][k + 1]]]).sum(1)
        err = np.linalg.norm(pk - ref["pos"], axis=1)[ok]
        assert err.max() <= 1e-5 * diag, (k, err.max() / diag)
    assert np.array_equal(rec["step_face"][K], out["face"].cpu().numpy())
    assert np.abs(rec["step_bary"][K] - out["bary"].cpu().numpy()).max() == 0.0


def test_field_steps_match_the_oracle_chain():
    """The whole chain against the oracle's chain of K walks, for a field smooth at the scale of the
    faces (the vertex values of a linear field, u(x) = A x): face sequences of every step bit-exact
    on unflagged queries, the end point within 1e-5 of the bbox diagonal."""
    import torch
    S = sg()
    rng, X32, F, q, _ = _setup()
    Xd = X32.astype(np.float64)
    U = (Xd @ (0.8 * rng.normal(size=(3, 3))).T).astype(np.float32)
    mesh = S.Mesh(X32, F)
    b32 = parity.as_f32(q.bary)
    out = S.exp_map_field_steps(mesh, q.face, b32, U, K, want_hash=True)
    torch.cuda.synchronize()
    xo, ho, so = oracle_chain(oracle.Mesh(Xd, F), Xd, F, q.face, b32.astype(np.float64), U.astype(np.float64), K,
                              1.0 / K)
    st_g = out["step_status"].cpu().numpy().astype(np.uint32)
    flag = ((np.bitwise_or.reduce(st_g, 0) | so) & parity.FLAGS) != 0
    ok = ~flag
    assert ok.mean() > 0.9
    hg = out["step_hash"].cpu().numpy().view(np.uint64).T
    bad = np.nonzero(ok & ~np.all(hg == ho, 1))[0]
    assert len(bad) == 0, f"step face sequences differ on {len(bad)} unflagged queries, e.g. {bad[:5]}"
    err = np.linalg.norm(out["pos"].cpu().numpy() - xo, axis=1)[ok]
    diag = meshgen.bbox_diag(X32)
    print("field steps: flagged", flag.mean(), "max end error / diag", err.max() / diag)
    assert err.max() <= 1e-5 * diag


@pytest.mark.parametrize("wrt", ["field", "start_bary"])
def test_field_steps_gradient_matches_central_differences(wrt):
    """d/dU and d/db_0 of sum_q g_q . x_K (GFD at step 1e-5, below the bend of chords that cross an
    edge near an intermediate end point) against FP64 central differences of the oracle chain."""
    import torch
    S = sg()
    rng, X32, F, q, U = _setup(nq=1500, seed=72)
    Xd = X32.astype(np.float64)
    om = oracle.Mesh(Xd, F)
    mesh = S.Mesh(X32, F)
    b32 = parity.as_f32(q.bary)
    b64 = b32.astype(np.float64)
    U64 = U.astype(np.float64)
    g = rng.normal(size=(len(q), 3))
    eps = 1e-5
    fwd = S.exp_map_field_steps(mesh, q.face, b32, U, K, want_hash=True)
    st = np.bitwise_or.reduce(fwd["step_status"].cpu().numpy().astype(np.uint32), 0)
    x0, h0, s0 = oracle_chain(om, Xd, F, q.face, b64, U64, K, 1.0 / K)
    keep = ((st | s0) & (parity.FLAGS | oracle.BOUNDARY | oracle.INVALID | oracle.VERTEX_HIT)) == 0
    # the same chain of faces on both sides (see test_each_step_matches_the_oracle)
    keep &= np.all(fwd["step_hash"].cpu().numpy().view(np.uint64).T == h0, 1)
    hf = 1e-6
    if wrt == "field":
        d = rng.normal(size=U.shape)
        xp, hp, _ = oracle_chain(om, Xd, F, q.face, b64, U64 + hf * d, K, 1.0 / K)
        xn, hn, _ = oracle_chain(om, Xd, F, q.face, b64, U64 - hf * d, K, 1.0 / K)
    else:
        d = rng.normal(size=(len(q), 3))
        d -= d.mean(1, keepdims=True)            # along the simplex (sum of the change zero)
        d *= (b64 > 1e-3).all(1, keepdims=True)  # away from the start face's edges
        xp, hp, _ = oracle_chain(om, Xd, F, q.face, b64 + hf * d, U64, K, 1.0 / K)
        xn, hn, _ = oracle_chain(om, Xd, F, q.face, b64 - hf * d, U64, K, 1.0 / K)
    keep &= np.all(hp == h0, 1) & np.all(hn == h0, 1)
    # a GFD column that swept a vertex at some step is a finite difference across it, not the derivative
    for k in range(K):
        r = S.exp_map_backward(mesh, "gfd", fwd["step_face"][k], fwd["step_bary"][k], fwd["step_v"][k],
                               fwd["step_face"][k + 1], fwd["step_bary"][k + 1], fwd["step_dir"][k],
                               fwd["step_status"][k], torch.zeros(len(q), 3, device="cuda"), eps_v=eps, eps_p=eps)
        keep &= (r["status"].cpu().numpy() & sg().ST_GFD_SPLIT) == 0
    assert keep.mean() > 0.8
    fd = np.einsum("qc,qc->q", xp - xn, g) / (2 * hf)
    gm = (g * keep[:, None]).astype(np.float32)
    r = S.exp_map_field_steps_backward(mesh, "gfd", fwd, U, K, 1.0 / K, gm, eps_v=eps, eps_p=eps)
    torch.cuda.synchronize()
    if wrt == "field":
        lhs = float(np.sum(r["grad_U"].cpu().numpy().astype(np.float64) * d))
    else:
        lhs = float(np.sum(r["grad_bary"].cpu().numpy().astype(np.float64) * d))
    rhs = float(np.sum(fd[keep]))
    scale = float(np.linalg.norm(fd[keep]))
    print(f"field steps d/d{wrt}: kept {keep.mean():.3f}, err / |fd| = {abs(lhs - rhs) / scale:.2e}")
    assert abs(lhs - rhs) <= 1e-3 * scale, (lhs, rhs, scale)


def test_field_steps_autograd_matches_the_direct_backward():
    import torch
    S = sg()
    rng, X32, F, q, U = _setup(nq=800, seed=73)
    mesh = S.Mesh(X32, F)
    b = torch.tensor(parity.as_f32(q.bary), device="cuda", requires_grad=True)
    Ut = torch.tensor(U, device="cuda", requires_grad=True)
    g = torch.tensor(rng.normal(size=(len(q), 3)).astype(np.float32), device="cuda")
    pos, face, bary, d, st = S.ExpMapFieldSteps.apply(mesh, torch.tensor(q.face, device="cuda"), b, Ut, K)
    (pos * g).sum().backward()
    fwd = S.exp_map_field_steps(mesh, q.face, parity.as_f32(q.bary), U, K)
    r = S.exp_map_field_steps_backward(mesh, "gfd", fwd, U, K, 1.0 / K, g)
    torch.cuda.synchronize()
    assert torch.equal(pos, fwd["pos"])
    assert torch.allclose(Ut.grad, r["grad_U"], rtol=1e-5, atol=1e-6)
    assert torch.allclose(b.grad, r["grad_bary"], rtol=1e-5, atol=1e-6)


def test_field_steps_edge_cases():
    """A zero field is the identity; an invalid start is INVALID with its start kept; K = 1 equals
    one sg_exp_map call with v = h u(x_0)."""
    import torch
    S = sg()
    rng, X32, F, q, U = _setup(nq=300, seed=74)
    mesh = S.Mesh(X32, F)
    b32 = parity.as_f32(q.bary)
    z = S.exp_map_field_steps(mesh, q.face, b32, np.zeros_like(U), K)
    p0 = (b32.astype(np.float64)[:, :, None] * X32.astype(np.float64)[F[q.face]]).sum(1)
    assert np.abs(z["pos"].cpu().numpy() - p0).max() < 1e-6
    assert np.array_equal(z["face"].cpu().numpy(), q.face)
    face = q.face.copy()
    face[0] = len(F)
    bad = S.exp_map_field_steps(mesh, face, b32, U, K)
    assert bad["status"][0].item() & S.ST_INVALID
    one = S.exp_map_field_steps(mesh, q.face, b32, U, 1, h=0.3)
    c = np.maximum(b32, 0.0)
    v = 0.3 * np.einsum("qj,qjc->qc", c, U[F[q.face]])
    ref = S.exp_map(mesh, q.face, b32, v.astype(np.float32), precision=32)
    torch.cuda.synchronize()
    ok = (((one["status"] | ref["status"]).cpu().numpy()) & parity.FLAGS) == 0
    assert np.array_equal(one["face"].cpu().numpy()[ok], ref["face"].cpu().numpy()[ok])
    assert np.abs(one["pos"].cpu().numpy() - ref["pos"].cpu().numpy())[ok].max() < 1e-5
    with pytest.raises(S.SgError):
        S.exp_map_field_steps(mesh, q.face, b32, U, 0)
