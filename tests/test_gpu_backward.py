"""GPU parity of the backward estimators (sg_exp_map_backward) against the FP64 oracle and
against FP64 central differences of the oracle walk.

Bars (relative error |a - b| / |b| per query, on queries whose perturbed oracle walks keep
the base face sequence, i.e. where the map is differentiable):
  EP grad_v vs oracle EP                      <= 1e-3
  GFD grad_v, grad_p vs central differences   <= 1e-3
  GFD vs oracle GFD                           <= 1e-3 (unsplit queries)
  grad_V . dX vs central differences          <= 1e-3 |fd| (summed over non-straddling queries;
                                              |fd| the norm of the per-query difference quotients)
  grad_V per vertex and component             <= 1e-3 |fd_v| (64 vertices, FP64 central differences)
"""
import numpy as np
import pytest

import meshgen
import oracle
from tests import parity
from tests.test_oracle_pins import fd_gradients

pytestmark = pytest.mark.gpu


def sg():
    import paper_2603_15780_gb300 as m
    return m


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-12)


def forward_backward(mesh, q, estimator, eps=1e-4, grad_V=False, g=None):
    import torch
    S = sg()
    f32 = parity.as_f32
    out = S.exp_map(mesh, q.face, f32(q.bary), f32(q.v))
    gg = f32(q.g_pos if g is None else g)
    r = S.exp_map_backward(mesh, estimator, q.face, f32(q.bary), f32(q.v), out["face"], out["bary"], out["dir"], out["status"],
                           gg, eps_v=eps, eps_p=eps, want_grad_V=grad_V)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in r.items()}
    res["status"] = res["status"].astype(np.uint32)
    res["fwd_status"] = out["status"].cpu().numpy().astype(np.uint32)
    return res


def f64(q):
    return (parity.as_f32(q.bary).astype(np.float64), parity.as_f32(q.v).astype(np.float64),
            parity.as_f32(q.g_pos).astype(np.float64))


@pytest.fixture(scope="module")
def sphere6():
    wl = meshgen.workload(2, scale=8000 / 1048576)
    X, F = wl.single
    X32 = parity.as_f32(X)
    return X32, F, wl.queries, sg().Mesh(X32, F), oracle.Mesh(X32.astype(np.float64), F)


def test_ep_matches_oracle_and_fd(sphere6):
    """Eq. proxy_func: J^v = R.  GPU EP grad_v vs the oracle's EP and vs central differences."""
    X32, F, q, mesh, om = sphere6
    b, v, g = f64(q)
    gpu = forward_backward(mesh, q, "ep")
    ref = oracle.ep_backward(om, q.face, b, v, g)
    ok = ((gpu["fwd_status"] | ref["flags"]) & (parity.FLAGS | oracle.BOUNDARY)) == 0
    assert ok.mean() > 0.95
    assert rel(gpu["grad_v"], ref["grad_v"])[ok].max() < 1e-3
    assert np.all(gpu["grad_p"] == 0) and np.all(gpu["grad_bary"] == 0)
    sub = np.arange(2000)
    qs = q.take(sub)
    qs = meshgen.Queries(qs.face, b[sub], v[sub], qs.w, g[sub])
    gv_fd, _, strad = fd_gradients(om, X32.astype(np.float64), F, qs)
    keep = ~strad & ok[sub]
    assert keep.mean() > 0.6
    assert rel(gpu["grad_v"][sub], gv_fd)[keep].max() < 1e-3


def test_gfd_matches_central_differences(sphere6):
    """Eqs. jv, jp: GPU GFD grad_v and grad_p within 1e-3 of FP64 central differences on
    queries whose perturbed walks keep the face sequence; grad_bary = <grad_p, x_k>."""
    X32, F, q, mesh, om = sphere6
    b, v, g = f64(q)
    sub = np.arange(3000)
    qs = meshgen.Queries(q.face[sub], b[sub], v[sub], q.w[sub], g[sub])
    gpu = forward_backward(mesh, qs, "gfd")
    gv_fd, gp_fd, strad = fd_gradients(om, X32.astype(np.float64), F, qs)
    keep = ~strad & ((gpu["status"] & (parity.FLAGS | oracle.BOUNDARY)) == 0)
    assert keep.mean() > 0.6
    e_v = rel(gpu["grad_v"], gv_fd)[keep]
    e_p = rel(gpu["grad_p"], gp_fd)[keep]
    assert e_v.max() < 1e-3, e_v.max()
    assert e_p.max() < 1e-3, e_p.max()
    P = X32.astype(np.float64)[F[qs.face]]
    gb = np.einsum("qkj,qj->qk", P, gpu["grad_p"])
    assert np.abs(gb - gpu["grad_bary"]).max() < 1e-4 * np.abs(gb).max()
    # the GPU's own split detection covers every straddling perturbation it did not flag
    split = (gpu["status"] & 256) != 0  # SG_ST_GFD_SPLIT
    print("gfd split fraction", split.mean(), "fd straddle fraction", strad.mean())


def test_gfd_matches_oracle_gfd(sphere6):
    """GPU GFD (lockstep re-walk + chords, literal walks where a vertex is swept) vs the
    oracle's literal two-round GFD, same eps."""
    X32, F, q, mesh, om = sphere6
    b, v, g = f64(q)
    sub = np.arange(4000)
    qs = meshgen.Queries(q.face[sub], b[sub], v[sub], q.w[sub], g[sub])
    gpu = forward_backward(mesh, qs, "gfd")
    ref = oracle.gfd_backward(om, qs.face, b[sub], v[sub], g[sub], 1e-4, 1e-4)
    quiet = ((gpu["status"] | ref["flags"]) & (parity.FLAGS | oracle.BOUNDARY)) == 0
    unsplit = quiet & ((gpu["status"] & 256) == 0)
    assert unsplit.mean() > 0.6
    assert rel(gpu["grad_v"], ref["grad_v"])[unsplit].max() < 1e-3
    assert rel(gpu["grad_p"], ref["grad_p"])[unsplit].max() < 1e-3
    # Queries with a swept vertex: the GPU's FP32 literal walks (restarted at the first swept
    # corner) against the oracle's FP64 literal walks from the start, element-wise.  A literal
    # column is (p'' - p') / eps with float32 end points: their rounding, about 6e-8 on this unit
    # sphere, over eps = 1e-4 is about 1e-3 of a unit column, and grad_p solves a 2x2 system of two
    # such columns.  Bar: grad_v within 1e-3; grad_p within 1e-3 at the 99th percentile, 2e-3 at
    # most.
    split = quiet & ((gpu["status"] & 256) != 0)
    assert split.sum() > 100, split.sum()
    s_v, s_p = rel(gpu["grad_v"], ref["grad_v"])[split], rel(gpu["grad_p"], ref["grad_p"])[split]
    print("split queries", split.sum(), "grad_v max", s_v.max(), "grad_p p99", np.quantile(s_p, 0.99),
          "max", s_p.max())
    assert s_v.max() < 1e-3
    assert np.quantile(s_p, 0.99) < 1e-3 and s_p.max() < 2e-3


def test_flat_mesh_gradients_closed_form():
    """On a flat mesh Exp(p, v) = p + v: grad_v = grad_p = in-plane part of g (both
    estimators), and grad_V = b_k * in-plane(g) on the start face's vertices plus
    b'_j (g . n) n on the end face's vertices."""
    rng = np.random.default_rng(31)
    X, F = meshgen.flat_grid(25, rng, jitter=0.25)
    X32 = parity.as_f32(X)
    q = meshgen.sample_queries(X, F, 3000, rng, 0.05, 0.3, 0)
    mesh = sg().Mesh(X32, F)
    gpl = parity.as_f32(q.g_pos).astype(np.float64).copy()
    gpl[:, 2] = 0.0
    for est in ("ep", "gfd"):
        r = forward_backward(mesh, q, est, grad_V=True)
        ok = ((r["fwd_status"] | r["status"]) & (oracle.BOUNDARY | parity.FLAGS)) == 0
        assert ok.mean() > 0.7
        assert rel(r["grad_v"], gpl)[ok].max() < 1e-3
        if est == "gfd":
            assert rel(r["grad_p"], gpl)[ok].max() < 1e-3
    # grad_V closed form on a subset of clean queries
    import torch
    S = sg()
    out = S.exp_map(mesh, q.face, parity.as_f32(q.bary), parity.as_f32(q.v))
    st = out["status"].cpu().numpy().astype(np.uint32)
    clean = (st & (oracle.BOUNDARY | parity.FLAGS | oracle.VERTEX_HIT)) == 0
    g = parity.as_f32(q.g_pos) * clean[:, None]
    r = S.exp_map_backward(mesh, "ep", q.face, parity.as_f32(q.bary), parity.as_f32(q.v), out["face"],
                           out["bary"], out["dir"], out["status"], g, want_grad_V=True)
    gV = r["grad_V"].cpu().numpy()
    expect = np.zeros_like(gV, dtype=np.float64)
    ef = out["face"].cpu().numpy()
    eb = out["bary"].cpu().numpy().astype(np.float64)
    b32 = parity.as_f32(q.bary).astype(np.float64)
    for i in np.nonzero(clean)[0]:
        gi = g[i].astype(np.float64)
        for k in range(3):
            expect[F[q.face[i], k], :2] += b32[i, k] * gi[:2]
            expect[F[ef[i], k], 2] += eb[i, k] * gi[2]
    assert np.abs(gV - expect).max() < 1e-3 * np.abs(expect).max()


def test_vertex_gradient_matches_central_differences():
    """grad_V (a.e. derivative with the face sequence held fixed): <grad_V, dX> vs FP64 central
    differences of sum_q g_q . Exp_q(X) along random vertex directions dX, summed over
    queries whose face sequence is unchanged at X +- h dX."""
    rng = np.random.default_rng(32)
    X, F = meshgen.icosphere(4, 0.01, rng)
    X32 = parity.as_f32(X)
    Xd = X32.astype(np.float64)
    q = meshgen.sample_queries(X, F, 1500, rng, 0.1, 1.0, 0)
    b, v, g = f64(q)
    mesh = sg().Mesh(X32, F)
    om = oracle.Mesh(Xd, F)
    base = oracle.exp_map(om, q.face, b, v)
    h = 1e-5
    for trial in range(3):
        dX = rng.normal(size=X.shape)
        op = oracle.exp_map(oracle.Mesh(Xd + h * dX, F), q.face, b, v)
        on = oracle.exp_map(oracle.Mesh(Xd - h * dX, F), q.face, b, v)
        keep = (op["hash"] == base["hash"]) & (on["hash"] == base["hash"])
        keep &= (base["status"] & (oracle.BOUNDARY | oracle.VERTEX_HIT | parity.FLAGS)) == 0
        assert keep.mean() > 0.8
        fd = (np.einsum("ij,ij->i", op["pos"], g) - np.einsum("ij,ij->i", on["pos"], g)) / (2 * h)
        gm = (g * keep[:, None]).astype(np.float32)
        r = forward_backward(mesh, q, "ep", grad_V=True, g=gm)
        lhs = float(np.sum(r["grad_V"].astype(np.float64) * dX))
        rhs = float(np.sum(fd[keep]))
        scale = float(np.linalg.norm(fd[keep]))
        assert abs(lhs - rhs) <= 1e-3 * scale, (lhs, rhs, scale)
        # per-query check on a few queries
        for i in np.nonzero(keep)[0][:5]:
            gi = np.zeros_like(gm); gi[i] = gm[i]
            ri = forward_backward(mesh, q, "ep", grad_V=True, g=gi)
            li = float(np.sum(ri["grad_V"].astype(np.float64) * dX))
            assert abs(li - fd[i]) <= 2e-3 * max(abs(fd[i]), 1e-3 * np.abs(dX).max() * np.linalg.norm(g[i])), (i, li, fd[i])


def test_vertex_gradient_per_vertex_central_differences():
    """grad_V vertex by vertex on the 81,920-face noisy icosphere of the benchmark: for the 64
    vertices with the largest gradient under 4096 queries (L ~ U[0.1, 1]), every component
    against the FP64 central difference of sum_q g_q . Exp_q(X) in that one coordinate, over the
    queries whose oracle face sequence is unchanged at X +- h e_(v,c) (the others get a zero
    upstream gradient on the GPU too).  Bar: |gpu - fd| <= 1e-3 |fd_v| per component, |fd_v| the
    norm of the vertex's difference quotient."""
    import torch
    S = sg()
    wl = meshgen.workload(2, scale=4096 / 1048576)
    X, F = wl.single
    X32 = parity.as_f32(X)
    Xd = X32.astype(np.float64)
    q = wl.queries
    b, v, g = f64(q)
    mesh = S.Mesh(X32, F)
    out = S.exp_map(mesh, q.face, parity.as_f32(q.bary), parity.as_f32(q.v))
    base = oracle.exp_map(oracle.Mesh(Xd, F), q.face, b, v)
    ok = (base["status"] & (oracle.BOUNDARY | oracle.VERTEX_HIT | parity.FLAGS)) == 0
    ok &= (out["status"].cpu().numpy() & parity.FLAGS) == 0

    def grad_V(mask):
        gm = torch.tensor((g * mask[:, None]).astype(np.float32), device="cuda")
        r = S.exp_map_backward(mesh, "gfd", q.face, parity.as_f32(q.bary), parity.as_f32(q.v), out["face"],
                               out["bary"], out["dir"], out["status"], gm, want_grad_V=True)
        torch.cuda.synchronize()
        return r["grad_V"].cpu().numpy().astype(np.float64)

    full = grad_V(ok)
    verts = np.argsort(-np.linalg.norm(full, axis=1))[:64]
    h = 1e-5
    gpu = np.zeros((64, 3))
    fd = np.zeros((64, 3))
    kept = []
    for i, vv in enumerate(verts):
        for c in range(3):
            Xp = Xd.copy(); Xp[vv, c] += h
            Xn = Xd.copy(); Xn[vv, c] -= h
            op = oracle.exp_map(oracle.Mesh(Xp, F), q.face, b, v)
            on = oracle.exp_map(oracle.Mesh(Xn, F), q.face, b, v)
            keep = ok & (op["hash"] == base["hash"]) & (on["hash"] == base["hash"])
            kept.append(keep[(op["pos"] != on["pos"]).any(1)].mean() if (op["pos"] != on["pos"]).any() else 1.0)
            fd[i, c] = np.sum(np.einsum("ij,ij->i", op["pos"] - on["pos"], g)[keep]) / (2 * h)
            gpu[i, c] = grad_V(keep)[vv, c]
    scale = np.linalg.norm(fd, axis=1)[:, None]
    err = np.abs(gpu - fd) / scale
    print("per-vertex grad_V: max rel", err.max(), "median", np.median(err), "queries kept near the vertices",
          float(np.mean(kept)))
    assert scale.min() > 0
    assert err.max() <= 1e-3, (err.max(), verts[np.argmax(err.max(1))])


def test_autograd_function_routes_gradients():
    """torch.autograd: ExpMap.apply gives grad for v, bary and the vertex tensor V."""
    import torch
    wl = meshgen.workload(0, scale=0.1)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    q = wl.queries
    v = torch.tensor(parity.as_f32(q.v), device="cuda", requires_grad=True)
    bary = torch.tensor(parity.as_f32(q.bary), device="cuda", requires_grad=True)
    V = torch.tensor(X32, device="cuda", requires_grad=True)
    face = torch.tensor(q.face, device="cuda")
    pos, *_ = sg().ExpMap.apply(mesh, face, bary, v, "gfd", V)
    loss = (pos * torch.tensor(parity.as_f32(q.g_pos), device="cuda")).sum()
    loss.backward()
    assert v.grad is not None and torch.isfinite(v.grad).all()
    assert bary.grad is not None and V.grad is not None
    assert V.grad.abs().sum() > 0


@pytest.mark.parametrize("estimator", ["ep", "gfd"])
def test_backward_on_the_sliver_heightfield(estimator):
    """Both estimators on a sample of the 4.2M-face sliver heightfield (~1.7k crossings per walk,
    most walks in the mixed walk under the automatic precision) against the oracle's estimator, per
    query at 1e-3 relative (of the query's gradient (grad_v, grad_p)), on queries neither side flags.  The literal GFD walks of a query walked
    by the mixed walk are mixed-precision walks with the perturbation and the column's difference
    in FP64 (FP32 literal walks carry their ~2e-7 end-point error into a difference divided by
    eps = 1e-4).  Queries whose FP32 re-walk left the forward's path are reported (their GFD columns
    are all literal walks, so they are compared as well)."""
    wl = meshgen.workload(4, scale=3000 / 16777216)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    q = wl.queries
    b, v, g = f64(q)
    om = oracle.Mesh(X32.astype(np.float64), F)
    r = forward_backward(mesh, q, estimator)
    ref = (oracle.ep_backward if estimator == "ep" else oracle.gfd_backward)(om, q.face, b, v, g)
    flag = ((r["fwd_status"] | r["status"] | ref["flags"]) & parity.FLAGS) != 0
    # error of the query's whole gradient (grad_v, grad_p): on a walk that stops at the boundary
    # the par column vanishes and the perp column is small (the perturbed ray meets the boundary
    # edge a short way off), so grad_v alone can be a near-zero vector beside the position columns
    gg = np.concatenate([r["grad_v"], r["grad_p"]], 1)
    gr = np.concatenate([ref["grad_v"], ref["grad_p"]], 1)
    e = rel(gg, gr)
    ev = rel(r["grad_v"], ref["grad_v"])
    mixed = (r["fwd_status"] & sg().ST_MIXED) != 0
    div = (r["status"] & sg().ST_REWALK_DIVERGED) != 0
    ok = ~flag
    print(f"heightfield {estimator}: flagged {flag.mean():.3f}, mixed {mixed.mean():.3f}, re-walk diverged "
          f"{div.mean():.3f}, gradient rel median {np.median(e[ok]):.2e} p99 {np.quantile(e[ok], 0.99):.2e} "
          f"max {e[ok].max():.2e}; grad_v alone: median {np.median(ev[ok]):.2e} max {ev[ok].max():.2e}")
    assert ok.mean() > 0.4
    assert mixed.mean() > 0.9
    assert (e[ok] <= 1e-3).all(), np.nonzero(ok & (e > 1e-3))[0][:10]
