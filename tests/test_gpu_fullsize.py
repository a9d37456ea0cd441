"""The benchmarked step at full size: noisy icosphere s6 (81,920 faces) with 1,048,576 queries,
L ~ U[0.1, 1], forward + EP + GFD + vertex gradient, in the launch configuration the benchmark
times (persistent kernels, queries in walk-length order, FP64-escalated classification,
caller-provided workspaces).  Sampled outputs are checked one by one against the FP64 oracle;
the vertex gradient, a sum over every query, is checked against FP64 central differences of
the oracle over the whole batch.

Bars: those of tests/parity.py (forward) and tests/test_gpu_backward.py (relative 1e-3 for EP,
for GFD on unsplit queries and against central differences, and for <grad_V, dX>)."""
import numpy as np
import pytest

import meshgen
import oracle
from tests import parity
from tests.test_oracle_pins import fd_gradients

pytestmark = pytest.mark.gpu

EPS = 1e-4


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-12)


@pytest.fixture(scope="module")
def step():
    import torch
    import paper_2603_15780_gb300 as sg
    wl = meshgen.workload(2)
    X, F = wl.single
    X32 = parity.as_f32(X)
    q = wl.queries
    assert len(q) == 1048576
    dev = "cuda"
    mesh = sg.Mesh(X32, F)
    face = torch.tensor(q.face, device=dev)
    bary = torch.tensor(parity.as_f32(q.bary), device=dev)
    v = torch.tensor(parity.as_f32(q.v), device=dev)
    g = torch.tensor(parity.as_f32(q.g_pos), device=dev)
    nq = len(q)
    opts = sg.default_opts(kernel=2, sort=-1, fp64_escalate=1)
    ws = torch.empty(sg.workspace_size(mesh, nq, opts), dtype=torch.uint8, device=dev)
    bopts = sg.default_opts(sort=-1)
    bws = torch.empty(sg.backward_workspace_size(mesh, "gfd", nq, True), dtype=torch.uint8, device=dev)
    fw = sg.exp_map(mesh, face, bary, v, workspace=ws, opts=opts, want_hash=True)

    def backward(est, gg, grad_V=False):
        gV = torch.zeros(mesh.n_vertices, 3, device=dev) if grad_V else None
        r = sg.exp_map_backward(mesh, est, face, bary, v, fw["face"], fw["bary"], fw["dir"], fw["status"], gg,
                                eps_v=EPS, eps_p=EPS, grad_V=gV, opts=bopts, workspace=bws)
        torch.cuda.synchronize()
        out = {k: t.cpu().numpy() for k, t in r.items() if t is not None}
        if grad_V:
            out["grad_V"] = gV.cpu().numpy()
        out["status"] = out["status"].astype(np.uint32)
        return out

    ep = backward("ep", g)
    gfd = backward("gfd", g, grad_V=True)
    fwd = {k: t.cpu().numpy() for k, t in fw.items() if k != "_workspace" and t is not None}
    fwd["status"] = fwd["status"].astype(np.uint32)
    fwd["hash"] = fwd["hash"].view(np.uint64)
    idx = np.sort(np.random.default_rng(77).choice(nq, 2000, replace=False))
    return {"X32": X32, "F": F, "q": q, "mesh": mesh, "fwd": fwd, "ep": ep, "gfd": gfd, "idx": idx,
            "backward": backward, "torch_g": g}


def _sample(q, idx):
    b, v, g = (parity.as_f32(a).astype(np.float64) for a in (q.bary, q.v, q.g_pos))
    return meshgen.Queries(q.face[idx], b[idx], v[idx], q.w[idx], g[idx])


def test_forward_sampled(step):
    X32, F, q, idx = step["X32"], step["F"], step["q"], step["idx"]
    ref, _ = parity.run_oracle(X32, F, q.take(idx), 0)
    sub = {k: a[idx] for k, a in step["fwd"].items()}
    r = parity.compare(sub, ref, meshgen.bbox_diag(X32.astype(np.float64)), 0, what="icosphere s6 1M")
    print("forward", r)


def test_ep_sampled(step):
    X32, F, q, idx = step["X32"], step["F"], step["q"], step["idx"]
    qs = _sample(q, idx)
    om = oracle.Mesh(X32.astype(np.float64), F)
    ref = oracle.ep_backward(om, qs.face, qs.bary, qs.v, qs.g_pos)
    gpu = {k: a[idx] for k, a in step["ep"].items() if k != "grad_V"}
    ok = ((step["fwd"]["status"][idx] | ref["flags"]) & (parity.FLAGS | oracle.BOUNDARY)) == 0
    assert ok.mean() > 0.95
    assert rel(gpu["grad_v"], ref["grad_v"])[ok].max() < 1e-3


def test_gfd_sampled(step):
    """Quiet queries within 1e-3 of the oracle's literal GFD and, where the perturbed FP64
    walks keep the face sequence, of central differences.  Split queries (a perturbation sweeps
    a vertex, so central differences do not apply) are evaluated on the GPU by literal walks
    restarted at the first swept corner, and compared with the oracle's literal walks from the
    start."""
    X32, F, q, idx = step["X32"], step["F"], step["q"], step["idx"]
    qs = _sample(q, idx)
    Xd = X32.astype(np.float64)
    om = oracle.Mesh(Xd, F)
    gpu = {k: a[idx] for k, a in step["gfd"].items() if k != "grad_V"}
    ref = oracle.gfd_backward(om, qs.face, qs.bary, qs.v, qs.g_pos, EPS, EPS)
    quiet = ((gpu["status"] | ref["flags"]) & (parity.FLAGS | oracle.BOUNDARY)) == 0
    split = (gpu["status"] & 256) != 0  # SG_ST_GFD_SPLIT
    unsplit = quiet & ~split
    assert unsplit.mean() > 0.6
    assert rel(gpu["grad_v"], ref["grad_v"])[unsplit].max() < 1e-3
    assert rel(gpu["grad_p"], ref["grad_p"])[unsplit].max() < 1e-3
    gv_fd, gp_fd, strad = fd_gradients(om, Xd, F, qs)
    keep = quiet & ~strad
    assert keep.mean() > 0.6
    e_v, e_p = rel(gpu["grad_v"], gv_fd)[keep], rel(gpu["grad_p"], gp_fd)[keep]
    qsplit = quiet & split
    s_v, s_p = rel(gpu["grad_v"], ref["grad_v"])[qsplit], rel(gpu["grad_p"], ref["grad_p"])[qsplit]
    print("gfd split fraction", split.mean(), "max rel err vs FD: grad_v", e_v.max(), "grad_p", e_p.max(),
          "split vs oracle literal: n", qsplit.sum(), "grad_v median/p90/max", np.median(s_v), np.quantile(s_v, 0.9),
          s_v.max(), "grad_p median/p90/max", np.median(s_p), np.quantile(s_p, 0.9), s_p.max())
    assert e_v.max() < 1e-3 and e_p.max() < 1e-3
    assert qsplit.sum() > 50
    assert s_v.max() < 1e-3 and s_p.max() < 1e-3


def test_vertex_gradient_full_batch(step):
    """<grad_V, dX> over all queries whose oracle face sequence is unchanged at X +- h dX
    (the others get a zero upstream gradient) vs central differences of sum_q g_q . Exp_q."""
    import torch
    X32, F, q = step["X32"], step["F"], step["q"]
    Xd = X32.astype(np.float64)
    b, v, g = (parity.as_f32(a).astype(np.float64) for a in (q.bary, q.v, q.g_pos))
    # 64 crossings per walk on average: a small step keeps most face sequences unchanged
    h = 2e-6
    dX = np.random.default_rng(78).normal(size=Xd.shape)
    base = oracle.exp_map(oracle.Mesh(Xd, F), q.face, b, v)
    op = oracle.exp_map(oracle.Mesh(Xd + h * dX, F), q.face, b, v)
    on = oracle.exp_map(oracle.Mesh(Xd - h * dX, F), q.face, b, v)
    keep = (op["hash"] == base["hash"]) & (on["hash"] == base["hash"])
    keep &= (base["status"] & (oracle.BOUNDARY | oracle.VERTEX_HIT | parity.FLAGS)) == 0
    keep &= (step["fwd"]["status"] & parity.FLAGS) == 0
    assert keep.mean() > 0.5
    fd = (np.einsum("ij,ij->i", op["pos"], g) - np.einsum("ij,ij->i", on["pos"], g)) / (2 * h)
    gm = torch.tensor((g * keep[:, None]).astype(np.float32), device="cuda")
    r = step["backward"]("gfd", gm, grad_V=True)
    lhs = float(np.sum(r["grad_V"].astype(np.float64) * dX))
    rhs = float(np.sum(fd[keep]))
    # the sum of N per-query values each within a relative error e is within e |fd|_2 when the
    # errors are independent: the norm, not the sum of magnitudes, is the scale
    scale = float(np.linalg.norm(fd[keep]))
    print("grad_V full batch", lhs, rhs, scale, "kept", keep.mean(), "err / |fd|", abs(lhs - rhs) / scale)
    assert abs(lhs - rhs) <= 1e-3 * scale, (lhs, rhs, scale)
