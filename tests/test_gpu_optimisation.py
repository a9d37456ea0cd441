"""End-to-end use of the backward pass: optimise the tangent vectors of a batch so that the end
points reach arbitrary targets, L = sum ||Exp_p(v) - p_hat||^2 (the evaluation protocol of the
paper's gradient benchmark, App. "Speed-up GFD and EP through batching" and "Gradient
evaluation on more meshes"), with both estimators through torch.autograd."""
import numpy as np
import pytest

import meshgen
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("est", ["ep", "gfd"])
def test_reach_targets_by_gradient_descent(est):
    import torch
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(121)
    X, F = meshgen.icosphere(4, 0.004, rng)
    X32 = parity.as_f32(X)
    mesh = sg.Mesh(X32, F)
    n = 1024
    q = meshgen.sample_queries(X, F, n, rng, 0.3, 1.2, 0)
    dev = "cuda"
    face = torch.tensor(q.face, device=dev)
    bary = torch.tensor(parity.as_f32(q.bary), device=dev)
    v_true = torch.tensor(parity.as_f32(q.v), device=dev)
    with torch.no_grad():
        target = sg.exp_map(mesh, face, bary, v_true)["pos"]
    # start from the true vectors rotated by up to 0.4 rad and scaled by 0.7 .. 1.3 in the plane
    n0 = torch.nn.functional.normalize(torch.cross(X32t(X32, F, q.face, 1) - X32t(X32, F, q.face, 0),
                                                   X32t(X32, F, q.face, 2) - X32t(X32, F, q.face, 0), dim=1), dim=1)
    ang = torch.tensor(rng.uniform(-0.4, 0.4, n), dtype=torch.float32, device=dev)[:, None]
    scl = torch.tensor(rng.uniform(0.7, 1.3, n), dtype=torch.float32, device=dev)[:, None]
    v0 = scl * (torch.cos(ang) * v_true + torch.sin(ang) * torch.cross(n0, v_true, dim=1))
    v = v0.clone().requires_grad_(True)
    opt = torch.optim.Adam([v], lr=0.02)
    sched = torch.optim.lr_scheduler.ExponentialLR(opt, gamma=0.985)
    losses = []
    for it in range(300):
        opt.zero_grad()
        pos, *_ = sg.ExpMap.apply(mesh, face, bary, v, est)
        d = ((pos - target) ** 2).sum(1)
        loss = d.sum()
        loss.backward()
        opt.step()
        sched.step()
        losses.append(float(torch.sqrt(d).mean()))
    print(est, "mean distance", losses[0], "->", losses[-1])
    assert losses[-1] < 0.05 * losses[0]
    # most queries reach their target closely
    final = torch.sqrt(((sg.exp_map(mesh, face, bary, v.detach())["pos"] - target) ** 2).sum(1))
    assert float((final < 1e-2).float().mean()) > 0.9


def X32t(X32, F, face, k):
    import torch
    return torch.tensor(X32[F[face, k]], device="cuda")
