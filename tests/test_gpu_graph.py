"""GPU tests of the launch autotuner and of CUDA-graph capture of sg_exp_map on a multi-mesh
batch (many meshes of uneven size, mesh-tagged queries, one persistent launch)."""
import numpy as np
import pytest

import meshgen
from tests import parity

pytestmark = pytest.mark.gpu


def _batch():
    import torch
    import paper_2603_15780_gb300 as sg
    wl = meshgen.workload(3, scale=0.001)
    meshes = [(parity.as_f32(X), F) for X, F in wl.meshes]
    mesh = sg.Mesh(meshes)
    q = wl.queries
    T = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    return sg, mesh, q, T(q.face, torch.int32), T(q.bary), T(q.v), T(q.mesh_id, torch.int32)


def test_graph_replay_matches_direct_call_and_tracks_inputs():
    import torch
    sg, mesh, q, face, bary, v, mid = _batch()
    ref = sg.exp_map(mesh, face, bary, v, mesh_id=mid, want_hash=False)
    from paper_2603_15780_gb300.autotune import GraphedExpMap
    g = GraphedExpMap(mesh, face, bary, v, mesh_id=mid)
    out = g.replay()
    torch.cuda.synchronize()
    for k in ("face", "status", "ncross"):
        assert torch.equal(out[k], ref[k]), k
    assert (out["pos"] - ref["pos"]).abs().max().item() < 1e-6
    # new inputs in the static buffers: the replay follows them
    g.inputs["v"].mul_(0.5)
    out = g.replay()
    ref2 = sg.exp_map(mesh, face, bary, v * 0.5, mesh_id=mid)
    torch.cuda.synchronize()
    assert torch.equal(out["face"], ref2["face"])
    assert (out["pos"] - ref2["pos"]).abs().max().item() < 1e-6


def test_autotuner_picks_a_valid_configuration():
    import torch
    sg, mesh, q, face, bary, v, mid = _batch()
    from paper_2603_15780_gb300 import autotune
    best, table = autotune.tune(mesh, face, bary, v, mesh_id=mid, reps=2)
    assert len(table) == len(autotune.candidates())
    assert min(ms for _, ms in table) > 0
    out = sg.exp_map(mesh, face, bary, v, mesh_id=mid, opts=best)
    ref = sg.exp_map(mesh, face, bary, v, mesh_id=mid)
    torch.cuda.synchronize()
    st = (out["status"] | ref["status"]).cpu().numpy()
    ok = (st & (sg.ST_NEAR_VERTEX | sg.ST_NEAR_EDGE)) == 0
    assert np.array_equal(out["face"].cpu().numpy()[ok], ref["face"].cpu().numpy()[ok])


@pytest.mark.parametrize("pick", ["tuned", "plain-4-per-thread", "persistent-32-per-thread"])
def test_tuned_and_swept_launches_match_the_oracle(pick):
    """The launch the autotuner picks on the multi-mesh batch, and the two ends of its
    queries-per-thread axis, at the full parity bar against the oracle mesh by mesh (face
    sequences bit-exact on unflagged queries, end points within 1e-5 of each mesh's diagonal)."""
    sg, mesh, q, face, bary, v, mid = _batch()
    from paper_2603_15780_gb300 import autotune
    if pick == "tuned":
        opts, _ = autotune.tune(mesh, face, bary, v, mesh_id=mid, reps=2)
    elif pick == "plain-4-per-thread":
        opts = sg.default_opts(kernel=sg.KERNEL_PLAIN, sort=0, fp64_escalate=0, queries_per_thread=4)
    else:
        opts = sg.default_opts(kernel=sg.KERNEL_PERSISTENT, queries_per_thread=32)
    gpu = parity.run_gpu(mesh, q, 0, mesh_id=q.mesh_id, opts=opts)
    wl = meshgen.workload(3, scale=0.001)
    for m in range(0, 64, 9):
        sel = np.nonzero(q.mesh_id == m)[0]
        X, F = wl.meshes[m]
        ref, _ = parity.run_oracle(parity.as_f32(X), F, q.take(sel), 0)
        sub = {k: val[sel] for k, val in gpu.items()}
        # flagged with probability ~1.5e-4 per crossing: bound 2e-4 per crossing plus three
        # binomial standard deviations of the mesh's sample (a few dozen queries on the small ones)
        p = 2e-4 * float(ref["ncross"].mean()) + 0.005
        parity.compare(sub, ref, meshgen.bbox_diag(X), 0, what=f"{pick} mesh {m}",
                       max_flagged=p + 3 * np.sqrt(p / len(sel)))


def test_graph_of_forward_and_both_backwards():
    """The forward, EP on a second stream and GFD with the vertex gradient, captured as one CUDA
    graph (memsets, the length orders, the task list and every counter inside) and replayed:
    the per-query gradients equal the eager calls' bit for bit, the vertex gradient to float
    rounding (atomic order), and a replay follows new values in the captured input buffers."""
    import torch
    import paper_2603_15780_gb300 as sg
    rng = np.random.default_rng(61)
    X, F = meshgen.icosphere(5, 0.003, rng)
    q = meshgen.sample_queries(X, F, 70000, rng, 0.1, 1.0, 0)  # above the length-order threshold
    mesh = sg.Mesh(parity.as_f32(X), F)
    T = lambda a, dt=torch.float32: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    face, bary, v, g = T(q.face, torch.int32), T(q.bary), T(q.v), T(q.g_pos)
    nq = len(q)
    ws = torch.empty(sg.workspace_size(mesh, nq), dtype=torch.uint8, device="cuda")
    bws = torch.empty(sg.backward_workspace_size(mesh, "gfd", nq, True), dtype=torch.uint8, device="cuda")
    ews = torch.empty(sg.backward_workspace_size(mesh, "ep", nq, False), dtype=torch.uint8, device="cuda")
    gV = torch.zeros(mesh.n_vertices, 3, device="cuda")
    side = torch.cuda.Stream()

    def step():
        cs = torch.cuda.current_stream()
        o = sg.exp_map(mesh, face, bary, v, workspace=ws)
        done = torch.cuda.Event()
        done.record(cs)
        side.wait_event(done)
        with torch.cuda.stream(side):
            ep = sg.exp_map_backward(mesh, "ep", face, bary, v, o["face"], o["bary"], o["dir"], o["status"], g,
                                     workspace=ews)
            ep_done = torch.cuda.Event()
            ep_done.record(side)
        gV.zero_()
        r = sg.exp_map_backward(mesh, "gfd", face, bary, v, o["face"], o["bary"], o["dir"], o["status"], g,
                                grad_V=gV, workspace=bws)
        cs.wait_event(ep_done)
        return o, ep, r

    eager = step()
    torch.cuda.synchronize()
    eager = [{k: t.clone() for k, t in d.items() if torch.is_tensor(t)} for d in eager]
    eager_gV = gV.clone()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(cap):
        step()
    torch.cuda.current_stream().wait_stream(cap)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        outs = step()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for ref, got in zip(eager, outs):
        for k in ("face", "bary", "pos", "status", "grad_v", "grad_p", "grad_bary"):
            if k in ref:
                assert torch.equal(ref[k], got[k]), k
    assert (gV - eager_gV).abs().max().item() <= 1e-5 * eager_gV.abs().max().item()
    # new upstream gradient in the captured buffer: the replay follows it
    g.mul_(-2.0)
    graph.replay()
    r2 = sg.exp_map_backward(mesh, "gfd", face, bary, v, outs[0]["face"], outs[0]["bary"], outs[0]["dir"],
                             outs[0]["status"], g)
    torch.cuda.synchronize()
    assert torch.equal(outs[2]["grad_v"], r2["grad_v"])
    assert torch.equal(outs[2]["grad_v"], -2.0 * eager[2]["grad_v"]) or \
        (outs[2]["grad_v"] + 2.0 * eager[2]["grad_v"]).abs().max().item() < 1e-5
