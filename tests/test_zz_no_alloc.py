"""GPU test of sg_exp_map_noalloc, the exponential-map entry point for callers that cannot
allocate device memory at call time (code whose device memory is owned by another
framework's pool, or loops where a cudaMalloc/cudaFree would synchronise the device).

It is called here through the C ABI and must reproduce sg_exp_map's results on calls in a
row on the persistent kernel (each call finds the previous call's leftovers in the shared
scratch array: queue counter, sort histogram, permutation), run the double-float walk and
the automatic precision (whose escalation list lives in the same array) on the double-float
records built with the mesh, and reject a batch too large for its fixed scratch without launching anything.
This file is collected last so a failure here cannot hide the other tests' results.
"""
import ctypes as C

import numpy as np
import pytest

import meshgen
from tests import parity

pytestmark = pytest.mark.gpu


def _noalloc(sg, mesh, face, bary, v, w, nw, opts, torch):
    nq = face.numel()
    dev = face.device
    out = {"face": torch.empty(nq, dtype=torch.int32, device=dev), "bary": torch.empty(nq, 3, device=dev),
           "pos": torch.empty(nq, 3, device=dev), "dir": torch.empty(nq, 3, device=dev),
           "w": torch.empty(nq, max(nw, 1), 3, device=dev), "status": torch.empty(nq, dtype=torch.int32, device=dev),
           "ncross": torch.empty(nq, dtype=torch.int32, device=dev),
           "hash": torch.empty(nq, dtype=torch.int64, device=dev)}
    P = lambda t: C.c_void_p(t.data_ptr())
    stream = torch.cuda.current_stream()
    rc = sg.lib().sg_exp_map_noalloc(mesh.handle, nq, None, P(face), P(bary), P(v), None, nw,
                                     P(w) if nw else None, P(out["face"]), P(out["bary"]), P(out["pos"]),
                                     P(out["dir"]), P(out["w"]) if nw else None, P(out["status"]),
                                     P(out["ncross"]), P(out["hash"]), C.byref(opts), C.c_void_p(stream.cuda_stream))
    return rc, out


def _check_same(out, ref, diag, what):
    for k in ("face", "status", "ncross", "hash"):
        assert torch_equal(out[k], ref[k]), f"{what}: {k} differs"
    for k in ("pos", "bary", "dir", "w"):
        if k in ref and ref[k] is not None and k in out:
            err = (out[k][..., :ref[k].shape[-1]] - ref[k]).abs().max().item()
            assert err <= 1e-5 * diag, f"{what}: {k} differs by {err}"


def torch_equal(a, b):
    import torch
    return torch.equal(a, b)


def test_noalloc_matches_exp_map_on_two_calls():
    """Two calls in a row on the persistent kernel, whose work queue lives in the shared scratch
    array: the second call, of another size and order, starts from the first call's leftovers
    (counter, histogram, permutation).  Each call is checked against sg_exp_map with the same
    options, bit for bit on the discrete outputs."""
    import torch
    import paper_2603_15780_gb300 as sg
    X, F = meshgen.icosphere(3)
    X32 = parity.as_f32(X)
    mesh = sg.Mesh(X32, F)
    rng = np.random.default_rng(77)
    q = meshgen.sample_queries(X, F, 100000, rng, 0.0, 3.0, 1)
    diag = meshgen.bbox_diag(X)
    # (queries, options): a length-ordered batch of 100,000, then a start-face sorted batch of
    # 70,001 in reverse order, then an unsorted one of 65,536 -- all above the size where the
    # automatic choice would skip the queue
    calls = [(np.arange(100000), dict(kernel=2, sort=2)),
             (np.arange(100000)[::-1][:70001].copy(), dict(kernel=2, sort=1)),
             (np.arange(65536) * 3 % 100000, dict(kernel=2, sort=0))]
    for call, (idx, kw) in enumerate(calls):
        face = torch.tensor(q.face[idx], device="cuda")
        bary = torch.tensor(parity.as_f32(q.bary[idx]), device="cuda")
        v = torch.tensor(parity.as_f32(q.v[idx]), device="cuda")
        w = torch.tensor(parity.as_f32(q.w[idx, :1]), device="cuda")
        ref = sg.exp_map(mesh, face, bary, v, w, want_hash=True, **kw)
        rc, out = _noalloc(sg, mesh, face, bary, v, w, 1, sg.default_opts(**kw), torch)
        torch.cuda.synchronize()
        assert rc == 0, f"call {call}: status {rc}"
        _check_same(out, ref, diag, f"call {call} {kw}")


def test_noalloc_wider_precisions():
    """The double-float walk (precision 48) and the automatic precision walk on double-float
    records that sg_mesh_create builds with the mesh, so the allocation-free entry point runs
    them without allocating; each call matches sg_exp_map.  The automatic precision's batch
    includes walks beyond the FP32 walk's crossing budget, which go through the escalation list
    in the shared array."""
    import torch
    import paper_2603_15780_gb300 as sg
    X, F = meshgen.icosphere(4)
    mesh = sg.Mesh(parity.as_f32(X), F)
    rng = np.random.default_rng(78)
    q = meshgen.sample_queries(X, F, 70000, rng, 0.0, 12.0, 1)
    face = torch.tensor(q.face, device="cuda")
    bary = torch.tensor(parity.as_f32(q.bary), device="cuda")
    v = torch.tensor(parity.as_f32(q.v), device="cuda")
    w = torch.tensor(parity.as_f32(q.w[:, :1]), device="cuda")
    for kw in (dict(kernel=2, precision=48), dict(precision=0), dict(precision=0, sort=1)):
        ref = sg.exp_map(mesh, face, bary, v, w, want_hash=True, **kw)
        rc, out = _noalloc(sg, mesh, face, bary, v, w, 1, sg.default_opts(**kw), torch)
        torch.cuda.synchronize()
        assert rc == 0, f"{kw}: status {rc}"
        if kw["precision"] == 0:
            assert ((out["status"] & 4096) != 0).any(), "no walk escalated"
        _check_same(out, ref, meshgen.bbox_diag(X), str(kw))


def test_noalloc_rejects_batches_beyond_its_scratch():
    import torch
    import paper_2603_15780_gb300 as sg
    X, F = meshgen.icosphere(2)
    mesh = sg.Mesh(parity.as_f32(X), F)
    nq = 9 * 1024 * 1024          # sorted layout needs > 32 MiB of scratch
    opts = sg.default_opts(sort=1)
    assert sg.workspace_size(mesh, nq, opts) > (32 << 20)
    face = torch.zeros(nq, dtype=torch.int32, device="cuda")
    bary = torch.full((nq, 3), 1.0 / 3.0, device="cuda")
    v = torch.zeros(nq, 3, device="cuda")
    rc, _ = _noalloc(sg, mesh, face, bary, v, None, 0, opts, torch)
    torch.cuda.synchronize()
    assert rc == 5                # SG_ERR_OOM: nothing launched
    # without the sort (and without the automatic precision's escalation list) the scratch is a
    # single counter: the same batch is accepted
    opts0 = sg.default_opts(sort=0, precision=32)
    rc, out = _noalloc(sg, mesh, face, bary, v, None, 0, opts0, torch)
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.equal(out["face"], face)
