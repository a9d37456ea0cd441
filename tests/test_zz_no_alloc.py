"""GPU test of sg_exp_map_noalloc, the exponential-map entry point for callers that cannot
allocate device memory at call time (code whose device memory is owned by another
framework's pool, or loops where a cudaMalloc/cudaFree would synchronise the device).

It is called here through the C ABI and must reproduce sg_exp_map's results on two
calls in a row (the second call finds the first call's leftovers in the shared scratch
array), and reject a batch too large for its fixed scratch without launching anything.
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


def test_noalloc_matches_exp_map_on_two_calls():
    import torch
    import paper_2603_15780_gb300 as sg
    wl = meshgen.workload(0)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg.Mesh(X32, F)
    q = wl.queries
    diag = meshgen.bbox_diag(X)
    batches = [np.arange(len(q)), np.arange(len(q))[::-1][:3001].copy()]   # second call: other size/order
    for call, idx in enumerate(batches):
        face = torch.tensor(q.face[idx], device="cuda")
        bary = torch.tensor(parity.as_f32(q.bary[idx]), device="cuda")
        v = torch.tensor(parity.as_f32(q.v[idx]), device="cuda")
        w = torch.tensor(parity.as_f32(q.w[idx]), device="cuda")
        ref = sg.exp_map(mesh, face, bary, v, w, want_hash=True)
        opts = sg.default_opts()
        rc, out = _noalloc(sg, mesh, face, bary, v, w, 1, opts, torch)
        torch.cuda.synchronize()
        assert rc == 0, f"call {call}: status {rc}"
        for k in ("face", "status", "ncross", "hash"):
            assert torch.equal(out[k], ref[k]), f"call {call}: {k} differs"
        for k in ("pos", "bary", "dir", "w"):
            err = (out[k] - ref[k]).abs().max().item()
            assert err <= 1e-5 * diag, f"call {call}: {k} differs by {err}"


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
    # without the sort the scratch is a single counter: the same batch is accepted
    opts0 = sg.default_opts(sort=0)
    rc, out = _noalloc(sg, mesh, face, bary, v, None, 0, opts0, torch)
    torch.cuda.synchronize()
    assert rc == 0
    assert torch.equal(out["face"], face)
