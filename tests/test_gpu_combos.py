"""GPU parity of feature combinations against the FP64 oracle: hole avoidance on a non-orientable
strip (flipped adjacencies in the boundary fans) and on a batch of a closed and a holey mesh,
the FP64 walk on a Klein bottle, and the trace on a Moebius strip."""
import numpy as np
import pytest

import meshgen
import oracle
from tests import parity

pytestmark = pytest.mark.gpu


def sg():
    import paper_2603_15780_gb300 as m
    return m


def test_hole_avoidance_on_a_moebius_strip():
    """The Moebius strip's boundary is one loop; its fans cross the flipped seam.  Hole avoidance
    with carried vectors against the oracle."""
    X, F = meshgen.mobius(96, 12)
    X32 = parity.as_f32(X)
    rng = np.random.default_rng(111)
    q = meshgen.sample_queries(X, F, 4000, rng, 0.1, 2.0, 1)
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, q, 1, boundary_mode=1)
    ref, _ = parity.run_oracle(X32, F, q, 1, boundary_mode=1)
    parity.compare(gpu, ref, meshgen.bbox_diag(X), 1, what="moebius hole", max_flagged=0.1)
    assert ((gpu["status"] & oracle.HOLE) != 0).mean() > 0.2
    assert ((gpu["status"] & 512) != 0).mean() > 0.02   # SG_ST_FLIPPED: some ends across the seam


def test_hole_avoidance_in_a_batch_of_closed_and_holey_meshes():
    rng = np.random.default_rng(112)
    Xa, Fa = meshgen.icosphere(3, 0.003, rng)
    Xb, Fb = meshgen.remove_faces(*meshgen.icosphere(4, 0.003, rng), 0.06, rng)
    qa = meshgen.sample_queries(Xa, Fa, 2000, rng, 0.1, 2.0, 1)
    qb = meshgen.sample_queries(Xb, Fb, 3000, rng, 0.1, 2.0, 1)
    mesh = sg().Mesh([(parity.as_f32(Xa), Fa), (parity.as_f32(Xb), Fb)])
    q = meshgen.Queries(np.concatenate([qa.face, qb.face]), np.concatenate([qa.bary, qb.bary]),
                        np.concatenate([qa.v, qb.v]), np.concatenate([qa.w, qb.w]),
                        np.concatenate([qa.g_pos, qb.g_pos]))
    mid = np.repeat(np.arange(2, dtype=np.int32), [2000, 3000])
    gpu = parity.run_gpu(mesh, q, 1, mesh_id=mid, boundary_mode=1)
    for k, (X, F, qq, sl) in enumerate(((Xa, Fa, qa, slice(0, 2000)), (Xb, Fb, qb, slice(2000, 5000)))):
        ref, _ = parity.run_oracle(parity.as_f32(X), F, qq, 1, boundary_mode=1)
        parity.compare({key: val[sl] for key, val in gpu.items()}, ref, meshgen.bbox_diag(X), 1,
                       what=f"batch mesh {k}", max_flagged=0.1)
    assert not np.any(gpu["status"][:2000] & oracle.HOLE)
    assert ((gpu["status"][2000:] & oracle.HOLE) != 0).mean() > 0.2


@pytest.mark.parametrize("prec", [64, 48, 40], ids=["fp64", "double-float", "mixed"])
def test_fp64_walk_on_a_klein_bottle(prec):
    X, F = meshgen.klein_bottle(64, 32)
    X32 = parity.as_f32(X)
    rng = np.random.default_rng(113)
    q = meshgen.sample_queries(X, F, 4000, rng, 0.5, 4.0, 2)
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, q, 2, precision=prec)
    ref, _ = parity.run_oracle(X32, F, q, 2)
    parity.compare(gpu, ref, meshgen.bbox_diag(X), 2, what=f"klein precision {prec}", pos_tol=1e-6, dir_tol=1e-5)
    assert ((gpu["status"] & 512) != 0).mean() > 0.05


def test_trace_on_a_moebius_strip():
    import torch
    X, F = meshgen.mobius(96, 12)
    X32 = parity.as_f32(X)
    rng = np.random.default_rng(114)
    q = meshgen.sample_queries(X, F, 3000, rng, 0.1, 2.0, 0)
    mesh = sg().Mesh(X32, F)
    f32 = parity.as_f32
    out = sg().exp_map_trace(mesh, q.face, f32(q.bary), f32(q.v), path_cap=128, want_hash=True)
    torch.cuda.synchronize()
    tr = {k: v.cpu().numpy() for k, v in out.items()}
    tr["status"] = tr["status"].astype(np.uint32)
    ref, _ = parity.run_oracle(X32, F, q, 0, path_cap=128)
    ok = ((tr["status"] | ref["status"]) & parity.FLAGS) == 0
    assert ok.mean() > 0.9
    assert np.array_equal(tr["path_len"][ok], ref["path_len"][ok])
    diag = meshgen.bbox_diag(X)
    for i in np.nonzero(ok)[0]:
        n = min(int(tr["path_len"][i]), 128)
        assert np.array_equal(tr["path_face"][i, :n], ref["path"][i, :n])
        assert np.abs(tr["path_pt"][i, :n] - ref["path_pt"][i, :n]).max() <= 1e-5 * diag
