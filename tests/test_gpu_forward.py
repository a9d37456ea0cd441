"""GPU parity of the forward exponential map (sg_exp_map) against the FP64 oracle.

Every test calls the CUDA library through its C ABI (ctypes binding) and compares with
the oracle on identical float32 inputs; tolerances are stated in tests/parity.py.
"""
import math
import os

import numpy as np
import pytest

import meshgen
import oracle
from tests import parity

pytestmark = pytest.mark.gpu


def sg():
    import paper_2603_15780_gb300 as m
    return m


KERNELS = [
    dict(kernel=1),                                  # plain: one thread per query, FP32
    dict(kernel=2, sort=1, fp64_escalate=1),         # persistent, sorted, FP64 classification
    dict(kernel=2, sort=0, fp64_escalate=0, block=128),
    dict(kernel=2, sort=2, fp64_escalate=1),         # persistent, longest walks first
]


@pytest.mark.parametrize("kw", KERNELS, ids=["plain", "persistent-sorted-fp64", "persistent-unsorted",
                                             "persistent-length-order"])
def test_icosphere_s3_full_workload(kw):
    """Workload 0 in full: icosphere s3, 4096 queries, one carried vector."""
    wl = meshgen.workload(0)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, wl.queries, 1, **kw)
    ref, om = parity.run_oracle(X32, F, wl.queries, 1)
    r = parity.compare(gpu, ref, meshgen.bbox_diag(X), 1, what=str(kw))
    parity.check_flag_semantics(gpu, ref, om.lref)
    assert r["flagged"] < 0.02


def test_flat_mesh_is_straight():
    """Flat jittered grid: Exp = p + v (Sec. 4, theta = 2pi everywhere)."""
    rng = np.random.default_rng(21)
    X, F = meshgen.flat_grid(41, rng, jitter=0.3)
    q = meshgen.sample_queries(X, F, 5000, rng, 0.0, 0.4, 2)
    mesh = sg().Mesh(parity.as_f32(X), F)
    gpu = parity.run_gpu(mesh, q, 2)
    ok = (gpu["status"] & oracle.BOUNDARY) == 0
    p0 = (parity.as_f32(q.bary).astype(np.float64)[:, :, None] * parity.as_f32(X)[F[q.face]]).sum(1)
    expect = p0 + parity.as_f32(q.v)
    assert np.abs(gpu["pos"] - expect)[ok].max() < 2e-6
    assert np.abs(gpu["w"] - parity.as_f32(q.w))[ok].max() < 2e-6


def test_polycube_face_sequences_exact():
    """Polycube with small-integer coordinates: GPU face sequences equal the exact rational
    walker (bit-exact hashes), end points to FP32 accuracy."""
    from fractions import Fraction
    from tests.exact_walker import Polycube
    X, F = meshgen.polycube([(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (2, 1, 1)])
    pc = Polycube(X, F)
    rng = np.random.default_rng(22)
    rows = []
    for _ in range(400):
        f = int(rng.integers(len(F)))
        r = rng.integers(1, 15, size=3)
        bary = [Fraction(int(x), int(r.sum())) for x in r]
        ax = [c for c in range(3) if c != pc.axis[f]]
        d = [0, 0, 0]
        d[ax[0]] = int(rng.integers(-9, 10)); d[ax[1]] = int(rng.integers(-9, 10))
        if d[ax[0]] == 0 and d[ax[1]] == 0:
            d[ax[0]] = 1
        t = Fraction(int(rng.integers(1, 64)), 8)
        ex = pc.walk(f, bary, d, t)
        if ex is None:
            continue
        rows.append((f, [float(b) for b in bary], [float(x * t) for x in d], ex))
    face = np.array([r[0] for r in rows], np.int32)
    bary = np.array([r[1] for r in rows])
    v = np.array([r[2] for r in rows])
    q = meshgen.Queries(face, bary, v, np.zeros((len(rows), 0, 3)), np.zeros((len(rows), 3)))
    mesh = sg().Mesh(parity.as_f32(X), F)
    gpu = parity.run_gpu(mesh, q, 0)
    n = 0
    for i, (_, _, _, (faces, pend)) in enumerate(rows):
        if gpu["status"][i] & parity.FLAGS:
            continue
        assert gpu["hash"][i] == oracle.fnv_hash(faces), i
        assert np.abs(gpu["pos"][i] - np.array([float(c) for c in pend])).max() < 1e-5 * meshgen.bbox_diag(X)
        n += 1
    assert n > 250


def test_cube_corner_worked_examples():
    """The hand-worked cube examples (tests/golden), including two straightest vertex hits."""
    X, F = meshgen.polycube([(0, 0, 0)])
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "cube_worked_examples.txt"))
    from tests.test_oracle_pins import locate
    face, bary, v = [], [], []
    for r in rows:
        f, b = locate(X, F, r[0:3])
        face.append(f); bary.append(b); v.append(r[3:6] / np.linalg.norm(r[3:6]) * r[6])
    q = meshgen.Queries(np.array(face, np.int32), np.array(bary), np.array(v), np.zeros((len(face), 0, 3)),
                        np.zeros((len(face), 3)))
    mesh = sg().Mesh(parity.as_f32(X), F)
    gpu = parity.run_gpu(mesh, q, 0)
    assert np.abs(gpu["pos"] - rows[:, 7:10]).max() < 2e-6, gpu["pos"]
    assert np.all((gpu["status"][1:] & oracle.VERTEX_HIT) != 0)


@pytest.mark.parametrize("theta", [1.3 * math.pi, 2.4 * math.pi])
def test_cone_apex_straightest_rule(theta):
    """Rays aimed exactly at a cone apex leave at theta/2 (GPU vs FP64 oracle)."""
    n = 9
    X, F = meshgen.cone_fan(n, theta)
    X32 = parity.as_f32(X)
    rng = np.random.default_rng(23)
    face, bary, v = [], [], []
    for _ in range(64):
        f0 = int(rng.integers(n))
        u = X32[F[f0][1]].astype(np.float64); w = X32[F[f0][2]].astype(np.float64)
        b1, b2 = rng.uniform(0.05, 0.5), rng.uniform(0.05, 0.4)
        b = np.array([1 - b1 - b2, b1, b2])
        p = b1 * u + b2 * w
        rho = np.linalg.norm(p)
        face.append(f0); bary.append(b); v.append(-p / rho * (rho + rng.uniform(0.05, 0.3)))
    q = meshgen.Queries(np.array(face, np.int32), np.array(bary), np.array(v), np.zeros((64, 0, 3)),
                        np.zeros((64, 3)))
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, q, 0)
    # the float32-rounded rays miss the apex by ~1e-8: give the oracle the GPU's snap radius
    ref, _ = parity.run_oracle(X32, F, q, 0, tau_snap=1e-6)
    hit = (ref["status"] & oracle.VERTEX_HIT) != 0
    assert hit.mean() > 0.9
    assert np.all((gpu["status"][hit] & oracle.VERTEX_HIT) != 0)
    # outgoing rays near an edge are flagged on either side; compare the rest
    ok = hit & (((gpu["status"] | ref["status"]) & parity.FLAGS) == 0)
    assert ok.sum() > 40
    assert np.abs(gpu["pos"] - ref["pos"])[ok].max() < 2e-5


def test_vertex_on_a_fold_matches_development():
    """Rays aimed exactly at the vertices of a fold line (angle sum 2pi on a folded sheet): the
    GPU walk and its carried vector equal the development's straight line and unchanged vector,
    refolded, whether FP32 snaps the vertex or passes beside it; against the FP64 oracle the
    walks snapped on both sides agree in face sequence and end point."""
    from tests import test_oracle_pins as pins
    nx, ny, c = 9, 7, 4
    X, F, P = meshgen.folded_strip(nx, ny, 3.0, 2.0, [(c, 0.9)])
    X32 = parity.as_f32(X)
    rng = np.random.default_rng(62)
    qs = pins.fold_vertex_queries(X, F, P, c, nx, ny, 300, rng)
    n = len(qs)
    q = meshgen.Queries(np.array([t[0] for t in qs], np.int32), np.array([t[1] for t in qs]),
                        np.array([t[2] for t in qs]), np.array([[t[3]] for t in qs]), np.zeros((n, 3)))
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, q, 1)
    diag = meshgen.bbox_diag(X)
    checked = 0
    for i, (f, b, v3, w3, p0, d, L, wf) in enumerate(qs):
        if gpu["status"][i] & (oracle.BOUNDARY | oracle.NEAR_EDGE):
            continue
        g, bg = pins.locate(P, F, p0 + L * d, tol=1e-9)
        A, B, C = P[F[g]]
        a, bb, cc = X[F[g]]
        M2 = np.stack([B - A, C - A], 1)
        to3 = lambda u: (lambda k: k[0] * (bb - a) + k[1] * (cc - a))(np.linalg.lstsq(M2, u, rcond=None)[0])
        assert gpu["face"][i] == g, i
        assert np.linalg.norm(gpu["pos"][i] - bg @ X[F[g]]) <= 1e-5 * diag, i
        assert np.abs(gpu["dir"][i] - to3(d)).max() <= 2e-4, i
        assert np.abs(gpu["w"][i, 0] - to3(wf)).max() <= 2e-4, i
        checked += 1
    assert checked > n // 2
    # the oracle snaps at the GPU's radius: the float32 rays miss the vertex by ~1e-7 l_ref
    ref, _ = parity.run_oracle(X32, F, q, 1, tau_snap=1e-6)
    both = ((gpu["status"] & ref["status"]) & oracle.VERTEX_HIT) != 0
    assert both.mean() > 0.5
    ok = both & (((gpu["status"] | ref["status"]) & parity.FLAGS) == 0)
    assert np.array_equal(gpu["hash"][ok], ref["hash"][ok]) and np.array_equal(gpu["face"][ok], ref["face"][ok])
    assert np.linalg.norm(gpu["pos"] - ref["pos"], axis=1)[ok].max() <= 1e-5 * diag


def test_torus_subset_two_carried_vectors():
    """Workload-1 mesh (noisy torus 262,144 faces), 50k of its queries, 2 carried vectors."""
    wl = meshgen.workload(1, scale=50000 / 4194304)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, wl.queries, 2)
    ref, om = parity.run_oracle(X32, F, wl.queries, 2)
    r = parity.compare(gpu, ref, meshgen.bbox_diag(X), 2, what="torus")
    parity.check_flag_semantics(gpu, ref, om.lref)
    print("torus", r)


def test_heightfield_slivers_and_boundary():
    """Workload-4 mesh (1449^2 heightfield, 10% sliver vertices, ~1.8k crossings per walk) at the
    full parity bar with the default options: face sequences bit-exact on every query neither side
    flags, end points within 1e-5 of the bbox diagonal.  The FP32 walk's accumulated direction
    error passes vertices on the wrong side beyond ~256 crossings, so the automatic precision walks
    those queries in the mixed walk (SG_ST_MIXED); the escalated and flagged fractions are printed
    and bounded, and the boundary stops must agree."""
    wl = meshgen.workload(4, scale=20000 / 16777216)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, wl.queries, 0)
    ref, _ = parity.run_oracle(X32, F, wl.queries, 0)
    diag = meshgen.bbox_diag(X)
    r = parity.compare(gpu, ref, diag, 0, max_flagged=0.25, what="heightfield, automatic precision")
    mixed = (gpu["status"] & 4096) != 0
    nc = ref["ncross"]
    stats = dict(r, escalated=float(mixed.mean()), mean_ncross=float(nc.mean()),
                 boundary=float(((ref["status"] & oracle.BOUNDARY) != 0).mean()),
                 fp32_max_ncross=int(gpu["ncross"][~mixed].max()))
    print("heightfield", stats)
    assert ((ref["status"] & oracle.BOUNDARY) != 0).mean() > 0.3
    # every walk the FP32 walk kept stayed below its crossing budget, and the long ones escalated
    assert gpu["ncross"][~mixed].max() < 256
    assert mixed[gpu["ncross"] >= 256].all()
    assert 0.5 < mixed.mean() < 1.0


def test_heightfield_fp32_walk_diverges_beyond_its_range():
    """The same sample with the plain FP32 walk (precision 32): below 256 crossings its face
    sequences are bit-exact on unflagged queries; beyond, they differ on a few percent -- the
    measurement that sets the automatic precision's crossing budget."""
    wl = meshgen.workload(4, scale=20000 / 16777216)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, wl.queries, 0, precision=32)
    ref, _ = parity.run_oracle(X32, F, wl.queries, 0)
    flagged = ((gpu["status"] | ref["status"]) & parity.FLAGS) != 0
    same = (gpu["hash"] == ref["hash"]) & (gpu["face"] == ref["face"])
    nc = ref["ncross"]
    short = (nc < 256) & ~flagged
    long_ = (nc >= 1000) & ~flagged
    print("fp32 heightfield: unflagged mismatches below 256 crossings", int((~same[short]).sum()), "of", int(short.sum()),
          "; from 1000 crossings", int((~same[long_]).sum()), "of", int(long_.sum()))
    assert same[short].all()
    assert (~same[long_]).mean() > 0.02


def test_multi_mesh_batch():
    """Workload 3 (64 uneven meshes in one object, mesh-tagged queries), 1% of the queries."""
    wl = meshgen.workload(3, scale=0.002)
    mesh = sg().Mesh([(parity.as_f32(X), F) for X, F in wl.meshes])
    q = wl.queries
    gpu = parity.run_gpu(mesh, q, 0, mesh_id=q.mesh_id)
    # A walk is flagged when it passes within tau_near l_ref = 1e-4 l_ref of a vertex, which
    # happens with probability about 1.5e-4 per crossing on these meshes: each mesh's flagged
    # fraction is bounded by 2e-4 times its mean crossing count (plus 1% for small samples).
    for m in (0, 1, 2, 17, 40, 63):
        sel = np.nonzero(q.mesh_id == m)[0]
        X, F = wl.meshes[m]
        X32 = parity.as_f32(X)
        ref, _ = parity.run_oracle(X32, F, q.take(sel), 0)
        sub = {k: v[sel] for k, v in gpu.items()}
        bound = 2e-4 * float(ref["ncross"].mean()) + 0.01
        r = parity.compare(sub, ref, meshgen.bbox_diag(X), 0, what=f"mesh {m}", max_flagged=bound)
        print(f"mesh {m}: {len(sel)} queries, mean crossings {ref['ncross'].mean():.0f}, flagged {r['flagged']:.4f} "
              f"(bound {bound:.4f}), mixed walk {((sub['status'] & 4096) != 0).mean():.3f}")


def test_edge_cases():
    """Empty batch, invalid queries, zero length, explicit lengths, starts on edges and
    vertices, MAX_STEPS."""
    import torch
    X, F = meshgen.icosphere(2)
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    out = sg().exp_map(mesh, np.zeros(0, np.int32), np.zeros((0, 3), np.float32), np.zeros((0, 3), np.float32))
    assert out["pos"].shape == (0, 3)
    rng = np.random.default_rng(24)
    q = meshgen.sample_queries(X, F, 64, rng, 0.1, 2.0, 0)
    q.face[0] = len(F) + 5               # invalid face
    q.bary[1] = [0.5, 0.5, 0.5]          # barycentrics do not sum to 1
    q.v[2] = 0.0                         # zero vector, zero length
    q.bary[3] = [0.0, 0.4, 0.6]          # on an edge
    q.bary[4] = [1.0, 0.0, 0.0]          # on a vertex, direction into the face
    a, b, c = X32[F[q.face[4]]].astype(np.float64)
    q.v[4] = ((b + c) / 2 - a) / np.linalg.norm((b + c) / 2 - a) * 0.7
    q.bary[5] = [1.0, 0.0, 0.0]          # on a vertex, direction out of the face
    a5, b5, c5 = X32[F[q.face[5]]].astype(np.float64)
    q.v[5] = -((b5 + c5) / 2 - a5) / np.linalg.norm((b5 + c5) / 2 - a5) * 0.7
    gpu = parity.run_gpu(mesh, q, 0)
    ref, _ = parity.run_oracle(X32, F, q, 0)
    assert gpu["status"][0] & oracle.INVALID and ref["status"][0] & oracle.INVALID
    assert gpu["status"][1] & oracle.INVALID and ref["status"][1] & oracle.INVALID
    assert not gpu["status"][2] & oracle.INVALID
    assert gpu["face"][2] == q.face[2]
    assert gpu["status"][3] & oracle.START_ON_EDGE and ref["status"][3] & oracle.START_ON_EDGE
    assert not gpu["status"][4] & oracle.INVALID and not ref["status"][4] & oracle.INVALID
    assert gpu["status"][5] & oracle.INVALID and ref["status"][5] & oracle.INVALID
    keep = np.ones(64, bool); keep[[0, 1, 5]] = False
    sub = {k: v[keep] for k, v in gpu.items()}
    subr = {k: v[keep] for k, v in ref.items()}
    parity.compare(sub, subr, meshgen.bbox_diag(X), 0, what="edge cases", max_flagged=0.1)
    # explicit lengths
    L = rng.uniform(0.0, 1.5, 64).astype(np.float32)
    q2 = meshgen.sample_queries(X, F, 64, rng, 0.1, 2.0, 0)
    gpu = parity.run_gpu(mesh, q2, 0, length=L)
    ref, _ = parity.run_oracle(X32, F, q2, 0, length=L)
    parity.compare(gpu, ref, meshgen.bbox_diag(X), 0, what="explicit length", max_flagged=0.1)
    # MAX_STEPS
    gpu = parity.run_gpu(mesh, q2, 0, max_steps=3)
    ref, _ = parity.run_oracle(X32, F, q2, 0, max_steps=3)
    long_ = (ref["status"] & oracle.MAX_STEPS) != 0
    assert long_.sum() > 10
    assert np.array_equal((gpu["status"] & oracle.MAX_STEPS) != 0, long_)
    assert np.array_equal(gpu["face"], ref["face"])


def test_ragged_sizes_and_workspace_reuse():
    """Batch sizes that leave ragged warps/blocks, through a caller-provided workspace."""
    import torch
    wl = meshgen.workload(0)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    ws = torch.empty(sg().workspace_size(mesh, 4096), dtype=torch.uint8, device="cuda")
    ref, _ = parity.run_oracle(X32, F, wl.queries, 0)
    for n in (1, 31, 33, 257, 1000, 4095):
        q = wl.queries.take(np.arange(n))
        gpu = parity.run_gpu(mesh, q, 0, workspace=ws)
        r = {k: v[:n] for k, v in ref.items()}
        parity.compare(gpu, r, meshgen.bbox_diag(X), 0, what=f"n={n}", max_flagged=0.1)


def test_full_size_torus_sampled():
    """Workload 1 at full size (4,194,304 queries, 2 carried vectors) in the launch
    configuration the benchmark uses; 20k sampled outputs checked against the oracle."""
    wl = meshgen.workload(1)
    X, F = wl.single
    X32 = parity.as_f32(X)
    mesh = sg().Mesh(X32, F)
    gpu = parity.run_gpu(mesh, wl.queries, 2)
    idx = np.random.default_rng(25).choice(len(wl.queries), 20000, replace=False)
    ref, _ = parity.run_oracle(X32, F, wl.queries.take(idx), 2)
    sub = {k: v[idx] for k, v in gpu.items()}
    r = parity.compare(sub, ref, meshgen.bbox_diag(X), 2, what="torus full")
    print("torus full", r)
