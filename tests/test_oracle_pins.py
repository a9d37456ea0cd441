"""Pins of the FP64 oracle against facts fixed by the paper and by geometry, not by itself.

Each test names the passage (section / algorithm / equation) whose content it pins.
None of these tests touches the CUDA library.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import meshgen
import oracle
from tests.exact_walker import Polycube

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def start_points(X, F, face, bary):
    return (np.asarray(bary)[:, :, None] * X[F[face]]).sum(1)


def locate(X, F, p, tol=1e-12):
    """(face, bary) of a 3-D point lying on the mesh (brute force over faces)."""
    for f in range(len(F)):
        a, b, c = X[F[f]]
        n = np.cross(b - a, c - a)
        if abs(np.dot(p - a, n)) > tol * np.linalg.norm(n):
            continue
        M = np.stack([b - a, c - a], 1)
        uv, *_ = np.linalg.lstsq(M, p - a, rcond=None)
        bb = np.array([1 - uv.sum(), uv[0], uv[1]])
        if bb.min() > 1e-9:
            return f, bb
    raise AssertionError("point not strictly inside any face")


# --------------------------------------------------------------------------- Sec. 4: flat
def test_flat_mesh_endpoint_is_p_plus_v():
    """Sec. 4: on a face (and across coplanar edges) theta = 2pi, so a straightest geodesic
    is a straight line: Exp_p(v) = p + v, transported vectors are unchanged."""
    rng = np.random.default_rng(1)
    X, F = meshgen.flat_grid(17, rng, jitter=0.3)
    m = oracle.Mesh(X, F)
    q = meshgen.sample_queries(X, F, 3000, rng, 0.0, 0.35, 2)
    out = oracle.exp_map(m, q.face, q.bary, q.v, q.w)
    ok = (out["status"] & oracle.BOUNDARY) == 0
    assert ok.mean() > 0.6
    p0 = start_points(X, F, q.face, q.bary)
    assert np.abs(out["pos"] - (p0 + q.v))[ok].max() < 1e-12
    d = q.v / np.linalg.norm(q.v, axis=1, keepdims=True)
    assert np.abs(out["dir"] - d)[ok].max() < 1e-12
    assert np.abs(out["w"] - q.w)[ok].max() < 1e-12
    # the walk really crossed many edges
    assert out["ncross"][ok].mean() > 3


# --------------------------------------------------------------------------- developable folds
@pytest.mark.parametrize("folds", [[(4, 0.7)], [(3, -1.1), (7, 0.5), (10, 1.4)]])
def test_folded_strip_matches_development(folds):
    """Alg. transport_over_edge: rotating about the shared edge by the dihedral angle is the
    unfolding isometry; on a developable fold the geodesic is the straight line of the
    development, refolded."""
    rng = np.random.default_rng(2)
    X, F, P = meshgen.folded_strip(13, 7, 3.0, 1.5, folds)
    m = oracle.Mesh(X, F)
    q = meshgen.sample_queries(X, F, 600, rng, 0.0, 2.0, 1)
    out = oracle.exp_map(m, q.face, q.bary, q.v, q.w)
    n_checked = 0
    for i in range(len(q)):
        if out["status"][i] & (oracle.BOUNDARY | oracle.NEAR_VERTEX | oracle.NEAR_EDGE):
            continue
        f = q.face[i]
        a, b, c = X[F[f]]
        A, B, Cc = P[F[f]]
        # express v in the 3-D face basis, map to the flat face basis (same barycentric map)
        M3 = np.stack([b - a, c - a], 1)
        coef, *_ = np.linalg.lstsq(M3, q.v[i], rcond=None)
        vflat = coef[0] * (B - A) + coef[1] * (Cc - A)
        pflat = q.bary[i] @ P[F[f]] + vflat
        g, bb = locate(P, F, pflat, tol=1e-9)
        expect = bb @ X[F[g]]
        assert g == out["face"][i]
        assert np.linalg.norm(out["pos"][i] - expect) < 1e-11
        n_checked += 1
    assert n_checked > 150


def fold_vertex_queries(X, F, P, fold_col, nx, ny, n, rng):
    """Rays of a folded strip aimed exactly at the interior vertices of the fold line
    `fold_col`, from random points left of it, with a carried vector at a random angle.  Returns
    per query the start face and barycentrics, the 3-D v and w, and the development's start
    point, direction and length (in the flat strip P)."""
    out = []
    xs, ys = np.unique(P[:, 0]), np.unique(P[:, 1])
    xc = xs[fold_col]
    for _ in range(n):
        V = np.array([xc, ys[int(rng.integers(1, ny - 1))], 0.0])
        # a start point strictly inside a face left of the fold line
        while True:
            p0 = np.array([rng.uniform(0.05, xc - 0.05), rng.uniform(0.05, ys[-1] - 0.05), 0.0])
            try:
                f, b = locate(P, F, p0, tol=1e-12)
            except AssertionError:
                continue
            break
        d = V - p0
        dist = np.linalg.norm(d)
        d /= dist
        L = dist + rng.uniform(0.1, 0.6)
        beta = rng.uniform(-math.pi, math.pi)
        wf = math.cos(beta) * d + math.sin(beta) * np.array([-d[1], d[0], 0.0])
        # the face's flat -> 3-D isometry, written through its edge vectors
        A, B, C = P[F[f]]
        a, bb, c = X[F[f]]
        M2 = np.stack([B - A, C - A], 1)
        to3 = lambda u: (lambda k: k[0] * (bb - a) + k[1] * (c - a))(np.linalg.lstsq(M2, u, rcond=None)[0])
        out.append((f, b, to3(d) * L, to3(wf), p0, d, L, wf))
    return out


@pytest.mark.parametrize("angle", [0.9, -1.7])
def test_vertex_on_a_fold_matches_development(angle):
    """Alg. transport_over_vertex at a vertex of angle sum 2pi on a folded (developable) sheet:
    the straightest ray through it is the development's straight line, refolded, and the carried
    vectors are the development's unchanged vectors, refolded -- whatever rule transports them
    at vertices of other angle sums.  Rays are aimed exactly at the vertices of the fold line."""
    nx, ny, c = 9, 7, 4
    X, F, P = meshgen.folded_strip(nx, ny, 3.0, 2.0, [(c, angle)])
    m = oracle.Mesh(X, F)
    th, bnd = m.theta()
    xs = np.unique(P[:, 0])
    on_fold = np.where((np.abs(P[:, 0] - xs[c]) < 1e-12) & ~bnd)[0]
    assert len(on_fold) == ny - 2 and np.abs(th[on_fold] - 2 * math.pi).max() < 1e-12
    rng = np.random.default_rng(61)
    qs = fold_vertex_queries(X, F, P, c, nx, ny, 120, rng)
    out = oracle.exp_map(m, [q[0] for q in qs], [q[1] for q in qs], [q[2] for q in qs], [[q[3]] for q in qs])
    checked = 0
    for i, (f, b, v3, w3, p0, d, L, wf) in enumerate(qs):
        st = out["status"][i]
        assert st & oracle.VERTEX_HIT, i
        if st & (oracle.BOUNDARY | oracle.NEAR_VERTEX | oracle.NEAR_EDGE):
            continue
        g, bg = locate(P, F, p0 + L * d, tol=1e-9)
        A, B, C = P[F[g]]
        a, bb, cc = X[F[g]]
        M2 = np.stack([B - A, C - A], 1)
        to3 = lambda u: (lambda k: k[0] * (bb - a) + k[1] * (cc - a))(np.linalg.lstsq(M2, u, rcond=None)[0])
        assert out["face"][i] == g
        assert np.abs(out["pos"][i] - bg @ X[F[g]]).max() < 1e-11
        assert np.abs(out["dir"][i] - to3(d)).max() < 1e-11
        assert np.abs(out["w"][i, 0] - to3(wf)).max() < 1e-11
        checked += 1
    assert checked > 60


# --------------------------------------------------------------------------- exact brute force
def _rational_queries(pc: Polycube, n, rng):
    qs = []
    for _ in range(n):
        f = int(rng.integers(len(pc.F)))
        r = rng.integers(1, 15, size=3)
        bary = [Fraction(int(x), int(r.sum())) for x in r]
        ax = [c for c in range(3) if c != pc.axis[f]]
        d = [0, 0, 0]
        d[ax[0]] = int(rng.integers(-9, 10))
        d[ax[1]] = int(rng.integers(-9, 10))
        if d[ax[0]] == 0 and d[ax[1]] == 0:
            d[ax[0]] = 1
        t = Fraction(int(rng.integers(1, 64)), 8)
        qs.append((f, bary, d, t))
    return qs


@pytest.mark.parametrize("cells", [[(0, 0, 0)], [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1)]])
def test_polycube_exact_face_sequences(cells):
    """Alg. geodesic_step + transport_over_edge on axis-aligned polycubes, where unfolding is a
    quarter turn and everything is rational: face sequences must match the exact walker
    bit for bit, end points to 1e-12."""
    X, F = meshgen.polycube(cells)
    pc = Polycube(X, F)
    m = oracle.Mesh(X, F)
    rng = np.random.default_rng(3)
    qs = _rational_queries(pc, 150, rng)
    matched = 0
    for f, bary, d, t in qs:
        ex = pc.walk(f, bary, d, t, points=True)
        if ex is None:
            continue
        faces, pend, pts = ex
        v = np.array([float(x * t) for x in d])
        out = oracle.exp_map(m, [f], [[float(b) for b in bary]], [v], path_cap=4096)
        if out["status"][0] & (oracle.NEAR_VERTEX | oracle.NEAR_EDGE):
            continue
        path = out["path"][0]
        path = list(path[path >= 0])
        assert path == faces
        assert out["path_len"][0] == len(faces)
        assert out["hash"][0] == oracle.fnv_hash(faces)
        assert np.abs(out["pos"][0] - np.array([float(c) for c in pend])).max() < 1e-12
        # the traced polyline: the exact entry point of every face
        exact = np.array([[float(c) for c in q] for q in pts])
        assert np.abs(out["path_pt"][0, :len(faces)] - exact).max() < 1e-11   # FP64 rounding over the walk
        matched += 1
    assert matched > 100


def test_traced_polyline_has_the_walked_length_and_crosses_shared_edges():
    """Geodesic tracing (the by-product of Sec. 1 and Sec. 4): inside each face the straightest
    geodesic is a straight segment, so the traced polyline (entry points, then the end point) is
    exactly L long, and each entry point after the first lies on the edge (or, after a vertex
    hit, the vertex) that the previous face and the entered face share."""
    rng = np.random.default_rng(17)
    X, F = meshgen.icosphere(3, 0.01, rng)
    m = oracle.Mesh(X, F)
    q = meshgen.sample_queries(X, F, 300, rng, 0.0, 2.5, 0)
    out = oracle.exp_map(m, q.face, q.bary, q.v, path_cap=512)
    L = np.linalg.norm(q.v, axis=1)
    checked = 0
    for i in range(len(L)):
        n = out["path_len"][i]
        if out["status"][i] & oracle.INVALID or n > 512:
            continue
        if L[i] == 0:
            assert n == 0
            continue
        faces, pts = out["path"][i, :n], out["path_pt"][i, :n]
        p0 = (q.bary[i][:, None] * X[F[q.face[i]]]).sum(0)
        assert np.abs(pts[0] - p0).max() < 1e-14
        poly = np.concatenate([pts, out["pos"][i][None]])
        length = np.linalg.norm(np.diff(poly, axis=0), axis=1).sum()
        assert abs(length - L[i]) <= 1e-12 * max(L[i], 1.0), (i, length, L[i])
        for k in range(1, n):
            shared = set(F[faces[k - 1]]) & set(F[faces[k]])
            if faces[k] == faces[k - 1]:
                shared = set(F[faces[k]])
            a = X[sorted(shared)]
            if len(shared) == 2:
                e = a[1] - a[0]
                t = np.clip(np.dot(pts[k] - a[0], e) / np.dot(e, e), 0.0, 1.0)
                dist = np.linalg.norm(a[0] + t * e - pts[k])
            else:  # vertex hit: the entry point is one of the shared vertices
                dist = np.linalg.norm(a - pts[k], axis=1).min()
            assert dist < 1e-12, (i, k, dist)
        checked += 1
    assert checked > 250


def _square_with_hole():
    X, F = meshgen.flat_grid(21)
    return meshgen.cut_hole(X, F, lambda c: (np.abs(c[:, 0] - 0.5) < 0.1) & (np.abs(c[:, 1] - 0.5) < 0.1))


def test_hole_avoidance_closed_forms_on_a_square_with_a_hole():
    """Hole avoidance (Sec. 4: trace along the boundary, resume with the last straightest
    direction), on the unit square with the hole [0.4, 0.6]^2, where every case has a closed form:
      - a ray into the hole's left side slides up that side to the corner (0.4, 0.6) and resumes
        there with its own direction: end = c + (L - |q - p| - |c - q|) d;
      - a ray that misses the hole is a straight line;
      - a ray leaving through the right side of the square slides up to the corner (1, 1), where
        no face receives it, keeps its sense along the boundary and slides left along the top:
        end = (1 - r, 1) with r the length left at the corner;
      - with boundary_mode 0 the same rays stop where they reach the boundary."""
    X, F = _square_with_hole()
    m = oracle.Mesh(X, F)
    rng = np.random.default_rng(71)
    n = 200
    a = rng.uniform(0.1, 1.0, n)
    d = np.stack([np.cos(a), np.sin(a), np.zeros(n)], 1)
    p = np.stack([np.full(n, 0.2), rng.uniform(0.42, 0.58, n), np.zeros(n)], 1)
    qy = p[:, 1] + 0.2 * np.tan(a)
    L = np.full(n, 0.5)
    # start faces and barycentrics of p
    face, bary = _locate(X, F, p)
    out = oracle.exp_map(m, face, bary, d * L[:, None], boundary_mode=1)
    into = qy < 0.6
    q = np.stack([np.full(n, 0.4), qy, np.zeros(n)], 1)
    rem = L - np.linalg.norm(q - p, axis=1) - (0.6 - qy)
    expect = np.where(into[:, None], np.array([0.4, 0.6, 0.0]) + rem[:, None] * d, p + L[:, None] * d)
    ok = (out["status"] & (oracle.NEAR_VERTEX | oracle.NEAR_EDGE)) == 0
    assert ok.mean() > 0.9 and into[ok].mean() > 0.3
    assert np.abs(out["pos"] - expect)[ok].max() < 1e-12
    assert np.all(((out["status"] & oracle.HOLE) != 0)[ok] == into[ok])
    assert np.all((out["status"] & oracle.BOUNDARY) == 0)
    stop = oracle.exp_map(m, face, bary, d * L[:, None])
    assert np.all(((stop["status"] & oracle.BOUNDARY) != 0)[ok] == into[ok])
    assert np.abs(stop["pos"] - np.where(into[:, None], q, expect))[ok].max() < 1e-12
    # out through the right side of the square, around the corner (1, 1)
    p2 = np.stack([np.full(n, 0.8), rng.uniform(0.7, 0.8, n), np.zeros(n)], 1)
    a2 = rng.uniform(0.1, 0.6, n)
    d2 = np.stack([np.cos(a2), np.sin(a2), np.zeros(n)], 1)
    q2y = p2[:, 1] + 0.2 * np.tan(a2)
    L2 = np.full(n, 0.8)
    f2, b2 = _locate(X, F, p2)
    o2 = oracle.exp_map(m, f2, b2, d2 * L2[:, None], boundary_mode=1)
    r2 = L2 - np.linalg.norm(np.stack([np.full(n, 1.0), q2y, np.zeros(n)], 1) - p2, axis=1) - (1.0 - q2y)
    use = (q2y < 1.0) & (r2 > 0) & (r2 < 1.0) & ((o2["status"] & (oracle.NEAR_VERTEX | oracle.NEAR_EDGE)) == 0)
    assert use.mean() > 0.5
    e2 = np.stack([1.0 - r2, np.ones(n), np.zeros(n)], 1)
    assert np.abs(o2["pos"] - e2)[use].max() < 1e-12


def _locate(X, F, p):
    """Face and barycentrics of planar points p (z = 0) on a planar mesh, by brute force."""
    A, B, C = X[F[:, 0], :2], X[F[:, 1], :2], X[F[:, 2], :2]
    face = np.zeros(len(p), np.int32)
    bary = np.zeros((len(p), 3))
    for i, x in enumerate(p[:, :2]):
        v0, v1, v2 = B - A, C - A, x - A
        d00 = (v0 * v0).sum(1); d01 = (v0 * v1).sum(1); d11 = (v1 * v1).sum(1)
        d20 = (v2 * v0).sum(1); d21 = (v2 * v1).sum(1)
        den = d00 * d11 - d01 * d01
        bv = (d11 * d20 - d01 * d21) / den
        bw = (d00 * d21 - d01 * d20) / den
        bu = 1 - bv - bw
        k = np.nonzero((bu >= 0) & (bv >= 0) & (bw >= 0))[0][0]
        face[i] = k
        bary[i] = (bu[k], bv[k], bw[k])
    return face, bary


def test_hole_avoidance_on_a_sphere_with_holes():
    """A sphere with 8% of its faces removed (every vertex keeps one fan, Sec. 4): with hole
    avoidance no walk stops at the boundary, walks that never touch it are unchanged, and a walk
    that does follows the same faces as the stopping walk up to the boundary."""
    rng = np.random.default_rng(72)
    X, F = meshgen.icosphere(3, 0.003, rng)
    X, F = meshgen.remove_faces(X, F, 0.08, rng)
    m = oracle.Mesh(X, F)
    q = meshgen.sample_queries(X, F, 600, rng, 0.1, 3.0, 1)
    stop = oracle.exp_map(m, q.face, q.bary, q.v, q.w, path_cap=512)
    hole = oracle.exp_map(m, q.face, q.bary, q.v, q.w, path_cap=512, boundary_mode=1)
    hit = (stop["status"] & oracle.BOUNDARY) != 0
    assert hit.mean() > 0.2
    assert not np.any(hole["status"] & oracle.BOUNDARY)
    assert np.all(((hole["status"] & oracle.HOLE) != 0) == hit)
    same = ~hit
    for k in ("face", "pos", "dir", "w", "hash"):
        assert np.array_equal(stop[k][same], hole[k][same]), k
    for i in np.nonzero(hit)[0]:
        n = min(stop["path_len"][i], 512)
        assert np.array_equal(stop["path"][i, :n], hole["path"][i, :n])
    # carried vectors stay unit and keep their angle to the direction
    cw = np.einsum("ij,ij->i", hole["w"][:, 0], hole["dir"])
    c0 = np.einsum("ij,ij->i", q.w[:, 0], q.v / np.linalg.norm(q.v, axis=1, keepdims=True))
    assert np.abs(np.linalg.norm(hole["w"][:, 0], axis=1) - 1).max() < 1e-9
    assert np.abs(cw - c0).max() < 1e-9


def test_cube_worked_examples():
    """Hand-worked examples (tests/golden/cube_worked_examples.txt): one edge-crossing walk and
    two vertex hits at a cube corner, where theta = 3pi/2 and the straightest rule of Sec. 4
    (theta_l = theta_r = theta/2) fixes the outgoing ray."""
    X, F = meshgen.polycube([(0, 0, 0)])
    m = oracle.Mesh(X, F)
    rows = np.loadtxt(os.path.join(GOLDEN, "cube_worked_examples.txt"))
    for r in rows:
        p, d, L, e = r[0:3], r[3:6], r[6], r[7:10]
        f, b = locate(X, F, p)
        v = d / np.linalg.norm(d) * L
        out = oracle.exp_map(m, [f], [b], [v])
        assert np.abs(out["pos"][0] - e).max() < 1e-12, (out["pos"][0], e)


# --------------------------------------------------------------------------- cone vertex rule
@pytest.mark.parametrize("theta", [1.3 * math.pi, 1.8 * math.pi, 2.4 * math.pi])
def test_cone_vertex_straightest_rule(theta):
    """Alg. transport_over_vertex / Sec. 4: a ray through a cone apex leaves at theta/2 from the
    reversed incoming ray (theta = sum of apex angles), for spherical (theta < 2pi) and
    hyperbolic (theta > 2pi) vertices; carried vectors keep their angle to the direction."""
    n = 9
    X, F = meshgen.cone_fan(n, theta)
    m = oracle.Mesh(X, F)
    th, bnd = m.theta()
    T = th[0]
    assert not bnd[0]
    # corner angles at the apex and the polar angle at which each face starts
    gam = []
    for f in F:
        u, w = X[f[1]] - X[0], X[f[2]] - X[0]
        gam.append(math.atan2(np.linalg.norm(np.cross(u, w)), np.dot(u, w)))
    G = np.concatenate([[0.0], np.cumsum(gam)])
    rng = np.random.default_rng(4)
    checked = 0
    for _ in range(40):
        f0 = int(rng.integers(n))
        a = float(rng.uniform(0.1, 0.9)) * gam[f0]      # polar angle inside face f0
        rho = float(rng.uniform(0.2, 0.6))
        lam = float(rng.uniform(0.05, 0.4))
        # point at polar angle a within face f0 at distance rho from the apex
        u = (X[F[f0][1]] - X[0]); u /= np.linalg.norm(u)
        w = (X[F[f0][2]] - X[0])
        w = w - np.dot(w, u) * u; w /= np.linalg.norm(w)
        p = rho * (math.cos(a) * u + math.sin(a) * w)
        dvec = -p / rho
        f, b = locate(X, F, p, tol=1e-10)
        assert f == f0
        n0 = np.cross(u, w)
        beta = float(rng.uniform(-math.pi, math.pi))    # carried vector at a signed angle beta
        w0 = math.cos(beta) * dvec + math.sin(beta) * np.cross(n0, dvec)
        out = oracle.exp_map(m, [f], [b], [dvec * (rho + lam)], [[w0]])
        assert out["status"][0] & oracle.VERTEX_HIT
        phi = (G[f0] + a + T / 2) % T
        j = int(np.searchsorted(G, phi, side="right") - 1)
        uj = X[F[j][1]] - X[0]; uj /= np.linalg.norm(uj)
        wj = X[F[j][2]] - X[0]
        wj = wj - np.dot(wj, uj) * uj; wj /= np.linalg.norm(wj)
        loc = phi - G[j]
        expect = lam * (math.cos(loc) * uj + math.sin(loc) * wj)
        if min(loc, gam[j] - loc) < 1e-6:
            continue  # outgoing ray along an edge (degenerate reading)
        assert np.abs(out["pos"][0] - expect).max() < 1e-12
        # carried vector: the same signed angle beta to the direction, about the end face's
        # normal (the fan is consistently oriented)
        nj = np.cross(uj, wj)
        dj = out["dir"][0]
        assert np.abs(out["w"][0, 0] - (math.cos(beta) * dj + math.sin(beta) * np.cross(nj, dj))).max() < 1e-12
        checked += 1
    assert checked > 30


# --------------------------------------------------------------------------- Gauss-Bonnet
def test_vertex_angle_sums_gauss_bonnet():
    """Sec. 4 defines theta(x) as the sum of incident corner angles; the discrete Gauss-Bonnet
    theorem fixes sum_v (2pi - theta_v) = 2 pi chi exactly for closed meshes."""
    X, F = meshgen.icosphere(3)
    th, b = oracle.Mesh(X, F).theta()
    assert not b.any()
    assert abs(np.sum(2 * np.pi - th) - 4 * np.pi) < 1e-9
    X, F = meshgen.torus(24, 12, 1.0, 0.4, 0.01, np.random.default_rng(5))
    th, _ = oracle.Mesh(X, F).theta()
    assert abs(np.sum(2 * np.pi - th)) < 1e-9
    X, F = meshgen.polycube([(0, 0, 0)])
    th, _ = oracle.Mesh(X, F).theta()
    corners = np.isclose(th, 1.5 * np.pi)
    assert corners.sum() == 8


def test_rejects_non_manifold_and_degenerate():
    """Sec. 4 manifold definition: an edge with three faces, or a vertex whose faces form two
    fans, is rejected; so is a zero-area face."""
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1.0]])
    F3 = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]])
    with pytest.raises(oracle.OracleError, match="non-manifold"):
        oracle.Mesh(X, F3)
    Xb = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [-1, 0, 0], [-1, -1, 0.0]])
    with pytest.raises(oracle.OracleError, match="non-manifold"):
        oracle.Mesh(Xb, np.array([[0, 1, 2], [0, 3, 4]]))
    Xd = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0.0]])
    with pytest.raises(oracle.OracleError, match="degenerate"):
        oracle.Mesh(Xd, np.array([[0, 1, 2]]))


# --------------------------------------------------------------------------- reversibility
@pytest.mark.parametrize("which", ["sphere", "torus"])
def test_reversibility(which):
    """Straightest geodesics are reversible away from vertices: tracing back from p' with
    -d' for the same length returns to p and visits the faces in reverse order."""
    rng = np.random.default_rng(6)
    if which == "sphere":
        X, F = meshgen.icosphere(3, 0.01, rng)
        q = meshgen.sample_queries(X, F, 400, rng, 0.0, 3.0, 0)
    else:
        X, F = meshgen.torus(48, 24, 1.0, 0.4, 0.002, rng)
        q = meshgen.sample_queries(X, F, 400, rng, 0.0, 2.0, 0)
    m = oracle.Mesh(X, F)
    fw = oracle.exp_map(m, q.face, q.bary, q.v, path_cap=2048)
    L = np.linalg.norm(q.v, axis=1)
    bk = oracle.exp_map(m, fw["face"], fw["bary"], -fw["dir"] * L[:, None], path_cap=2048)
    ok = ((fw["status"] | bk["status"]) & (oracle.NEAR_VERTEX | oracle.NEAR_EDGE | oracle.BOUNDARY)) == 0
    assert ok.mean() > 0.8
    p0 = start_points(X, F, q.face, q.bary)
    assert np.abs(bk["pos"] - p0)[ok].max() < 1e-9
    for i in np.nonzero(ok)[0][:100]:
        a = fw["path"][i][fw["path"][i] >= 0]
        b = bk["path"][i][bk["path"][i] >= 0]
        assert list(a[::-1]) == list(b)


# --------------------------------------------------------------------------- transport
def test_transport_preserves_norm_and_angle():
    """Sec. 4 'Parallel Transport': the angle between the carried vector and the curve tangent
    is constant (and on orientable meshes so is its sign); the norm is preserved."""
    rng = np.random.default_rng(7)
    X, F = meshgen.torus(40, 20, 1.0, 0.4, 0.003, rng)
    m = oracle.Mesh(X, F)
    q = meshgen.sample_queries(X, F, 500, rng, 0.0, 2.0, 2)
    q.w[:, 1] *= 2.5
    out = oracle.exp_map(m, q.face, q.bary, q.v, q.w)
    d0 = q.v / np.linalg.norm(q.v, axis=1, keepdims=True)
    n0 = np.cross(X[F[q.face, 1]] - X[F[q.face, 0]], X[F[q.face, 2]] - X[F[q.face, 0]])
    n1 = np.cross(X[F[out["face"], 1]] - X[F[out["face"], 0]], X[F[out["face"], 2]] - X[F[out["face"], 0]])
    for k in range(2):
        assert np.abs(np.linalg.norm(out["w"][:, k], axis=1) - np.linalg.norm(q.w[:, k], axis=1)).max() < 1e-12
        a0 = np.arctan2(np.einsum("ij,ij->i", np.cross(d0, q.w[:, k]), n0) / np.linalg.norm(n0, axis=1),
                        np.einsum("ij,ij->i", d0, q.w[:, k]))
        a1 = np.arctan2(np.einsum("ij,ij->i", np.cross(out["dir"], out["w"][:, k]), n1) / np.linalg.norm(n1, axis=1),
                        np.einsum("ij,ij->i", out["dir"], out["w"][:, k]))
        diff = np.angle(np.exp(1j * (a1 - a0)))
        assert np.abs(diff).max() < 1e-10
    # two carried vectors keep their mutual angle
    c0 = np.einsum("ij,ij->i", q.w[:, 0], q.w[:, 1])
    c1 = np.einsum("ij,ij->i", out["w"][:, 0], out["w"][:, 1])
    assert np.abs(c0 - c1).max() < 1e-11


# --------------------------------------------------------------------------- smooth trends
def sphere_exact(p, v):
    """Closed-form sphere Exp (Sec. 5.1 and App. 'Exp map on the Sphere')."""
    L = np.linalg.norm(v, axis=1, keepdims=True)
    return np.cos(L) * p + np.sin(L) * v / L


def test_sphere_error_decreases_with_resolution():
    """Sec. 5.1: errors against the closed-form sphere Exp come from discretisation and shrink
    as the mesh resolution grows."""
    errs = []
    for level in (2, 3, 4, 5):
        X, F = meshgen.icosphere(level)
        m = oracle.Mesh(X, F)
        rng = np.random.default_rng(8)
        q = meshgen.sample_queries(X, F, 2000, rng, 0.0, 1.5, 0)
        out = oracle.exp_map(m, q.face, q.bary, q.v)
        p0 = start_points(X, F, q.face, q.bary)
        ps = p0 / np.linalg.norm(p0, axis=1, keepdims=True)
        # tangent vector at the projected point with the same direction and length
        vs = q.v - np.einsum("ij,ij->i", q.v, ps)[:, None] * ps
        vs *= (np.linalg.norm(q.v, axis=1) / np.linalg.norm(vs, axis=1))[:, None]
        errs.append(np.linalg.norm(out["pos"] - sphere_exact(ps, vs), axis=1).mean())
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.25 * errs[0]


def torus_rk4(R, r, a0, b0, da, db, n=4000):
    """RK4 integration of the torus geodesic IVP (App. 'IVP on Torus', Eq. torus-geodesic)."""
    def rhs(s):
        a, b, ad, bd = s
        return np.array([ad, bd, 2 * r * math.sin(b) / (R + r * math.cos(b)) * ad * bd,
                         -(R + r * math.cos(b)) * math.sin(b) / r * ad * ad])
    s = np.array([a0, b0, da, db], float)
    h = 1.0 / n
    for _ in range(n):
        k1 = rhs(s); k2 = rhs(s + 0.5 * h * k1); k3 = rhs(s + 0.5 * h * k2); k4 = rhs(s + h * k3)
        s = s + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    a, b = s[0], s[1]
    return np.array([(R + r * math.cos(b)) * math.cos(a), (R + r * math.cos(b)) * math.sin(a), r * math.sin(b)])


def test_torus_error_against_ivp_decreases():
    """Sec. 5.1 / App. 'IVP on Torus': the mesh Exp approaches the smooth torus geodesic
    (Christoffel ODE, integrated by RK4) as the grid is refined."""
    R, r = 1.0, 0.4
    rng = np.random.default_rng(9)
    starts = [(rng.uniform(0, 2 * np.pi), rng.uniform(0, 2 * np.pi), rng.uniform(0, 2 * np.pi),
               rng.uniform(0.3, 1.0)) for _ in range(12)]
    errs = []
    for na in (64, 128, 256):
        X, F = meshgen.torus(na, na // 2, R, r)
        m = oracle.Mesh(X, F)
        e = []
        for a0, b0, psi, L in starts:
            P = np.array([(R + r * math.cos(b0)) * math.cos(a0), (R + r * math.cos(b0)) * math.sin(a0), r * math.sin(b0)])
            Fa = np.array([-(R + r * math.cos(b0)) * math.sin(a0), (R + r * math.cos(b0)) * math.cos(a0), 0])
            Fb = np.array([-r * math.sin(b0) * math.cos(a0), -r * math.sin(b0) * math.sin(a0), r * math.cos(b0)])
            u = math.cos(psi) * Fa / np.linalg.norm(Fa) + math.sin(psi) * Fb / np.linalg.norm(Fb)
            v = L * u
            da, db = v @ Fa / (Fa @ Fa), v @ Fb / (Fb @ Fb)
            exact = torus_rk4(R, r, a0, b0, da, db)
            # nearest mesh face to P, start at the projection of P into it
            c = X[F].mean(1)
            f = int(np.argmin(np.linalg.norm(c - P, axis=1)))
            A, B, Cc = X[F[f]]
            nrm = np.cross(B - A, Cc - A); nrm /= np.linalg.norm(nrm)
            Pp = P - np.dot(P - A, nrm) * nrm
            M = np.stack([B - A, Cc - A], 1)
            uv, *_ = np.linalg.lstsq(M, Pp - A, rcond=None)
            bary = np.array([1 - uv.sum(), uv[0], uv[1]])
            if bary.min() < 0:
                bary = np.clip(bary, 1e-3, None); bary /= bary.sum()
            out = oracle.exp_map(m, [f], [bary], [v - np.dot(v, nrm) * nrm])
            e.append(np.linalg.norm(out["pos"][0] - exact))
        errs.append(np.mean(e))
    assert errs[2] < errs[0], errs
    assert errs[2] < 2e-2, errs


# --------------------------------------------------------------------------- gradients
def _frames(X, F, face, v):
    a, b, c = X[F[face, 0]], X[F[face, 1]], X[F[face, 2]]
    n = np.cross(b - a, c - a); n /= np.linalg.norm(n, axis=1, keepdims=True)
    vp = v - np.einsum("ij,ij->i", v, n)[:, None] * n
    ep = vp / np.linalg.norm(vp, axis=1, keepdims=True)
    eq = np.cross(n, ep)
    eu = (b - a) / np.linalg.norm(b - a, axis=1, keepdims=True)
    ev = (c - a) / np.linalg.norm(c - a, axis=1, keepdims=True)
    return n, ep, eq, eu, ev


def fd_gradients(m, X, F, q, h=1e-4):
    """FP64 central differences of the oracle walk: grad_v along (e_par, e_perp) and grad_p
    along (e_u, e_v) of the start face, projected onto the end-face plane as in Eqs. jv, jp.
    Returns (grad_v, grad_p, straddle) where straddle marks queries whose +-h walks visit a
    different face sequence than the base walk."""
    n, ep, eq, eu, ev = _frames(X, F, q.face, q.v)
    base = oracle.exp_map(m, q.face, q.bary, q.v)
    fe = base["face"]
    n1 = np.cross(X[F[fe, 1]] - X[F[fe, 0]], X[F[fe, 2]] - X[F[fe, 0]])
    n1 /= np.linalg.norm(n1, axis=1, keepdims=True)

    def proj(x):
        return x - np.einsum("ij,ij->i", x, n1)[:, None] * n1

    strad = np.zeros(len(q), bool)
    cols = {}
    for name, e in (("par", ep), ("perp", eq)):
        op = oracle.exp_map(m, q.face, q.bary, q.v + h * e)
        om = oracle.exp_map(m, q.face, q.bary, q.v - h * e)
        strad |= (op["hash"] != base["hash"]) | (om["hash"] != base["hash"])
        cols[name] = proj((op["pos"] - om["pos"]) / (2 * h))
    g = q.g_pos
    gv = ep * np.einsum("ij,ij->i", cols["par"], g)[:, None] + eq * np.einsum("ij,ij->i", cols["perp"], g)[:, None]
    P = X[F[q.face]]
    Minv = []
    for name, e in (("u", eu), ("v", ev)):
        # p +- h e as barycentric coordinates of the same face
        dp = h * e
        M = np.stack([P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]], 2)
        uv = np.linalg.solve(np.einsum("qki,qkj->qij", M, M), np.einsum("qki,qk->qi", M, dp)[..., None])[..., 0]
        db = np.stack([-uv.sum(1), uv[:, 0], uv[:, 1]], 1)
        bp, bm = q.bary + db, q.bary - db
        inside = (bp.min(1) > 0) & (bm.min(1) > 0)
        strad |= ~inside
        bp = np.where(inside[:, None], bp, q.bary)
        bm = np.where(inside[:, None], bm, q.bary)
        op = oracle.exp_map(m, q.face, bp, q.v)
        om = oracle.exp_map(m, q.face, bm, q.v)
        strad |= (op["hash"] != base["hash"]) | (om["hash"] != base["hash"])
        cols[name] = proj((op["pos"] - om["pos"]) / (2 * h))
    gu = np.einsum("ij,ij->i", cols["u"], g)
    gw = np.einsum("ij,ij->i", cols["v"], g)
    a11 = np.einsum("ij,ij->i", eu, eu); a12 = np.einsum("ij,ij->i", eu, ev); a22 = np.einsum("ij,ij->i", ev, ev)
    det = a11 * a22 - a12 * a12
    c0 = (a22 * gu - a12 * gw) / det
    c1 = (-a12 * gu + a11 * gw) / det
    gp = c0[:, None] * eu + c1[:, None] * ev
    strad |= (base["status"] & (oracle.NEAR_VERTEX | oracle.BOUNDARY | oracle.NEAR_EDGE)) != 0
    return gv, gp, strad


def _rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-30)


def test_ep_and_gfd_match_central_differences():
    """Eq. proxy_func (EP, J^v = R) and Eqs. jv/jp (GFD) against FP64 central differences of
    the walk, on queries whose perturbed walks stay in the same face strip (where the map is
    affine and both estimators are exact)."""
    rng = np.random.default_rng(10)
    X, F = meshgen.icosphere(4, 0.003, rng)
    m = oracle.Mesh(X, F)
    q = meshgen.sample_queries(X, F, 600, rng, 0.1, 1.0, 0)
    gv_fd, gp_fd, strad = fd_gradients(m, X, F, q)
    keep = ~strad
    assert keep.mean() > 0.6
    ep = oracle.ep_backward(m, q.face, q.bary, q.v, q.g_pos)
    assert _rel(ep["grad_v"], gv_fd)[keep].max() < 1e-6
    assert np.all(ep["grad_p"] == 0)
    gfd = oracle.gfd_backward(m, q.face, q.bary, q.v, q.g_pos, 1e-4, 1e-4)
    assert _rel(gfd["grad_v"], gv_fd)[keep].max() < 1e-6
    assert _rel(gfd["grad_p"], gp_fd)[keep].max() < 1e-6
    # grad_bary_k = <grad_p, x_k>
    P = X[F[q.face]]
    assert np.abs(gfd["grad_bary"] - np.einsum("qkj,qj->qk", P, gfd["grad_p"])).max() < 1e-12


def test_flat_gradients_closed_form():
    """On a plane Exp(p, v) = p + v, so J^v = J^p = identity on the plane: the VJPs of EP
    (grad_v) and GFD (grad_v, grad_p) equal the in-plane part of the upstream gradient."""
    rng = np.random.default_rng(11)
    X, F = meshgen.flat_grid(15, rng, jitter=0.2)
    m = oracle.Mesh(X, F)
    q = meshgen.sample_queries(X, F, 400, rng, 0.05, 0.3, 0)
    fw = oracle.exp_map(m, q.face, q.bary, q.v)
    gpl = q.g_pos.copy(); gpl[:, 2] = 0
    ok = (fw["status"] & (oracle.BOUNDARY | oracle.NEAR_EDGE)) == 0
    ep = oracle.ep_backward(m, q.face, q.bary, q.v, q.g_pos)
    gfd = oracle.gfd_backward(m, q.face, q.bary, q.v, q.g_pos)
    ok &= (gfd["flags"] & oracle.BOUNDARY) == 0
    assert ok.mean() > 0.7
    assert np.abs(ep["grad_v"] - gpl)[ok].max() < 1e-12
    assert np.abs(gfd["grad_v"] - gpl)[ok].max() < 1e-8
    assert np.abs(gfd["grad_p"] - gpl)[ok].max() < 1e-8


def test_gfd_tracks_sphere_jacobian():
    """App. 'Exp map on the Sphere' (Eqs. jp_sphere, jv_sphere) and Fig. diff-acc: GFD gradients
    for v closely follow the closed-form sphere gradients on a fine mesh (cosine similarity),
    EP's v-gradient is a good approximation of it."""
    X, F = meshgen.icosphere(5)
    m = oracle.Mesh(X, F)
    rng = np.random.default_rng(12)
    q = meshgen.sample_queries(X, F, 300, rng, 0.2, 1.2, 0)
    p0 = start_points(X, F, q.face, q.bary)
    ps = p0 / np.linalg.norm(p0, axis=1, keepdims=True)
    n, ep_, eq_, _, _ = _frames(X, F, q.face, q.v)
    vproj = q.v - np.einsum("ij,ij->i", q.v, n)[:, None] * n
    L = np.linalg.norm(vproj, axis=1)
    cs_gfd, cs_ep = [], []
    gfd = oracle.gfd_backward(m, q.face, q.bary, q.v, q.g_pos, 1e-3, 1e-3)
    ep = oracle.ep_backward(m, q.face, q.bary, q.v, q.g_pos)
    for i in range(len(q)):
        v = vproj[i]
        Lv = L[i]
        vv = np.outer(v, v)
        Jv = (np.eye(3) - np.outer(ps[i], v)) / Lv * math.sin(Lv) - vv / Lv ** 3 * math.sin(Lv) + vv / Lv ** 2 * math.cos(Lv)
        gsm = q.g_pos[i] @ Jv
        # compare within the start tangent plane
        T = np.stack([ep_[i], eq_[i]])
        a, b = T @ gsm, T @ gfd["grad_v"][i]
        cs_gfd.append(a @ b / np.linalg.norm(a) / np.linalg.norm(b))
        b2 = T @ ep["grad_v"][i]
        cs_ep.append(a @ b2 / np.linalg.norm(a) / np.linalg.norm(b2))
    assert np.median(cs_gfd) > 0.97, np.median(cs_gfd)
    assert np.median(cs_ep) > 0.97, np.median(cs_ep)


# --------------------------------------------------------------------------- non-orientable
def test_non_orientable_meshes_gauss_bonnet_and_transport():
    """App. 'Main differences with SotA implementation': only triangle adjacency is stored, so
    non-orientable meshes (Moebius strip, Klein bottle) work.  Gauss-Bonnet gives
    sum(2pi - theta) = 2 pi chi = 0 on the Klein bottle; transport keeps |w| and the unsigned
    angle between w and the direction (the sign has no global meaning on such surfaces)."""
    X, F = meshgen.klein_bottle(64, 32)
    m = oracle.Mesh(X, F)
    th, b = m.theta()
    assert not b.any()
    assert abs(np.sum(2 * np.pi - th)) < 1e-9
    rng = np.random.default_rng(41)
    q = meshgen.sample_queries(X, F, 800, rng, 1.0, 8.0, 2)
    out = oracle.exp_map(m, q.face, q.bary, q.v, q.w)
    ok = (out["status"] & (oracle.NEAR_VERTEX | oracle.BOUNDARY)) == 0
    assert out["ncross"][ok].mean() > 20
    d0 = q.v / np.linalg.norm(q.v, axis=1, keepdims=True)
    for k in range(2):
        assert np.abs(np.linalg.norm(out["w"][:, k], axis=1) - 1.0)[ok].max() < 1e-12
        c0 = np.einsum("ij,ij->i", d0, q.w[:, k])
        c1 = np.einsum("ij,ij->i", out["dir"], out["w"][:, k])
        assert np.abs(c0 - c1)[ok].max() < 1e-10
    # reversibility also holds across orientation flips
    L = np.linalg.norm(q.v, axis=1)
    bk = oracle.exp_map(m, out["face"], out["bary"], -out["dir"] * L[:, None])
    ok &= (bk["status"] & (oracle.NEAR_VERTEX | oracle.NEAR_EDGE)) == 0
    p0 = start_points(X, F, q.face, q.bary)
    assert np.abs(bk["pos"] - p0)[ok].max() < 1e-9


# --------------------------------------------------------------------------- inverse transport
@pytest.mark.parametrize("which", ["torus", "klein"])
def test_inverse_transport_is_the_reverse_walk(which):
    """App. 'Additional Details on Mesh-LBFGS and GCVT': the adjoint of the parallel transport
    moves a vector backwards on the curve.  The oracle's adjoint (from its definition with the
    carried start basis) must equal an independent walk from p' along -d' for the same length
    carrying u, on orientable and non-orientable meshes; it inverts the forward transport and
    is the identity on a flat mesh."""
    rng = np.random.default_rng(43)
    if which == "torus":
        X, F = meshgen.torus(40, 20, 1.0, 0.4, 0.003, rng)
        q = meshgen.sample_queries(X, F, 500, rng, 0.0, 2.0, 2)
    else:
        X, F = meshgen.klein_bottle(64, 32)
        q = meshgen.sample_queries(X, F, 500, rng, 1.0, 8.0, 2)
    m = oracle.Mesh(X, F)
    u = rng.normal(size=(len(q.face), 2, 3))
    back, fw = oracle.transport_back(m, q.face, q.bary, q.v, u)
    L = np.linalg.norm(q.v, axis=1)
    bk = oracle.exp_map(m, fw["face"], fw["bary"], -fw["dir"] * L[:, None], u)
    ok = ((fw["status"] | bk["status"]) & (oracle.NEAR_VERTEX | oracle.NEAR_EDGE | oracle.BOUNDARY)) == 0
    assert ok.mean() > 0.8
    assert np.array_equal(bk["face"][ok], q.face[ok])
    assert np.abs(bk["w"] - back)[ok].max() < 1e-9
    # inverse of the forward transport: Pi* (Pi w) = w projected onto the start face
    fw2 = oracle.exp_map(m, q.face, q.bary, q.v, q.w)
    rt, _ = oracle.transport_back(m, q.face, q.bary, q.v, fw2["w"])
    x0, x1, x2 = X[F[q.face, 0]], X[F[q.face, 1]], X[F[q.face, 2]]
    n = np.cross(x1 - x0, x2 - x0)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    wp = q.w - np.einsum("qkj,qj->qk", q.w, n)[..., None] * n[:, None, :]
    assert np.abs(rt - wp)[ok].max() < 1e-10


def test_inverse_transport_flat_and_empty_path():
    """On a flat mesh parallel transport is the identity, so is its inverse; a zero vector v
    walks an empty path and carries every vector unchanged (projected onto the face)."""
    rng = np.random.default_rng(44)
    X, F = meshgen.flat_grid(13, rng, jitter=0.3)
    m = oracle.Mesh(X, F)
    q = meshgen.sample_queries(X, F, 300, rng, 0.0, 0.4, 0)
    u = np.c_[rng.normal(size=(300, 2)), np.zeros(300)]
    back, fw = oracle.transport_back(m, q.face, q.bary, q.v, u)
    ok = (fw["status"] & (oracle.NEAR_VERTEX | oracle.BOUNDARY)) == 0
    assert ok.mean() > 0.5
    assert np.abs(back - u)[ok].max() < 1e-12
    # zero vector: out = u projected onto the start face, on a curved mesh
    Xs, Fs = meshgen.icosphere(2, 0.0, rng)
    ms = oracle.Mesh(Xs, Fs)
    qs = meshgen.sample_queries(Xs, Fs, 50, rng, 0.1, 0.2, 0)
    us = rng.normal(size=(50, 3))
    w0 = oracle.exp_map(ms, qs.face, qs.bary, np.zeros((50, 3)), us[:, None, :])
    b0, _ = oracle.transport_back(ms, qs.face, qs.bary, np.zeros((50, 3)), us)
    n = np.cross(Xs[Fs[qs.face, 1]] - Xs[Fs[qs.face, 0]], Xs[Fs[qs.face, 2]] - Xs[Fs[qs.face, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    up = us - np.einsum("qj,qj->q", us, n)[:, None] * n
    assert np.abs(w0["w"][:, 0] - up).max() < 1e-14
    assert np.abs(b0 - up).max() < 1e-14
