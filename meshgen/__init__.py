"""Seeded synthetic meshes and queries for the straightest-geodesic exponential map.

This module only *builds inputs*: triangle meshes (icospheres, tori, heightfields,
sliver-jittered grids, small test shapes) and batches of queries (start face,
barycentric point, tangent vector, carried tangent vectors, upstream gradients).
It holds none of the method's arithmetic (no walking, unfolding, transport or
differentiation), so both the CPU oracle and the CUDA path may consume it.

All randomness is NumPy PCG64.  Meshes are built in float64; callers cast to
float32 when they feed the CUDA library.  The workload recipes mirror the paper's
evaluation setting (meshes with 1e3..4e6 faces, Sec. 5.1; random tangent vectors
and lengths, Sec. 5.1 and App. "Gradient evaluation on more meshes").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "icosphere", "torus", "heightfield", "jitter_slivers", "flat_grid", "folded_strip",
    "polycube", "cone_fan", "sample_queries", "Queries", "workload", "WORKLOADS",
    "face_areas", "bbox_diag",
]


def rng_for(index: int) -> np.random.Generator:
    """PCG64 stream for workload `index` (seed = 1000 + index)."""
    return np.random.Generator(np.random.PCG64(1000 + index))


# --------------------------------------------------------------------------- meshes
def icosphere(level: int, radial_noise: float = 0.0, rng: np.random.Generator | None = None):
    """Unit icosphere: icosahedron, `level` rounds of 4-way midpoint subdivision,
    vertices projected to the unit sphere.  V = 10*4^s + 2, F = 20*4^s.
    Optional radial noise r = 1 + N(0, radial_noise^2) per vertex."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    V = [np.array(v, float) / np.linalg.norm(v) for v in V]
    F = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = V[a] + V[b]
                V.append(m / np.linalg.norm(m))
                cache[key] = len(V) - 1
            return cache[key]

        nf = []
        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = nf
    X = np.array(V, dtype=np.float64)
    Fa = np.array(F, dtype=np.int32)
    if radial_noise > 0.0:
        assert rng is not None
        X = X * (1.0 + rng.normal(0.0, radial_noise, size=(len(X), 1)))
    return X, Fa


def torus(na: int, nb: int, R: float = 1.0, r: float = 0.4, noise: float = 0.0,
          rng: np.random.Generator | None = None):
    """Torus F(a, b) = ((R + r cos b) cos a, (R + r cos b) sin a, r sin b) sampled on an
    na x nb (alpha, beta) grid, each quad split by the fixed (i,j)-(i+1,j+1) diagonal,
    faces wound with outward normals.  Optional N(0, noise^2) per coordinate."""
    a = 2.0 * np.pi * np.arange(na) / na
    b = 2.0 * np.pi * np.arange(nb) / nb
    A, B = np.meshgrid(a, b, indexing="ij")
    X = np.stack([(R + r * np.cos(B)) * np.cos(A), (R + r * np.cos(B)) * np.sin(A),
                  r * np.sin(B)], -1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(na), np.arange(nb), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00 = i * nb + j
    v10 = ((i + 1) % na) * nb + j
    v11 = ((i + 1) % na) * nb + (j + 1) % nb
    v01 = i * nb + (j + 1) % nb
    F = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)])
    F = F.astype(np.int32)
    # wind every face so its normal points away from the tube centre line
    _orient_outward_torus(X, F, R)
    if noise > 0.0:
        assert rng is not None
        X = X + rng.normal(0.0, noise, size=X.shape)
    return X, F


def _orient_outward_torus(X, F, R):
    p0, p1, p2 = X[F[:, 0]], X[F[:, 1]], X[F[:, 2]]
    n = np.cross(p1 - p0, p2 - p0)
    c = (p0 + p1 + p2) / 3.0
    rho = np.linalg.norm(c[:, :2], axis=1, keepdims=True)
    core = np.concatenate([c[:, :2] / rho * R, np.zeros((len(c), 1))], 1)
    flip = np.einsum("ij,ij->i", n, c - core) < 0
    F[flip] = F[flip][:, [0, 2, 1]]


def sinusoid_params(rng: np.random.Generator, k: int = 8):
    """Eight random plane waves: a_k, b_k ~ U[-4, 4], phi_k ~ U[0, 2pi)."""
    return rng.uniform(-4, 4, k), rng.uniform(-4, 4, k), rng.uniform(0, 2 * np.pi, k)


def heightfield(n: int, rng: np.random.Generator, amp: float = 0.05, waves=None):
    """n x n vertex grid on [0,1]^2 with z = sum_k amp*sin(2pi(a_k x + b_k y) + phi_k);
    each cell split by the (i,j)-(i+1,j+1) diagonal, normals +z.  F = 2 (n-1)^2."""
    a, b, ph = waves if waves is not None else sinusoid_params(rng)
    xs = np.linspace(0.0, 1.0, n)
    Xg, Yg = np.meshgrid(xs, xs, indexing="ij")
    Z = np.zeros_like(Xg)
    for k in range(len(a)):
        Z += amp * np.sin(2 * np.pi * (a[k] * Xg + b[k] * Yg) + ph[k])
    X = np.stack([Xg, Yg, Z], -1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00, v10, v11, v01 = i * n + j, (i + 1) * n + j, (i + 1) * n + j + 1, i * n + j + 1
    F = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)])
    return X, F.astype(np.int32), (a, b, ph)


def jitter_slivers(X, n: int, rng: np.random.Generator, frac: float = 0.10, waves=None,
                   amp: float = 0.05):
    """Move `frac` of all vertices, drawn from the independent set {(i,j): i, j even,
    interior}, along a random grid axis by U[0.45, 0.4995]*h (h = grid step), then
    re-evaluate the height law at the new (x, y).  Neighbours never move, so faces
    get aspect ratios up to ~1e3 without inverting."""
    h = 1.0 / (n - 1)
    ii, jj = np.meshgrid(np.arange(2, n - 2, 2), np.arange(2, n - 2, 2), indexing="ij")
    cand = (ii * n + jj).ravel()
    k = min(len(cand), int(round(frac * n * n)))
    pick = rng.choice(cand, size=k, replace=False)
    axis = rng.integers(0, 2, size=k)
    sign = rng.choice([-1.0, 1.0], size=k)
    mag = rng.uniform(0.45, 0.4995, size=k) * h
    Y = X.copy()
    Y[pick, axis] += sign * mag
    if waves is not None:
        a, b, ph = waves
        z = np.zeros(k)
        for q in range(len(a)):
            z += amp * np.sin(2 * np.pi * (a[q] * Y[pick, 0] + b[q] * Y[pick, 1]) + ph[q])
        Y[pick, 2] = z
    return Y


def flat_grid(n: int, rng: np.random.Generator | None = None, jitter: float = 0.0):
    """Planar n x n grid in z = 0 on [0,1]^2 (optionally with in-plane jitter of interior
    vertices), a developable surface where every straightest geodesic is a straight line."""
    xs = np.linspace(0.0, 1.0, n)
    Xg, Yg = np.meshgrid(xs, xs, indexing="ij")
    X = np.stack([Xg, Yg, np.zeros_like(Xg)], -1).reshape(-1, 3)
    if jitter > 0:
        h = 1.0 / (n - 1)
        inner = (Xg.ravel() > 0) & (Xg.ravel() < 1) & (Yg.ravel() > 0) & (Yg.ravel() < 1)
        X[inner, :2] += rng.uniform(-jitter * h, jitter * h, size=(inner.sum(), 2))
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00, v10, v11, v01 = i * n + j, (i + 1) * n + j, (i + 1) * n + j + 1, i * n + j + 1
    F = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)])
    return X, F.astype(np.int32)


def cut_hole(X, F, inside):
    """Remove the faces whose centroid satisfies inside(centroid) (a boolean function of [k,3]
    points) and drop unused vertices.  Returns (X, F)."""
    return _compact(X, F[~inside(X[F].mean(1))])


def remove_faces(X, F, frac: float, rng: np.random.Generator):
    """Remove about frac * |F| random faces while keeping the mesh manifold in the sense of
    Sec. 4 (every vertex keeps one connected fan): a face is removed only if, for each of its
    vertices, the remaining incident faces still form one fan (connected through shared
    edges at that vertex) and at least one remains.  Returns (X, F) without unused vertices."""
    nF = len(F)
    alive = np.ones(nF, bool)
    inc = [[] for _ in range(len(X))]
    for f, t in enumerate(F):
        for v in t:
            inc[v].append(f)

    def one_fan(v, drop):
        fs = [f for f in inc[v] if alive[f] and f != drop]
        if not fs:
            return False
        # union through shared edges (v, u)
        seen = {fs[0]}
        stack = [fs[0]]
        while stack:
            f = stack.pop()
            others = set(F[f]) - {v}
            for g in fs:
                if g not in seen and len(others & (set(F[g]) - {v})) == 1:
                    seen.add(g)
                    stack.append(g)
        return len(seen) == len(fs)

    target = int(frac * nF)
    removed = 0
    for f in rng.permutation(nF):
        if removed >= target:
            break
        if all(one_fan(v, f) for v in F[f]):
            alive[f] = False
            removed += 1
    return _compact(X, F[alive])


def _compact(X, F):
    used = np.unique(F)
    remap = -np.ones(len(X), np.int64)
    remap[used] = np.arange(len(used))
    return X[used], remap[F].astype(np.int32)


def folded_strip(nx: int, ny: int, width: float, height: float, folds, rng=None, jitter=0.0):
    """A planar grid strip [0,width] x [0,height] folded along vertical grid lines.
    `folds` is a list of (column index, angle) pairs: the part of the strip right of
    that column is rotated by `angle` about the fold line.  Returns (X, F, develop)
    where `develop(x)` maps a 3-D point of the folded strip back to the plane."""
    xs = np.linspace(0.0, width, nx)
    ys = np.linspace(0.0, height, ny)
    Xg, Yg = np.meshgrid(xs, ys, indexing="ij")
    P = np.stack([Xg, Yg, np.zeros_like(Xg)], -1).reshape(-1, 3)
    X = P.copy()
    col = np.repeat(np.arange(nx), ny)
    # apply folds from right to left so later folds move earlier-rotated parts rigidly
    for c, ang in sorted(folds, key=lambda t: -t[0]):
        x0 = xs[c]
        sel = col > c
        ca, sa = math.cos(ang), math.sin(ang)
        dx = X[sel, 0] - x0
        dz = X[sel, 2]
        X[sel, 0] = x0 + ca * dx - sa * dz
        X[sel, 2] = sa * dx + ca * dz
    i, j = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00, v10, v11, v01 = i * ny + j, (i + 1) * ny + j, (i + 1) * ny + j + 1, i * ny + j + 1
    F = np.concatenate([np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)])
    return X, F.astype(np.int32), P


def polycube(cells, split: str = "fixed"):
    """Closed surface of a union of unit cubes at integer coordinates `cells`
    (iterable of (i,j,k)).  Each boundary unit square is split into two triangles by
    a fixed diagonal, wound outward.  Coordinates are small integers, exact in any
    floating-point format."""
    cells = set(map(tuple, cells))
    quads = []
    dirs = [((1, 0, 0), 0), ((-1, 0, 0), 0), ((0, 1, 0), 1), ((0, -1, 0), 1), ((0, 0, 1), 2),
            ((0, 0, -1), 2)]
    for c in sorted(cells):
        for d, ax in dirs:
            nb = (c[0] + d[0], c[1] + d[1], c[2] + d[2])
            if nb in cells:
                continue
            s = 1 if sum(d) > 0 else 0
            base = list(c)
            base[ax] += s
            u, w = [a for a in range(3) if a != ax]
            p0 = tuple(base)
            p1 = list(base); p1[u] += 1; p1 = tuple(p1)
            p2 = list(base); p2[u] += 1; p2[w] += 1; p2 = tuple(p2)
            p3 = list(base); p3[w] += 1; p3 = tuple(p3)
            # outward normal = d; (u, w) cross product sign decides the winding
            e = [0, 0, 0]; e[u] = 1
            f = [0, 0, 0]; f[w] = 1
            n = np.cross(e, f)
            q = [p0, p1, p2, p3]
            if np.dot(n, d) < 0:
                q = [p0, p3, p2, p1]
            quads.append(q)
    index: dict[tuple, int] = {}
    V = []
    F = []
    for q in quads:
        ids = []
        for p in q:
            if p not in index:
                index[p] = len(V)
                V.append(p)
            ids.append(index[p])
        F.append((ids[0], ids[1], ids[2]))
        F.append((ids[0], ids[2], ids[3]))
    return np.array(V, dtype=np.float64), np.array(F, dtype=np.int32)


def cone_fan(n: int, theta: float, slant: float = 1.0, ring: bool = True):
    """A cone around an apex at the origin: n congruent triangles (apex, r_i, r_{i+1})
    whose apex angles sum to `theta` (< 2pi: convex cone, > 2pi: saddle).  Rim
    vertices alternate in height for theta > 2pi so the fan embeds.  `slant` is the
    apex-to-rim distance.  Returns (X, F) with vertex 0 the apex; the rim is the
    boundary."""
    gam = theta / n
    # choose rim points with pairwise apex angle gam; place on a curve that embeds
    pts = [np.zeros(3)]
    if theta <= 2 * math.pi:
        # right circular cone with opening such that unrolled angle = theta
        sin_half = theta / (2 * math.pi)  # rim radius / slant
        rr = slant * sin_half
        hh = -slant * math.sqrt(max(0.0, 1 - sin_half ** 2))
        for i in range(n):
            a = 2 * math.pi * i / n
            pts.append(np.array([rr * math.cos(a), rr * math.sin(a), hh]))
        # exact apex angle between consecutive rim points, rescale n-gon to hit gam
        # (the regular n-gon on a circular cone has apex angle slightly different
        #  from theta/n; accept the realised total angle and report it)
    else:
        # saddle: rim points on a wavy circle z = h cos(2 a) with constant slant
        for i in range(n):
            a = 2 * math.pi * i / n
            pts.append(np.array([math.cos(a), math.sin(a), 0.0]))
        # bisect the wave height so that the realised total angle matches theta
        lo, hi = 0.0, 5.0
        for _ in range(200):
            h = 0.5 * (lo + hi)
            P = [np.zeros(3)] + [np.array([math.cos(2 * math.pi * i / n),
                                            math.sin(2 * math.pi * i / n),
                                            h * math.cos(2 * (2 * math.pi * i / n))])
                                  for i in range(n)]
            tot = 0.0
            for i in range(n):
                u = P[1 + i]; w = P[1 + (i + 1) % n]
                tot += math.atan2(np.linalg.norm(np.cross(u, w)), np.dot(u, w))
            if tot < theta:
                lo = h
            else:
                hi = h
        pts = P
        pts = [p if i == 0 else p / np.linalg.norm(p) * slant for i, p in enumerate(pts)]
    X = np.array(pts)
    F = np.array([(0, 1 + i, 1 + (i + 1) % n) for i in range(n)], dtype=np.int32)
    return X, F


def mobius(nu: int, nv: int, R: float = 1.0, w: float = 0.4):
    """Moebius strip: centre circle of radius R, half-width w, nu x nv grid with a half twist;
    the seam joins column nu-1 to column 0 with the width coordinate reversed, so the faces
    across it are oppositely wound (a non-orientable surface with one boundary loop)."""
    X = []
    for i in range(nu):
        u = 2 * np.pi * i / nu
        for j in range(nv):
            t = -w + 2 * w * j / (nv - 1)
            X.append([(R + t * np.cos(u / 2)) * np.cos(u), (R + t * np.cos(u / 2)) * np.sin(u),
                      t * np.sin(u / 2)])
    F = []
    for i in range(nu):
        for j in range(nv - 1):
            a, b = i * nv + j, i * nv + j + 1
            if i + 1 < nu:
                c, d = (i + 1) * nv + j + 1, (i + 1) * nv + j
            else:
                c, d = (nv - 1 - (j + 1)), (nv - 1 - j)
            F += [(a, d, c), (a, c, b)]
    return np.array(X, float), np.array(F, np.int32)


def klein_bottle(nu: int, nv: int, R: float = 2.0):
    """Figure-8 Klein bottle immersion on an nu x nv grid: (u + 2pi, v) is identified with
    (u, -v), so the closing column is glued with v reversed (closed, non-orientable)."""
    X = []
    for i in range(nu):
        u = 2 * np.pi * i / nu
        for j in range(nv):
            v = 2 * np.pi * j / nv
            r = R + np.cos(u / 2) * np.sin(v) - np.sin(u / 2) * np.sin(2 * v)
            X.append([r * np.cos(u), r * np.sin(u), np.sin(u / 2) * np.sin(v) + np.cos(u / 2) * np.sin(2 * v)])
    F = []
    for i in range(nu):
        for j in range(nv):
            a, b = i * nv + j, i * nv + (j + 1) % nv
            if i + 1 < nu:
                c, d = (i + 1) * nv + (j + 1) % nv, (i + 1) * nv + j
            else:
                c, d = (nv - (j + 1)) % nv, (nv - j) % nv
            F += [(a, d, c), (a, c, b)]
    return np.array(X, float), np.array(F, np.int32)


# --------------------------------------------------------------------------- queries
def face_areas(X, F):
    e1 = X[F[:, 1]] - X[F[:, 0]]
    e2 = X[F[:, 2]] - X[F[:, 0]]
    return 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)


def bbox_diag(X):
    return float(np.linalg.norm(X.max(0) - X.min(0)))


def _tangent_frame(X, F, face):
    x0, x1, x2 = X[F[face, 0]], X[F[face, 1]], X[F[face, 2]]
    e1 = x1 - x0
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    n = np.cross(x1 - x0, x2 - x0)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    e2 = np.cross(n, e1)
    return e1, e2


@dataclass
class Queries:
    """A batch of exponential-map queries.

    face   int32[Q]     start face (local to its mesh)
    bary   f64[Q,3]     barycentric point (b_u, b_v, b_w) on the start face
    v      f64[Q,3]     ambient tangent vector, |v| = geodesic length
    w      f64[Q,k,3]   carried unit tangent vectors (k may be 0)
    g_pos  f64[Q,3]     upstream gradient of the end point (for backward tests)
    mesh_id int32[Q]    mesh of each query (multi-mesh batches), or None
    """
    face: np.ndarray
    bary: np.ndarray
    v: np.ndarray
    w: np.ndarray
    g_pos: np.ndarray
    mesh_id: np.ndarray | None = None

    def __len__(self):
        return len(self.face)

    def take(self, idx):
        return Queries(self.face[idx], self.bary[idx], self.v[idx], self.w[idx], self.g_pos[idx],
                       None if self.mesh_id is None else self.mesh_id[idx])


def sample_queries(X, F, nq: int, rng: np.random.Generator, L_lo: float, L_hi: float,
                   n_w: int = 1) -> Queries:
    """Area-weighted start faces; barycentrics uniform on the simplex
    (1-sqrt r1, sqrt r1 (1-r2), sqrt r1 r2); direction angle phi ~ U[0, 2pi) measured
    from e1 = (x1-x0)/|x1-x0| toward e2 = n x e1; length ~ U[L_lo, L_hi]; carried unit
    tangents at angles ~ U[0, 2pi); upstream gradient ~ N(0, I)."""
    A = face_areas(X, F)
    cdf = np.cumsum(A)
    cdf /= cdf[-1]
    face = np.searchsorted(cdf, rng.random(nq), side="right").astype(np.int32)
    face = np.minimum(face, len(F) - 1)
    r1 = rng.random(nq)
    r2 = rng.random(nq)
    s1 = np.sqrt(r1)
    bary = np.stack([1 - s1, s1 * (1 - r2), s1 * r2], 1)
    phi = rng.uniform(0.0, 2 * np.pi, nq)
    L = rng.uniform(L_lo, L_hi, nq)
    e1, e2 = _tangent_frame(X, F, face)
    d = np.cos(phi)[:, None] * e1 + np.sin(phi)[:, None] * e2
    v = L[:, None] * d
    w = np.zeros((nq, n_w, 3))
    for k in range(n_w):
        psi = rng.uniform(0.0, 2 * np.pi, nq)
        w[:, k] = np.cos(psi)[:, None] * e1 + np.sin(psi)[:, None] * e2
    g = rng.normal(0.0, 1.0, (nq, 3))
    return Queries(face, bary, v, w, g)


# --------------------------------------------------------------------------- workloads
@dataclass
class Workload:
    name: str
    meshes: list  # list of (X f64[N,3], F i32[F,3])
    queries: Queries
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def single(self):
        assert len(self.meshes) == 1
        return self.meshes[0]


def _mesh_kind_for(m: int, Fm: int, rng):
    kind = m % 3
    if kind == 0:  # icosphere with F nearest to Fm
        s = int(round(math.log(Fm / 20.0, 4)))
        s = max(1, min(8, s))
        return icosphere(s), f"icosphere s{s}"
    if kind == 1:  # torus grid a x b with 2ab ~ Fm, a/b = 2
        b = max(3, int(round(math.sqrt(Fm / 4.0))))
        a = 2 * b
        return torus(a, b), f"torus {a}x{b}"
    n = max(3, int(round(math.sqrt(Fm / 2.0)))) + 1
    X, F, _ = heightfield(n, rng)
    return (X, F), f"heightfield {n}x{n}"


def workload(index: int, scale: float = 1.0) -> Workload:
    """The five synthetic workloads (index 0..4).  `scale` < 1 shrinks the query count
    (mesh unchanged) for CPU-side checks; scale = 1 gives the full sizes.

    0 icosphere s3 (642 V, 1280 F), 4096 queries, L ~ U[0, pi], 1 carried vector
    1 torus R=1 r=0.4 512x256 (262,144 F), noise 0.002, 4M queries, L ~ U[0, 2], 2 vectors
    2 noisy icosphere s6 (81,920 F, radial 0.003), 1M queries, L ~ U[0.1, 1.0]
    3 64 uneven meshes (icosphere/torus/heightfield, F log-uniform [1e3, 5e5]),
      q_m = clamp(2 F_m, 1e3, 1e6), L ~ U[0, 0.5 diag_m]
    4 heightfield 1449^2 (4,193,408 F) with 10% sliver jitter, 16M queries, L ~ U[0, 3 diag]
    """
    rng = rng_for(index)
    if index == 0:
        X, F = icosphere(3)
        q = sample_queries(X, F, max(1, int(4096 * scale)), rng, 0.0, math.pi, 1)
        return Workload("icosphere-s3 1280F 4096q", [(X, F)], q)
    if index == 1:
        X, F = torus(512, 256, 1.0, 0.4, 0.002, rng)
        q = sample_queries(X, F, max(1, int(4194304 * scale)), rng, 0.0, 2.0, 2)
        return Workload("torus-512x256 262144F 4Mq 2w", [(X, F)], q)
    if index == 2:
        X, F = icosphere(6, 0.003, rng)
        q = sample_queries(X, F, max(1, int(1048576 * scale)), rng, 0.1, 1.0, 0)
        return Workload("icosphere-s6-noisy 81920F 1Mq fwd+bwd", [(X, F)], q)
    if index == 3:
        meshes, qs, names = [], [], []
        Fm = np.round(np.exp(rng.uniform(math.log(1e3), math.log(5e5), 64))).astype(int)
        for m in range(64):
            (X, F), nm = _mesh_kind_for(m, int(Fm[m]), rng)
            meshes.append((X, F))
            names.append(nm)
        for m, (X, F) in enumerate(meshes):
            qm = int(np.clip(2 * len(F), 1e3, 1e6))
            qm = max(1, int(qm * scale))
            q = sample_queries(X, F, qm, rng, 0.0, 0.5 * bbox_diag(X), 0)
            q.mesh_id = np.full(qm, m, np.int32)
            qs.append(q)
        cat = Queries(np.concatenate([q.face for q in qs]), np.concatenate([q.bary for q in qs]),
                      np.concatenate([q.v for q in qs]), np.concatenate([q.w for q in qs]),
                      np.concatenate([q.g_pos for q in qs]),
                      np.concatenate([q.mesh_id for q in qs]))
        return Workload("64 uneven meshes", meshes, cat, extra={"names": names})
    if index == 4:
        n = 1449
        X, F, waves = heightfield(n, rng)
        X = jitter_slivers(X, n, rng, 0.10, waves)
        d = bbox_diag(X)
        q = sample_queries(X, F, max(1, int(16777216 * scale)), rng, 0.0, 3 * d, 0)
        return Workload("heightfield-1449 4193408F slivers 16Mq", [(X, F)], q)
    raise ValueError(index)


WORKLOADS = {0: "icosphere-s3", 1: "torus-262k", 2: "icosphere-s6-noisy", 3: "multi-mesh-64",
             4: "heightfield-slivers"}
