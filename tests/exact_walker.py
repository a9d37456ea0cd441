"""Exact rational straight-line walker for polycube surfaces (a pin for the oracle).

On a polycube every face is an axis-aligned unit-square half, so unfolding across an
edge is either the identity (coplanar neighbour) or a quarter turn about an axis-
aligned edge, and every quantity stays rational.  This walker therefore produces the
exact face sequence and end point of a straightest geodesic that touches no vertex,
with `fractions.Fraction` arithmetic and brute-force neighbour search, independent of
the floating-point oracle.  Rays that meet a vertex exactly return None (vertex hits
are pinned separately by the cone closed form and the hand-worked cube examples).
"""
from __future__ import annotations

from fractions import Fraction as Q


def _sub(a, b):
    return tuple(x - y for x, y in zip(a, b))


def _dot(a, b):
    return sum(x * y for x, y in zip(a, b))


def _add(a, b, s=1):
    return tuple(x + s * y for x, y in zip(a, b))


def _scale(a, s):
    return tuple(x * s for x in a)


class Polycube:
    def __init__(self, X, F):
        self.X = [tuple(Q(int(round(c))) for c in x) for x in X]
        self.F = [tuple(int(i) for i in f) for f in F]
        self.edge_faces: dict[frozenset, list[int]] = {}
        for fi, f in enumerate(self.F):
            for k in range(3):
                e = frozenset((f[k], f[(k + 1) % 3]))
                self.edge_faces.setdefault(e, []).append(fi)
        # constant axis of each face (its plane is axis-aligned)
        self.axis = []
        for f in self.F:
            pts = [self.X[i] for i in f]
            ax = [a for a in range(3) if pts[0][a] == pts[1][a] == pts[2][a]]
            assert len(ax) == 1
            self.axis.append(ax[0])

    def _in_plane_normal(self, fi, a, b):
        """Unit in-plane normal of edge (a, b) pointing into face fi; exact because the
        edge of a non-coplanar fold is axis-aligned."""
        third = [i for i in self.F[fi] if i not in (a, b)][0]
        xa, xb, xc = self.X[a], self.X[b], self.X[third]
        e = _sub(xb, xa)
        t = _sub(xc, xa)
        ee = _dot(e, e)
        u = _add(t, e, -_dot(t, e) / ee)
        nz = [c for c in u if c != 0]
        assert len(nz) == 1, "fold edge must be axis-aligned"
        return tuple(Q(0) if c == 0 else Q(1 if c > 0 else -1) for c in u)

    def walk(self, face, bary, d, t_total, max_steps=10000, points=False):
        """Walk from point sum(bary * corners) on `face` along d for parameter t_total
        (length = t_total * |d|).  Returns (faces, end_point) or None on a vertex hit; with
        points=True, (faces, end_point, entry_points): the exact point at which the walk
        enters each face of `faces` (the start point, then each edge crossing)."""
        f = face
        p = tuple(sum(Q(b) * self.X[i][c] for b, i in zip(bary, self.F[f])) for c in range(3))
        d = tuple(Q(x) for x in d)
        t_rem = Q(t_total)
        faces = [f]
        pts = [p]
        entry = None
        for _ in range(max_steps):
            best = None
            tri = self.F[f]
            for k in range(3):
                a, b = tri[k], tri[(k + 1) % 3]
                if entry is not None and frozenset((a, b)) == entry:
                    continue
                xa, xb = self.X[a], self.X[b]
                e = _sub(xb, xa)
                # solve p + t d = xa + s e in the face's plane (drop the constant axis)
                ax = [c for c in range(3) if c != self.axis[f]]
                m00, m01 = d[ax[0]], -e[ax[0]]
                m10, m11 = d[ax[1]], -e[ax[1]]
                r0, r1 = xa[ax[0]] - p[ax[0]], xa[ax[1]] - p[ax[1]]
                det = m00 * m11 - m01 * m10
                if det == 0:
                    continue
                t = (r0 * m11 - m01 * r1) / det
                s = (m00 * r1 - r0 * m10) / det
                if t < 0 or s < 0 or s > 1:
                    continue
                if t == 0 and entry is None:
                    # starting on this edge: only leave through it if d points outward
                    pass
                if best is None or t < best[0]:
                    best = (t, s, a, b)
            if best is None:
                return None
            t, s, a, b = best
            if t >= t_rem:
                return (faces, _add(p, d, t_rem), pts) if points else (faces, _add(p, d, t_rem))
            if s == 0 or s == 1:
                return None  # exact vertex hit
            p = _add(p, d, t)
            t_rem -= t
            nbrs = [g for g in self.edge_faces[frozenset((a, b))] if g != f]
            if not nbrs:
                return (faces, p, pts) if points else (faces, p)  # boundary (closed polycubes have none)
            g = nbrs[0]
            if self.axis[g] != self.axis[f] or self.X[self.F[g][0]][self.axis[g]] != self.X[tri[0]][self.axis[f]]:
                e = _sub(self.X[b], self.X[a])
                ee = _dot(e, e)
                uf = self._in_plane_normal(f, a, b)
                ug = self._in_plane_normal(g, a, b)
                de = _dot(d, e) / ee
                du = _dot(d, uf)
                d = _add(_scale(e, de), ug, -du)
            f = g
            entry = frozenset((a, b))
            faces.append(f)
            pts.append(p)
        return None
