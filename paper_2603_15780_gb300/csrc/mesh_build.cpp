// mesh_build.cpp -- host construction of the packed walk records (FP64 arithmetic).
//
// Sec. 4: a mesh M = {X, F} is manifold when each edge has one or two faces and the
// faces around each vertex form one fan; points are (face, barycentric) pairs; the
// total angle theta(x) at a vertex is the sum of incident corner angles.  App. "Main
// differences with SotA implementation": only triangle adjacencies are stored (no
// half-edges), so non-orientable meshes are accepted; the orientation of each
// adjacency is kept as one "flip" bit so the intrinsic walk can unfold consistently.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include <cuda_runtime.h>

#include "sgeo_internal.h"

namespace {

struct D3 {
    double x, y, z;
};
inline D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline D3 cross(D3 a, D3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(D3 a) { return std::sqrt(dot(a, a)); }
inline D3 scale(D3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }

inline int bits(float f) {
    int i;
    std::memcpy(&i, &f, 4);
    return i;
}

// 21 bits of x spread to every third bit of a 63-bit Z-order (Morton) code
inline uint64_t spread3(uint64_t x) {
    x &= 0x1fffffULL;
    x = (x | (x << 32)) & 0x1f00000000ffffULL;
    x = (x | (x << 16)) & 0x1f0000ff0000ffULL;
    x = (x | (x << 8)) & 0x100f00f00f00f00fULL;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ULL;
    x = (x | (x << 2)) & 0x1249249249249249ULL;
    return x;
}

// The spatial rank of the faces of one mesh: their order along the Z-order curve of the face
// centroids in the mesh's bounding cube (ties by face id), offset by the mesh's first face.  It
// orders queries by start face so that a warp's walks start in one patch of the surface.
void spatial_ranks(const float *V, const int32_t *Fm, int64_t v0, int64_t f0, int64_t nf, int32_t *rank) {
    std::vector<double> c(3 * nf);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t f = 0; f < nf; ++f)
        for (int k = 0; k < 3; ++k) {
            const double x = ((double)V[3 * (v0 + Fm[3 * f]) + k] + (double)V[3 * (v0 + Fm[3 * f + 1]) + k] +
                              (double)V[3 * (v0 + Fm[3 * f + 2]) + k]) / 3.0;
            c[3 * f + k] = x;
            lo[k] = std::min(lo[k], x);
            hi[k] = std::max(hi[k], x);
        }
    // one scale for the three axes (the largest extent), so that a thin dimension (a heightfield's
    // z) takes few of the curve's bits and the order follows the surface
    const double span = std::max(std::max(hi[0] - lo[0], hi[1] - lo[1]), hi[2] - lo[2]);
    std::vector<uint64_t> key(nf);
    for (int64_t f = 0; f < nf; ++f) {
        uint64_t code = 0;
        for (int k = 0; k < 3; ++k) {
            const double t = span > 0.0 ? (c[3 * f + k] - lo[k]) / span : 0.0;
            const uint64_t q = (uint64_t)std::min(std::max(t * 2097151.0, 0.0), 2097151.0);
            code |= spread3(q) << k;
        }
        key[f] = code;
    }
    std::vector<int64_t> idx(nf);
    std::iota(idx.begin(), idx.end(), (int64_t)0);
    std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return key[a] < key[b] || (key[a] == key[b] && a < b); });
    for (int64_t r = 0; r < nf; ++r) rank[idx[r]] = (int32_t)(f0 + r);
}

struct EdgeKey {
    int32_t a, b;  // a < b, local vertex ids
    int32_t f;     // local face
    int8_t k;      // local edge: corner k -> corner k+1
};

}  // namespace

sg_status sg_build_host_mesh(const float *V, const int64_t *v_off, const int32_t *F, const int64_t *f_off,
                             int32_t n_mesh, sg_host_mesh *out) {
    if (!V || !v_off || !F || !f_off || n_mesh <= 0) return SG_ERR_INVALID_ARG;
    if (v_off[0] != 0 || f_off[0] != 0) return SG_ERR_INVALID_ARG;
    for (int m = 0; m < n_mesh; ++m)
        if (v_off[m + 1] <= v_off[m] || f_off[m + 1] <= f_off[m]) return SG_ERR_INVALID_ARG;
    const int64_t nV = v_off[n_mesh], nF = f_off[n_mesh];
    if (nF >= SG_MAX_FACES || nV >= (1LL << 31)) return SG_ERR_INVALID_ARG;

    out->rec.assign(2 * nF, int4{0, 0, 0, 0});
    out->fv.assign(nF, int4{0, 0, 0, 0});
    out->frm.assign(2 * nF, float4{0, 0, 0, 0});
    out->half.assign(6 * nF, int4{0, 0, 0, 0});
    out->edges.clear();
    out->edges.reserve((size_t)(1.5 * nF) + 16);
    out->srank.assign(nF, 0);
    out->V.assign(nV, float4{0, 0, 0, 0});
    out->face_off.assign(n_mesh + 1, 0);
    out->lref.assign(n_mesh, 0.f);
    out->lref64.assign(n_mesh, 0.0);
    out->face_off64.assign(f_off, f_off + n_mesh + 1);
    out->vert_off64.assign(v_off, v_off + n_mesh + 1);
    for (int m = 0; m <= n_mesh; ++m) out->face_off[m] = (int32_t)f_off[m];

    std::vector<double> theta(nV, 0.0);
    std::vector<uint8_t> boundary(nV, 0);

    for (int m = 0; m < n_mesh; ++m) {
        const int64_t v0 = v_off[m], nv = v_off[m + 1] - v0;
        const int64_t f0 = f_off[m], nf = f_off[m + 1] - f0;
        auto X = [&](int32_t lv) { const float *p = V + 3 * (v0 + lv); return D3{p[0], p[1], p[2]}; };
        const int32_t *Fm = F + 3 * f0;
        for (int64_t i = 0; i < 3 * nf; ++i)
            if (Fm[i] < 0 || Fm[i] >= nv) return SG_ERR_INVALID_ARG;

        // ---- per-face intrinsic shape in the face's own 2-D frame
        for (int64_t f = 0; f < nf; ++f) {
            const int32_t *t = Fm + 3 * f;
            if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2]) return SG_ERR_DEGENERATE;
            D3 x0 = X(t[0]), x1 = X(t[1]), x2 = X(t[2]);
            D3 e1 = sub(x1, x0), e2 = sub(x2, x0);
            D3 n = cross(e1, e2);
            double l01 = norm(e1), nn = norm(n);
            if (!(nn > 1e-14 * std::max(dot(e1, e1), dot(e2, e2)))) return SG_ERR_DEGENERATE;
            D3 u = scale(e1, 1.0 / l01);
            D3 nh = scale(n, 1.0 / nn);
            D3 w = cross(nh, u);
            double x2x = dot(e2, u), x2y = dot(e2, w);
            double l12 = norm(sub(x2, x1)), l20 = norm(e2);
            int4 &r1 = out->rec[2 * (f0 + f) + 1];
            r1.x = bits((float)x2x);
            r1.y = bits((float)x2y);
            r1.z = bits((float)(1.0 / l12));
            r1.w = bits((float)(1.0 / l20));
            out->rec[2 * (f0 + f)].w = bits((float)l01);
            out->fv[f0 + f] = int4{(int)(v0 + t[0]), (int)(v0 + t[1]), (int)(v0 + t[2]), m};
            out->frm[2 * (f0 + f)] = float4{(float)u.x, (float)u.y, (float)u.z, (float)w.x};
            out->frm[2 * (f0 + f) + 1] = float4{(float)w.y, (float)w.z, 0.f, 0.f};
            // corner angles -> theta
            for (int k = 0; k < 3; ++k) {
                D3 a = sub(X(t[(k + 1) % 3]), X(t[k])), b = sub(X(t[(k + 2) % 3]), X(t[k]));
                theta[v0 + t[k]] += std::atan2(norm(cross(a, b)), dot(a, b));
            }
        }

        // ---- edge matching: sort the 3 nf half-edges by (min, max) vertex
        std::vector<EdgeKey> E(3 * nf);
        for (int64_t f = 0; f < nf; ++f)
            for (int k = 0; k < 3; ++k) {
                int32_t a = Fm[3 * f + k], b = Fm[3 * f + (k + 1) % 3];
                E[3 * f + k] = EdgeKey{std::min(a, b), std::max(a, b), (int32_t)f, (int8_t)k};
            }
        std::sort(E.begin(), E.end(), [](const EdgeKey &p, const EdgeKey &q) {
            if (p.a != q.a) return p.a < q.a;
            if (p.b != q.b) return p.b < q.b;
            if (p.f != q.f) return p.f < q.f;
            return p.k < q.k;
        });
        double lsum = 0.0;
        int64_t ne = 0;
        std::vector<int32_t> nbr(3 * nf, -1);
        std::vector<int32_t> hedge(3 * nf, -1);  // (edge id << 1) | non-canonical, per half-edge
        for (size_t i = 0; i < E.size();) {
            size_t j = i + 1;
            while (j < E.size() && E[j].a == E[i].a && E[j].b == E[i].b) ++j;
            if (j - i > 2) return SG_ERR_NONMANIFOLD;
            lsum += norm(sub(X(E[i].a), X(E[i].b)));
            ++ne;
            if (j - i == 2) {
                const EdgeKey &p = E[i], &q = E[i + 1];
                if (p.f == q.f) return SG_ERR_NONMANIFOLD;
                // same direction in both faces -> inconsistent orientation across this edge
                int32_t pa = Fm[3 * p.f + p.k], qa = Fm[3 * q.f + q.k];
                int flip = (pa == qa) ? 1 : 0;
                int64_t gq = f0 + q.f, gp = f0 + p.f;
                nbr[3 * p.f + p.k] = (int32_t)((gq << 3) | (flip << 2) | q.k);
                nbr[3 * q.f + q.k] = (int32_t)((gp << 3) | (flip << 2) | p.k);
                int64_t hp = 3 * gp + p.k, hq = 3 * gq + q.k;
                int64_t eid = (int64_t)out->edges.size();
                out->edges.push_back(int2{(int)std::min(hp, hq), (int)std::max(hp, hq)});
                hedge[3 * p.f + p.k] = (int32_t)((eid << 1) | (hp > hq ? 1 : 0));
                hedge[3 * q.f + q.k] = (int32_t)((eid << 1) | (hq > hp ? 1 : 0));
            } else {
                boundary[v0 + E[i].a] = 1;
                boundary[v0 + E[i].b] = 1;
            }
            i = j;
        }
        for (int64_t f = 0; f < nf; ++f) {
            int4 &r0 = out->rec[2 * (f0 + f)];
            r0.x = nbr[3 * f];
            r0.y = nbr[3 * f + 1];
            r0.z = nbr[3 * f + 2];
        }
        // ---- half-edge records: each face seen from each of its edges
        for (int64_t f = 0; f < nf; ++f) {
            const int32_t *t = Fm + 3 * f;
            D3 x0 = X(t[0]), x1 = X(t[1]), x2 = X(t[2]);
            D3 e1 = sub(x1, x0), e2 = sub(x2, x0);
            double l01 = norm(e1);
            D3 u = scale(e1, 1.0 / l01);
            D3 nh = scale(cross(e1, e2), 1.0 / norm(cross(e1, e2)));
            D3 w = cross(nh, u);
            double Px[3] = {0.0, l01, dot(e2, u)}, Py[3] = {0.0, 0.0, dot(e2, w)};
            for (int k = 0; k < 3; ++k) {
                int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                double ex = Px[k1] - Px[k], ey = Py[k1] - Py[k];
                double l = std::sqrt(ex * ex + ey * ey);
                double ca = ex / l, sa = ey / l;
                double rx = Px[k2] - Px[k], ry = Py[k2] - Py[k];
                double cx = rx * ca + ry * sa, cy = -rx * sa + ry * ca;
                auto link = [&](int edge) -> int32_t {
                    int32_t nb = nbr[3 * f + edge];
                    if (nb < 0) return -1;
                    int64_t g = nb >> 3;
                    int kp = nb & 3, fl = (nb >> 2) & 1;
                    return (int32_t)(((3 * g + kp) << 1) | fl);
                };
                int64_t h = 3 * (f0 + f) + k;
                out->half[2 * h] = int4{bits((float)l), bits((float)cx), bits((float)cy), link(k1)};
                out->half[2 * h + 1] = int4{link(k2), bits((float)ca), bits((float)sa), hedge[3 * f + k]};
            }
        }
        out->lref64[m] = lsum / (double)ne;
        out->lref[m] = (float)out->lref64[m];

        // ---- single-fan check: walking around each vertex through the adjacency must
        //      reach all of its incident faces
        std::vector<int32_t> deg(nv, 0), any(nv, -1);
        for (int64_t f = 0; f < nf; ++f)
            for (int k = 0; k < 3; ++k) {
                deg[Fm[3 * f + k]]++;
                any[Fm[3 * f + k]] = (int32_t)f;
            }
        for (int64_t v = 0; v < nv; ++v) {
            if (deg[v] == 0) continue;
            int64_t seen = 1;
            for (int dir = 0; dir < 2; ++dir) {
                int64_t f = any[v];
                const int32_t *t = Fm + 3 * f;
                int c = t[0] == v ? 0 : t[1] == v ? 1 : 2;
                // edges at corner c: local edge c (c -> c+1) and local edge c+2 (c+2 -> c)
                int e = dir == 0 ? c : (c + 2) % 3;
                for (int guard = 0; guard <= deg[v]; ++guard) {
                    int32_t nb = nbr[3 * f + e];
                    if (nb < 0) break;
                    int64_t g = (nb >> 3) - f0;
                    if (g == any[v]) break;
                    ++seen;
                    int kp = nb & 3;
                    const int32_t *tg = Fm + 3 * g;
                    int cg = tg[0] == v ? 0 : tg[1] == v ? 1 : 2;
                    // the other edge of g at corner cg
                    e = (kp == cg) ? (cg + 2) % 3 : cg;
                    f = g;
                }
                if (!boundary[v0 + v]) break;
            }
            if (seen != deg[v]) return SG_ERR_NONMANIFOLD;
        }
    }
    for (int64_t v = 0; v < nV; ++v) {
        const float *p = V + 3 * v;
        float th = (float)theta[v];
        out->V[v] = float4{p[0], p[1], p[2], boundary[v] ? -th : th};
    }
    for (int m = 0; m < n_mesh; ++m)
        spatial_ranks(V, F + 3 * f_off[m], v_off[m], f_off[m], f_off[m + 1] - f_off[m], out->srank.data() + f_off[m]);
    return SG_OK;
}
