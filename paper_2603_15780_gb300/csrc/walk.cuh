// walk.cuh -- device-side straightest-geodesic walker (intrinsic 2-D formulation).
//
// The paper walks in 3-D (Alg. geodesic_step, transport_over_edge, transport_over_vertex,
// App. "Implementation of the Geodesic Step").  Here each face carries its own 2-D frame
// (corner 0 at the origin, corner 1 on +x); a crossing maps the walker rigidly from the
// frame of f to the frame of its neighbour g through the shared edge, which is the
// unfolding isometry of Sec. 4 ("the neighbourhood of a point on an edge is isometric to a
// plane").  Per crossing the walker reads ONE 32-byte record (the face it enters).
//
// Decisions are orientation tests sigma_i = cross(d, P_i - p) = signed distance from the ray
// line to corner i: the exit edge is the one whose endpoints have sigma of opposite sign, and
// a vertex is hit when |sigma| <= tau_snap * l_ref.  When |sigma| < tau_near * l_ref the tests
// are re-evaluated in FP64 (ESC = true) and the query is flagged NEAR_VERTEX.
//
// Carried tangent vectors are kept as their (cos, sin) components relative to the walking
// direction: parallel transport holds the angle to the curve tangent constant (Sec. 4
// "Parallel Transport"), so they are rebuilt only at the end.  A parity bit records crossings
// of inconsistently oriented edges (non-orientable meshes) where the signed angle flips.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sgeo_internal.h"

#define SG_PARITY_BIT 0x80000000u
#define SG_FNV_OFFSET 0xcbf29ce484222325ULL
#define SG_FNV_PRIME 0x100000001b3ULL

struct FaceRec {
    int n0, n1, n2;
    float l01, x2x, x2y, il1, il2;
};

// One 32-byte record = one L2 sector, read as two 16-byte loads or, with W, as one 256-bit
// load (sm_100 and later).  The wide load halves the L2 requests per record and doubles the
// device's dependent-gather ceiling; the half-edge record of every crossing is read with it
// (1M queries on an 81,920-face sphere, queries in walk-length order: forward walk 0.437 ->
// 0.404 ms, backward re-walk 0.738 -> 0.716 ms, whose L2 tag lookups had run at 74% with two
// 16-byte loads and an atomic per crossing).
template <bool W = false>
__device__ __forceinline__ void ld_rec32(const int4 *__restrict__ p, int4 &a, int4 &b) {
    if (W) {
        asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
            : "l"(p));
    } else {
        a = __ldg(p);
        b = __ldg(p + 1);
    }
}

template <bool W = false>
__device__ __forceinline__ FaceRec load_rec(const int4 *__restrict__ rec, int f) {
    int4 a, b;
    ld_rec32<W>(rec + 2 * f, a, b);
    FaceRec r;
    r.n0 = a.x; r.n1 = a.y; r.n2 = a.z;
    r.l01 = __int_as_float(a.w);
    r.x2x = __int_as_float(b.x); r.x2y = __int_as_float(b.y);
    r.il1 = __int_as_float(b.z); r.il2 = __int_as_float(b.w);
    return r;
}

template <class T>
__device__ __forceinline__ T sel3(int k, T a, T b, T c) { return k == 0 ? a : (k == 1 ? b : c); }
__device__ __forceinline__ int nbr_of(const FaceRec &r, int k) { return sel3(k, r.n0, r.n1, r.n2); }
__device__ __forceinline__ float corner_x(const FaceRec &r, int k) { return sel3(k, 0.f, r.l01, r.x2x); }
__device__ __forceinline__ float corner_y(const FaceRec &r, int k) { return sel3(k, 0.f, 0.f, r.x2y); }
__device__ __forceinline__ float inv_len(const FaceRec &r, int k) { return sel3(k, __frcp_rn(r.l01), r.il1, r.il2); }
// half-edge record view of the same 8 words: l, cx, cy, linkR | linkL, ca, sa, -
__device__ __forceinline__ float hl(const FaceRec &r) { return __int_as_float(r.n0); }
__device__ __forceinline__ float hcx(const FaceRec &r) { return __int_as_float(r.n1); }
__device__ __forceinline__ float hcy(const FaceRec &r) { return __int_as_float(r.n2); }
__device__ __forceinline__ int hlinkR(const FaceRec &r) { return __float_as_int(r.l01); }
__device__ __forceinline__ int hlinkL(const FaceRec &r) { return __float_as_int(r.x2x); }
__device__ __forceinline__ float hca(const FaceRec &r) { return r.x2y; }
__device__ __forceinline__ float hsa(const FaceRec &r) { return r.il1; }
__device__ __forceinline__ int nxt(int k) { return k == 2 ? 0 : k + 1; }
__device__ __forceinline__ int prv(int k) { return k == 0 ? 2 : k - 1; }

struct WalkParams {
    const int4 *__restrict__ rec;
    const int4 *__restrict__ half;
    const int4 *__restrict__ fv;
    const float4 *__restrict__ frm;
    const float4 *__restrict__ V;
    const int32_t *__restrict__ face_off;
    const float *__restrict__ lref;
    int max_steps;
    float tau_near, tau_snap;
    int want_hash;
    // the mixed walk's double-float half-edge records and FP64 face axes (NULL elsewhere)
    const int4 *__restrict__ half48;
    const double *__restrict__ frm64;
};

// Walker state (all registers).  mode 7: on the entry edge of half-edge h (the hot case; R
// holds the half-edge record, (px, py) = (fraction s along the edge, 0), d in the edge
// frame; f is stale and recomputed as h / 3 on leaving this mode); modes 0..2 entered through local edge `mode`, 3..5 sitting on corner mode-3 after a
// vertex transport, 6 free start -- in these R holds the face record and p, d are in the face
// frame.  Every walk ends in a face mode.
#define SG_MODE_HALF 7
// hole avoidance: the walk reached the boundary on local edge mode-8 (at p) or on corner
// mode-11 of face f, and the boundary handling is pending (see hole_resolve)
#define SG_MODE_HOLE_EDGE 8
#define SG_MODE_HOLE_VERTEX 11
struct Walker {
    int f, h, mode, steps, ncross;
    float px, py, dx, dy;
    float Lh, Ll;        // remaining length as an unevaluated sum (compensated subtraction)
    uint32_t st;         // SG_ST_* | parity
    int foff;            // face offset of the query's mesh (hash uses local ids)
    float lref;
    uint64_t hash;
    FaceRec R;
    float dxl, dyl;      // mixed walk: low parts of the direction (double-float d = dx + dxl, ...)
};

__device__ __forceinline__ float sigma32(float dx, float dy, float cx, float cy, float px, float py) {
    // cross(d, C - p): signed distance of corner C from the ray line (d is unit)
    return fmaf(dx, cy - py, -dy * (cx - px));
}
__device__ __forceinline__ double sigma64(float dx, float dy, float cx, float cy, float px, float py) {
    return (double)dx * ((double)cy - (double)py) - (double)dy * ((double)cx - (double)px);
}

// FP64 -> FP32 keeping the sign of tiny values (a sign decides the exit edge)
__device__ __forceinline__ float f32_keep_sign(double x) {
    float f = (float)x;
    if (f == 0.f && x != 0.0) f = x > 0.0 ? 1.17549435e-38f : -1.17549435e-38f;
    return f;
}

__device__ __forceinline__ void walker_hash(Walker &w, int f, int want) {
    if (want) {
        w.hash ^= (uint64_t)(uint32_t)(f - w.foff);
        w.hash *= SG_FNV_PRIME;
    }
}

__device__ __forceinline__ void renorm(float &x, float &y) {
    float n2 = fmaf(x, x, y * y);
    float r = rsqrtf(n2);
    r = r * fmaf(-0.5f * n2 * r, r, 1.5f);  // one Newton step
    x *= r; y *= r;
}

// ------------------------------------------------------------------ double-float arithmetic
// Error-free transformations: Knuth's two-sum (TAOCP vol. 2, sec. 4.2.2), Dekker's fast two-sum
// (Dekker 1971, |a| >= |b|) and the exact product by one fused multiply-add.  Built on them, the
// double-float sum, product and quotient keep about 2^-46 relative error.  Each function below
// has a float32 numpy twin of the same name, operation for operation, in
// tests/test_double_float_arith.py, which checks these error bounds on the CPU; a change here
// goes there too.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return DF{s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = a * b;
    return DF{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
// the sum with both parts summed exactly: accurate under cancellation (c - x near a vertex)
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    const DF t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }
// the sum of two terms of equal sign (no cancellation): one two-sum of the high parts suffices
__device__ __forceinline__ DF df_add_same_sign(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    DF p = two_prod(a.hi, b.hi);
    p.lo = fmaf(a.hi, b.lo, p.lo);
    p.lo = fmaf(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    DF p = two_prod(a.hi, b);
    p.lo = fmaf(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
// quotient by long division: two FP32 quotient digits (the second from the remainder, formed
// in double-float) with one correctly rounded reciprocal of the divisor's high part
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float rb = __frcp_rn(b.hi);
    const float q1 = a.hi * rb;
    const DF r = df_sub(a, df_mul_f(b, q1));
    return fast_two_sum(q1, r.hi * rb);
}
// 1/sqrt(n): the FP32 estimate refined by one Newton step r + r (1 - n r^2) / 2, which squares
// its relative error
__device__ __forceinline__ DF df_rsqrt(DF n) {
    const float r = rsqrtf(n.hi);
    const DF e = df_sub(DF{1.f, 0.f}, df_mul(n, two_prod(r, r)));
    return fast_two_sum(r, 0.5f * r * e.hi);
}
__device__ __forceinline__ DF df_from(double x) {
    const float hi = (float)x;
    return DF{hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ bool df_ge(DF a, DF b) { return a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo); }
// a double-float pair in one double register pair (the low word holds hi), so the half-edge mode
// reuses the FP64 state's registers
__device__ __forceinline__ double dpack(DF a) { return __hiloint2double(__float_as_int(a.lo), __float_as_int(a.hi)); }
__device__ __forceinline__ DF dunpack(double d) {
    return DF{__int_as_float(__double2loint(d)), __int_as_float(__double2hiint(d))};
}

// a b + c d in double-float: the two exact products summed by one two-sum, all cross terms and
// rounding errors gathered into the low part
__device__ __forceinline__ DF df_dot2(DF a, DF b, DF c, DF d) {
    const DF p = two_prod(a.hi, b.hi), q = two_prod(c.hi, d.hi);
    DF s = two_sum(p.hi, q.hi);
    float lo = s.lo + (p.lo + q.lo);
    lo = fmaf(a.hi, b.lo, lo);
    lo = fmaf(a.lo, b.hi, lo);
    lo = fmaf(c.hi, d.lo, lo);
    lo = fmaf(c.lo, d.hi, lo);
    return fast_two_sum(s.hi, lo);
}

// ------------------------------------------------------------------ hole avoidance
// Sec. 4 "Straightest geodesics": instead of stopping at the boundary, the walk may trace along
// it and resume as soon as possible with the last straightest direction (App. transport_over_
// vertex / transport_over_edge, hole-avoidance branches).  The paper describes the face choice
// (its transport_error) without defining it; the reading used here:
//   - D is the direction, in 3-D, that the walker had when it reached the boundary;
//   - a face around the boundary vertex receives D when D projected onto its plane points
//     strictly into the face's corner at the vertex; the receiving face of least |D . n_f|
//     is taken and the straightest walk resumes from the vertex inside it;
//   - when no face receives D, the walk follows the boundary to the next boundary vertex,
//     keeping its sense along the boundary (at a vertex hit directly by the ray: the boundary
//     edge whose direction agrees best with D), spending the edge's length;
//   - a decision closer than tau_near is flagged NEAR_VERTEX.
__device__ __forceinline__ void frm_axes(const WalkParams &P, int f, float &e1x, float &e1y, float &e1z, float &e2x,
                                         float &e2y, float &e2z) {
    const float4 a = __ldg(P.frm + 2 * f), b = __ldg(P.frm + 2 * f + 1);
    e1x = a.x; e1y = a.y; e1z = a.z; e2x = a.w; e2y = b.x; e2z = b.y;
}

// The walker sits on corner c of face w.f (a boundary vertex; w.R is the face record).
// Returns true when the walk resumes (walker on a corner of the receiving face), false when
// it ended (length spent along the boundary, or MAX_STEPS).
__device__ __forceinline__ bool hole_vertex(Walker &w, const WalkParams &P, int c, int came_from, float Dx, float Dy,
                                            float Dz) {
    w.st |= SG_ST_HOLE;
    const float tau = P.tau_near;
    for (;;) {
        const int f0 = w.f;
        const FaceRec R0 = w.R;
        const int4 fv0 = __ldg(P.fv + f0);
        const int v0 = sel3(c, fv0.x, fv0.y, fv0.z);
        int bg = -1, bcg = 0;
        unsigned bfl = 0u;
        float bux = 0.f, buy = 0.f, berr = 3.0e38f, serr = 3.0e38f;
        // the boundary edges at v0 (face, corner of v0, corner of the other end, flip), in
        // scalars rather than arrays so that they stay in registers
        int nb = 0, ebf0 = 0, ebc0 = 0, ebo0 = 0, ebf1 = 0, ebc1 = 0, ebo1 = 0;
        unsigned ebfl0 = 0u, ebfl1 = 0u;
        // does face g (record Rg, v0 on its corner cg, orientation fl relative to f0) receive D?
        auto consider = [&](int g, const FaceRec &Rg, int cg, unsigned fl) {
            float e1x, e1y, e1z, e2x, e2y, e2z;
            frm_axes(P, g, e1x, e1y, e1z, e2x, e2y, e2z);
            float ux = Dx * e1x + Dy * e1y + Dz * e1z, uy = Dx * e2x + Dy * e2y + Dz * e2z;
            const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
            const float err = fabsf(Dx * nx + Dy * ny + Dz * nz);
            const float lu = sqrtf(ux * ux + uy * uy);
            if (!(lu > 1e-6f)) return;
            ux /= lu; uy /= lu;
            const float px = corner_x(Rg, cg), py = corner_y(Rg, cg);
            const float ax = corner_x(Rg, nxt(cg)) - px, ay = corner_y(Rg, nxt(cg)) - py;
            const float bx = corner_x(Rg, prv(cg)) - px, by = corner_y(Rg, prv(cg)) - py;
            const float sa = (ax * uy - ay * ux) * rsqrtf(ax * ax + ay * ay);
            const float sb = (ux * by - uy * bx) * rsqrtf(bx * bx + by * by);
            const float mg = fminf(sa, sb);
            if (fabsf(mg) < tau) w.st |= SG_ST_NEAR_VERTEX;
            if (!(mg > 0.f)) return;
            if (err < berr) {
                serr = berr; berr = err; bg = g; bcg = cg; bfl = fl; bux = ux; buy = uy;
            } else if (err < serr) {
                serr = err;
            }
        };
        consider(f0, R0, c, 0u);
        for (int dir = 0; dir < 2; ++dir) {
            int cur = f0, cur_c = c;
            FaceRec Rc = R0;
            unsigned fl = 0u;
            int e = dir == 0 ? c : prv(c);  // local edge c runs c -> c+1, local edge c-1 runs c-1 -> c
            for (int guard = 0; guard < 4096; ++guard) {
                const int nbv = nbr_of(Rc, e);
                if (nbv < 0) {  // boundary edge at v0
                    const int oc = (e == cur_c) ? nxt(e) : e;
                    if (nb == 0) { ebf0 = cur; ebc0 = cur_c; ebo0 = oc; ebfl0 = fl; }
                    else if (nb == 1) { ebf1 = cur; ebc1 = cur_c; ebo1 = oc; ebfl1 = fl; }
                    ++nb;
                    break;
                }
                const int g = nbv >> 3, kp = nbv & 3, gfl = (nbv >> 2) & 1;
                if (g == f0) break;
                fl ^= (unsigned)gfl;
                const FaceRec Rg = load_rec(P.rec, g);
                const bool x_end_cur = (cur_c == nxt(e));
                const bool x_start_g = (x_end_cur != (bool)gfl);
                const int cg = x_start_g ? kp : nxt(kp);
                const int yg = x_start_g ? nxt(kp) : kp;
                const int zg = 3 - cg - yg;
                consider(g, Rg, cg, fl);
                e = (nxt(cg) == zg) ? cg : zg;
                cur = g; cur_c = cg; Rc = Rg;
            }
        }
        if (bg >= 0) {
            if (serr - berr < tau) w.st |= SG_ST_NEAR_VERTEX;
            w.f = bg;
            w.R = load_rec(P.rec, bg);
            w.px = corner_x(w.R, bcg); w.py = corner_y(w.R, bcg);
            w.dx = bux; w.dy = buy;
            w.mode = 3 + bcg;
            if (bfl) w.st ^= SG_PARITY_BIT;
            walker_hash(w, bg, P.want_hash);
            return true;
        }
        if (nb == 0) { w.st |= SG_ST_BOUNDARY; return false; }
        nb = nb > 2 ? 2 : nb;
        int k = 0;
        if (nb == 2) {
            const int4 t0 = __ldg(P.fv + ebf0);
            const int o0 = sel3(ebo0, t0.x, t0.y, t0.z);
            if (came_from >= 0) {
                k = (o0 == came_from) ? 1 : 0;
            } else {
                const int4 t1 = __ldg(P.fv + ebf1);
                const int o1 = sel3(ebo1, t1.x, t1.y, t1.z);
                const float4 xv = __ldg(P.V + v0), x0 = __ldg(P.V + o0), x1 = __ldg(P.V + o1);
                const float a0x = x0.x - xv.x, a0y = x0.y - xv.y, a0z = x0.z - xv.z;
                const float a1x = x1.x - xv.x, a1y = x1.y - xv.y, a1z = x1.z - xv.z;
                const float d0 = (Dx * a0x + Dy * a0y + Dz * a0z) * rsqrtf(a0x * a0x + a0y * a0y + a0z * a0z);
                const float d1 = (Dx * a1x + Dy * a1y + Dz * a1z) * rsqrtf(a1x * a1x + a1y * a1y + a1z * a1z);
                k = d1 > d0 ? 1 : 0;
                if (fabsf(d1 - d0) < tau) w.st |= SG_ST_NEAR_VERTEX;
            }
        }
        const int fb = k ? ebf1 : ebf0, cb = k ? ebc1 : ebc0, co = k ? ebo1 : ebo0;
        if (k ? ebfl1 : ebfl0) w.st ^= SG_PARITY_BIT;
        if (fb != w.f) {
            w.f = fb;
            w.R = load_rec(P.rec, fb);
            walker_hash(w, fb, P.want_hash);
        }
        const float ax = corner_x(w.R, cb), ay = corner_y(w.R, cb);
        if (w.steps >= P.max_steps) {
            w.st |= SG_ST_MAX_STEPS;
            w.px = ax; w.py = ay; w.mode = 3 + cb;
            return false;
        }
        w.steps++;
        const float bx = corner_x(w.R, co), by = corner_y(w.R, co);
        const float ex = bx - ax, ey = by - ay, le = sqrtf(ex * ex + ey * ey);
        const float L = w.Lh + w.Ll;
        if (L <= le) {
            const float t = L / le;
            w.px = fmaf(t, ex, ax); w.py = fmaf(t, ey, ay);
            w.Lh = 0.f; w.Ll = 0.f;
            float e1x, e1y, e1z, e2x, e2y, e2z;
            frm_axes(P, fb, e1x, e1y, e1z, e2x, e2y, e2z);
            float ux = Dx * e1x + Dy * e1y + Dz * e1z, uy = Dx * e2x + Dy * e2y + Dz * e2z;
            const float lu = sqrtf(ux * ux + uy * uy);
            if (lu > 1e-6f) { w.dx = ux / lu; w.dy = uy / lu; } else { w.dx = ex / le; w.dy = ey / le; }
            w.mode = 6;
            return false;
        }
        {   // compensated L -= le
            float a = w.Lh, b = -le;
            float sum = a + b;
            float bb = sum - a;
            float err = (a - (sum - bb)) + (b - bb);
            w.Lh = sum;
            w.Ll += err;
        }
        came_from = v0;
        c = co;
        w.px = bx; w.py = by; w.mode = 3 + co;
    }
}

// The walk reached boundary edge j of face w.f at (w.px, w.py) (face frame, w.R the face
// record): slide along it toward the endpoint the direction points to (corner j+1 when
// d . (P_{j+1} - P_j) >= 0, else corner j).  Returns false when the length ran out on the edge;
// true when the walker reached that endpoint, which is then corner *c of w.f, with *came the
// vertex it slid from.
__device__ __forceinline__ bool hole_edge(Walker &w, const WalkParams &P, int j, int *c, int *came) {
    w.st |= SG_ST_HOLE;
    const FaceRec &R = w.R;
    const float ax = corner_x(R, j), ay = corner_y(R, j), bx = corner_x(R, nxt(j)), by = corner_y(R, nxt(j));
    const float ex = bx - ax, ey = by - ay;
    const float de = (w.dx * ex + w.dy * ey) * rsqrtf(ex * ex + ey * ey);
    if (fabsf(de) < P.tau_near) w.st |= SG_ST_NEAR_VERTEX;
    const int tgt = de >= 0.f ? nxt(j) : j, oth = de >= 0.f ? j : nxt(j);
    const float tx = corner_x(R, tgt) - w.px, ty = corner_y(R, tgt) - w.py;
    const float dist = sqrtf(tx * tx + ty * ty);
    const float L = w.Lh + w.Ll;
    if (L <= dist) {
        const float t = dist > 0.f ? L / dist : 0.f;
        w.px = fmaf(t, tx, w.px); w.py = fmaf(t, ty, w.py);
        w.Lh = 0.f; w.Ll = 0.f;
        w.mode = 6;
        return false;
    }
    {   // compensated L -= dist
        float a = w.Lh, b = -dist;
        float sum = a + b;
        float bb = sum - a;
        float err = (a - (sum - bb)) + (b - bb);
        w.Lh = sum;
        w.Ll += err;
    }
    w.steps++;
    const int4 t3 = __ldg(P.fv + w.f);
    w.px = corner_x(R, tgt); w.py = corner_y(R, tgt); w.mode = 3 + tgt;
    *c = tgt;
    *came = sel3(oth, t3.x, t3.y, t3.z);
    return true;
}

// Applies a pending boundary event of hole avoidance.  The step code only marks the event
// (modes 8..13), so that a walk kernel can apply the events of several lanes together: each
// is a chain of dependent gathers around a vertex fan, and lanes waiting one by one on such
// chains would serialise the warp.  Returns true when the walk ended.
__device__ __forceinline__ bool hole_resolve(Walker &w, const WalkParams &P) {
    // D: the direction, in 3-D, that the walker has on reaching the boundary
    float e1x, e1y, e1z, e2x, e2y, e2z;
    frm_axes(P, w.f, e1x, e1y, e1z, e2x, e2y, e2z);
    const float Dx = w.dx * e1x + w.dy * e2x, Dy = w.dx * e1y + w.dy * e2y, Dz = w.dx * e1z + w.dy * e2z;
    int c = w.mode - SG_MODE_HOLE_VERTEX, came = -1;
    if (w.mode < SG_MODE_HOLE_VERTEX && !hole_edge(w, P, w.mode - SG_MODE_HOLE_EDGE, &c, &came)) return true;
    return !hole_vertex(w, P, c, came, Dx, Dy, Dz);
}

// Vertex transport: the walker reached corner c of face w.f with direction d.
// Straightest rule (Sec. 4, Alg. transport_over_vertex): leave along the ray that splits the
// total angle theta(x) in two equal halves with the reversed incoming ray.  The fan is walked
// from -d through the faces around x until the accumulated corner angles pass theta/2; the
// outgoing ray lies in that face at the excess angle from the shared edge.
// Returns false if the walk must stop (boundary vertex).
template <bool HOLE = false>
__device__ __forceinline__ bool vertex_transport(Walker &w, int c, const WalkParams &P) {
    int4 fvv = __ldg(P.fv + w.f);
    int vid = sel3(c, fvv.x, fvv.y, fvv.z);
    float th = __ldg(&P.V[vid].w);
    w.st |= SG_ST_VERTEX_HIT;
    float cx = corner_x(w.R, c), cy = corner_y(w.R, c);
    w.px = cx; w.py = cy;
    if (th < 0.f) {  // boundary vertex: original rule stops here (Sec. 4), or hole avoidance
        if (HOLE) {  // handled by hole_resolve on a later call
            w.mode = SG_MODE_HOLE_VERTEX + c;
            return true;
        }
        w.st |= SG_ST_BOUNDARY;
        return false;
    }
    const float half = 0.5f * th;
    float rx = -w.dx, ry = -w.dy;
    // first edge: local edge prv(c) runs from corner prv(c) to corner c = x
    int e = prv(c);
    float ex = corner_x(w.R, prv(c)) - cx, ey = corner_y(w.R, prv(c)) - cy;
    float A = atan2f(fabsf(rx * ey - ry * ex), rx * ex + ry * ey);
    if (A >= half) {
        // rotate r toward the edge by theta/2 inside this face
        float hx = ex - (ex * rx + ey * ry) * rx, hy = ey - (ex * rx + ey * ry) * ry;
        renorm(hx, hy);
        float sh, ch;
        sincosf(half, &sh, &ch);
        w.dx = ch * rx + sh * hx;
        w.dy = ch * ry + sh * hy;
        renorm(w.dx, w.dy);
        w.mode = 3 + c;
        walker_hash(w, w.f, P.want_hash);
        return true;
    }
    int cur_c = c;
    FaceRec Rc = w.R;
    for (int guard = 0; guard < 4096; ++guard) {
        int nb = nbr_of(Rc, e);
        if (nb < 0) {  // open fan reached although theta says interior: stop (inconsistent input)
            w.st |= SG_ST_BOUNDARY;
            return false;
        }
        int g = nb >> 3, kp = nb & 3, fl = (nb >> 2) & 1;
        if (fl) w.st ^= SG_PARITY_BIT;
        FaceRec Rg = load_rec(P.rec, g);
        bool x_end_cur = (cur_c == nxt(e));
        bool x_start_g = (x_end_cur != (bool)fl);
        int cg = x_start_g ? kp : nxt(kp);
        int yg = x_start_g ? nxt(kp) : kp;
        int zg = 3 - cg - yg;
        float gx = corner_x(Rg, cg), gy = corner_y(Rg, cg);
        float ux = corner_x(Rg, yg) - gx, uy = corner_y(Rg, yg) - gy;
        float zx = corner_x(Rg, zg) - gx, zy = corner_y(Rg, zg) - gy;
        float gam = atan2f(fabsf(ux * zy - uy * zx), ux * zx + uy * zy);
        if (A + gam >= half) {
            float beta = half - A;
            renorm(ux, uy);
            float hx = zx - (zx * ux + zy * uy) * ux, hy = zy - (zx * ux + zy * uy) * uy;
            renorm(hx, hy);
            float sb, cb;
            sincosf(beta, &sb, &cb);
            w.dx = cb * ux + sb * hx;
            w.dy = cb * uy + sb * hy;
            renorm(w.dx, w.dy);
            w.f = g;
            w.R = Rg;
            w.px = gx; w.py = gy;
            w.mode = 3 + cg;
            walker_hash(w, g, P.want_hash);
            return true;
        }
        A += gam;
        e = (nxt(cg) == zg) ? cg : zg;  // the other edge of g at x
        cur_c = cg;
        Rc = Rg;
    }
    w.st |= SG_ST_MAX_STEPS;
    return false;
}

// An edge crossing as seen by observers: exit edge j (local edge of the old face) with
// endpoints (x0,y0) -> (x1,y1) and crossing point q in the old frame, the remaining length
// after the crossing, the new face g entered through its local edge kp starting at (gax,gay)
// with edge vector (fx,fy) in the new frame, the flip bit, the new direction, and the
// rotations that take each frame's vectors to its face frame.
struct Cross {
    int j;
    float x0, y0, x1, y1, qx, qy, Lr;
    int g, kp, fl;
    float gax, gay, fx, fy, ndx, ndy;
    float ca0, sa0, ca1, sa1;  // rotations old frame -> old face frame, new frame -> new face frame
    float il;                  // 1 / |x1 - x0| (the crossed edge's inverse length)
    int ke;                    // the old face's entry edge (half-edge step), -1 from a face-frame step
    float s;                   // q = A + s (B - A)
    float da, dc;              // d . (B - A) and d x (B - A) (old frame, old direction)
};

// Observer of a walk (the backward pass hooks into the same step code as the forward).
struct NoHook {
    // general step: sigma of the three corners after classification, entry mode, snapped corner
    __device__ __forceinline__ void on_face(const Walker &, float, float, float, int, int) {}
    // half-edge step: sigma of the apex, its position and the walker position (edge frame)
    __device__ __forceinline__ void on_apex(const Walker &, float, float, float, float, float) {}
    // at an edge crossing (walker still in the old face, length already reduced)
    __device__ __forceinline__ void on_cross(const Walker &, const Cross &, const FaceRec &) {}
    // before a vertex transport at corner `hit` of the current face
    __device__ __forceinline__ void on_vertex(const Walker &, int) {}
};

// Leave the half-edge frame: position (xe, ye) and direction into the face frame of w.f,
// R becomes the face record (needed at the end of a walk and before a vertex transport).
template <bool MIX = false>
__device__ __forceinline__ void half_to_face(Walker &w, const WalkParams &P, float xe, float ye) {
    float ca = MIX ? 1.f : hca(w.R), sa = MIX ? 0.f : hsa(w.R);
    w.f = w.h / 3;  // not kept up to date on the hot path
    const int k = w.h - 3 * w.f;
    const FaceRec F = load_rec(P.rec, w.f);
    if (MIX) {  // the double-float record holds no rotation: edge k's direction in the face frame
        if (k == 1) { ca = (F.x2x - F.l01) * F.il1; sa = F.x2y * F.il1; }
        else if (k == 2) { ca = -F.x2x * F.il2; sa = -F.x2y * F.il2; }
        w.dxl = 0.f; w.dyl = 0.f;
    }
    w.px = corner_x(F, k) + ca * xe - sa * ye;
    w.py = corner_y(F, k) + sa * xe + ca * ye;
    const float dx = ca * w.dx - sa * w.dy, dy = sa * w.dx + ca * w.dy;
    w.dx = dx; w.dy = dy;
    w.R = F;
    w.mode = 6;
}

// The hot step: the walker sits on the entry edge A=(0,0) -> B=(l,0) of half-edge h at
// x = s*l, the apex is C=(cx,cy) with cy > 0.  sigma_A = dy x, sigma_B = -dy (l - x),
// sigma_C = dx cy - dy (cx - x).  The exit edge is B -> C when the apex lies left of the ray
// (sigma_C > 0), else C -> A.  The twin half-edge's frame has the crossed edge as its x axis
// (reversed unless the adjacency is flipped) and the new face on +y, so the new direction is
// (-+ d.e, d.n_out) / |e|, renormalised; no corner lookups are needed.
// MIX: the mixed walk -- the same step on the double-float half-edge record (l, cx, cy as hi + lo
// pairs and the two links, one 32-byte sector), the orientation tests, exit point and length in
// FP32 from the high parts, and the direction carried in double-float: its rotation into the next
// edge frame uses the double-float exit edge vector and double-float dot products, so the
// direction's error does not grow with the path (the FP32 walk's does).
template <bool ESC, bool HOLE, bool MIX, class Hook>
__device__ __forceinline__ bool half_step(Walker &w, const WalkParams &P, Hook &hook) {
    const FaceRec &R = w.R;
    const float near = P.tau_near * w.lref, snap = P.tau_snap * w.lref;
    const float L0 = MIX ? __int_as_float(R.n0) : hl(R);
    const float cx = MIX ? __int_as_float(R.n2) : hcx(R);
    const float cy = MIX ? R.x2x : hcy(R);
    const float x = w.px * L0;
    float sA = w.dy * x;
    float sB = -w.dy * (L0 - x);
    float sC = fmaf(w.dx, cy, -w.dy * (cx - x));
    bool hit = false;
    if (fabsf(sC) < near) {  // rare: the apex lies in the near band (the entry points require snap <= near)
        if (ESC) {
            // FP64 re-evaluation of the classification (exact products of the walker's state)
            w.st |= SG_ST_FP64;
            const double Ld = MIX ? (double)L0 + (double)__int_as_float(R.n1) : (double)L0;
            const double cxd = MIX ? (double)cx + (double)R.l01 : (double)cx;
            const double cyd = MIX ? (double)cy + (double)R.x2y : (double)cy;
            const double dxd = MIX ? (double)w.dx + (double)w.dxl : (double)w.dx;
            const double dyd = MIX ? (double)w.dy + (double)w.dyl : (double)w.dy;
            const double X = (double)w.px * Ld;
            sA = f32_keep_sign(dyd * X);
            sB = f32_keep_sign(-dyd * (Ld - X));
            sC = f32_keep_sign(dxd * cyd - dyd * (cxd - X));
        }
        hit = fabsf(sC) <= snap;  // a snapped apex is a hit, not a near miss
        if (!hit && fabsf(sC) < near) w.st |= SG_ST_NEAR_VERTEX;
    }
    hook.on_apex(w, sC, cx, cy, x, 0.f);
    const bool right = sC > 0.f;
    const float x0 = right ? L0 : cx, y0 = right ? 0.f : cy;
    const float x1 = right ? cx : 0.f, y1 = right ? cy : 0.f;
    float qx, qy, s;
    if (hit) {
        qx = cx; qy = cy;
        s = right ? 1.f : 0.f;
    } else {
        const float s0 = right ? sB : sC, s1 = right ? sC : sA;
        const float den = s0 - s1;
        s = __saturatef(den != 0.f ? __fdividef(s0, den) : 0.5f);  // clamped to [0, 1], NaN to 0
        qx = fmaf(s, x1 - x0, x0);
        qy = fmaf(s, y1 - y0, y0);
    }
    const float t = fmaxf(fmaf(qx - x, w.dx, qy * w.dy), 0.f);
    const float L = w.Lh + w.Ll;
    if (t >= L) {
        // final truncated in-face segment (reading: stop once the length is used up)
        const float xe = fmaf(L, w.dx, x), ye = L * w.dy;
        w.Lh = 0.f; w.Ll = 0.f;
        half_to_face<MIX>(w, P, xe, ye);
        const FaceRec &F = w.R;
        float d0 = fabsf(w.py);
        float d1 = fabsf((F.x2x - F.l01) * (w.py) - F.x2y * (w.px - F.l01)) * F.il1;
        float d2 = fabsf(F.x2x * w.py - F.x2y * w.px) * F.il2;
        if (fminf(fminf(d0, d1), d2) <= near) w.st |= SG_ST_NEAR_EDGE;
        return true;
    }
    {   // compensated L -= t: t < Lh + Ll here, so |Lh| >= |t| up to the tiny Ll and Dekker's
        // fast two-sum gives the exact rounding error of Lh - t
        const float sum = w.Lh - t;
        w.Ll += -t - (sum - w.Lh);
        w.Lh = sum;
    }
    if (hit) {
        half_to_face<MIX>(w, P, cx, cy);
        const int c = prv(w.h - 3 * w.f);  // the apex is corner k+2 of the face
        hook.on_vertex(w, c);
        return !vertex_transport<HOLE>(w, c, P);
    }
    const int link = MIX ? (right ? __float_as_int(R.il1) : __float_as_int(R.il2)) : (right ? hlinkR(R) : hlinkL(R));
    if (link < 0) {  // boundary edge: original rule stops (Sec. 4), or hole avoidance
        half_to_face<MIX>(w, P, qx, qy);
        const int k = w.h - 3 * w.f;
        if (HOLE) {  // handled by hole_resolve on a later call
            w.mode = SG_MODE_HOLE_EDGE + (right ? nxt(k) : prv(k));
            return false;
        }
        w.st |= SG_ST_BOUNDARY;
        return true;
    }
    const int hn = link >> 1, fl = link & 1;
    float ndx, ndy, re, eda = 0.f, edc = 0.f;
    if (MIX) {
        // the exit edge in double-float: B -> C = (cx - l, cy), C -> A = -(cx, cy)
        const DF Ld{L0, __int_as_float(R.n1)}, cxd{cx, R.l01}, cyd{cy, R.x2y};
        const DF dxd{w.dx, w.dxl}, dyd{w.dy, w.dyl};
        const DF ex = right ? df_sub(cxd, Ld) : df_neg(cxd), ey = right ? cyd : df_neg(cyd);
        const DF da = df_dot2(dxd, ex, dyd, ey);            // |e| (d . e_hat)
        const DF dc = df_dot2(dxd, ey, df_neg(dyd), ex);    // |e| (d . n_out)
        // one FP32 scale for both components keeps the angle to double-float precision
        re = rsqrtf(fmaf(da.hi, da.hi, dc.hi * dc.hi));
        const DF nx = df_mul_f(fl ? da : df_neg(da), re), ny = df_mul_f(dc, re);
        ndx = nx.hi; ndy = ny.hi;
        w.dxl = nx.lo; w.dyl = ny.lo;
    } else {
        const float ex = x1 - x0, ey = y1 - y0;
        const float da = fmaf(w.dx, ex, w.dy * ey);   // |e| (d . e_hat)
        const float dc = fmaf(w.dx, ey, -w.dy * ex);  // |e| (d . n_out)
        // |(da, dc)| = |e|: one reciprocal square root normalises it (rsqrtf's error, a few 1e-7,
        // does not accumulate: every step renormalises the direction it receives)
        re = rsqrtf(fmaf(da, da, dc * dc));
        ndx = (fl ? da : -da) * re; ndy = dc * re;
        eda = da; edc = dc;
    }
    const FaceRec G = load_rec<true>(MIX ? P.half48 : P.half, hn);
    if (!MIX) {
        const int k = w.h - 3 * (w.h / 3);
        const int g = hn / 3;
        hook.on_cross(w, Cross{right ? nxt(k) : prv(k), x0, y0, x1, y1, qx, qy, w.Lh + w.Ll, g, hn - 3 * g, fl,
                               0.f, 0.f, hl(G), 0.f, ndx, ndy, hca(R), hsa(R), hca(G), hsa(G), re, k, s, eda, edc},
                      G);
    }
    w.px = fl ? s : 1.f - s;
    w.py = 0.f;
    w.dx = ndx; w.dy = ndy;
    w.h = hn;
    w.R = G;
    if (fl) w.st ^= SG_PARITY_BIT;
    w.ncross++;
    if (P.want_hash) walker_hash(w, hn / 3, 1);
    return false;
}

template <bool ESC, bool HOLE, bool MIX, class Hook>
__device__ __forceinline__ bool general_step(Walker &w, const WalkParams &P, Hook &hook);

// One step of Alg. geodesic_step.  Returns true when the walk is finished.
template <bool ESC, bool HOLE = false, bool MIX = false, class Hook = NoHook>
__device__ __forceinline__ bool walker_step(Walker &w, const WalkParams &P, Hook &&hook = Hook()) {
    if (HOLE && w.mode >= SG_MODE_HOLE_EDGE) return hole_resolve(w, P);  // a pending boundary event
    if (w.steps >= P.max_steps) {
        if (w.mode == SG_MODE_HALF)
            half_to_face<MIX>(w, P, w.px * (MIX ? __int_as_float(w.R.n0) : hl(w.R)), 0.f);
        w.st |= SG_ST_MAX_STEPS;
        return true;
    }
    w.steps++;
    if (w.mode == SG_MODE_HALF) return half_step<ESC, HOLE, MIX>(w, P, hook);
    return general_step<ESC, HOLE, MIX>(w, P, hook);
}

// Step from a corner (after a vertex transport) or from a free start point (face frame); a
// crossing moves the walker into the half-edge frame of the face it enters.
template <bool ESC, bool HOLE, bool MIX, class Hook>
__device__ __forceinline__ bool general_step(Walker &w, const WalkParams &P, Hook &hook) {
    const FaceRec &R = w.R;
    const float near = P.tau_near * w.lref, snap = P.tau_snap * w.lref;
    float s0 = sigma32(w.dx, w.dy, 0.f, 0.f, w.px, w.py);
    float s1 = sigma32(w.dx, w.dy, R.l01, 0.f, w.px, w.py);
    float s2 = sigma32(w.dx, w.dy, R.x2x, R.x2y, w.px, w.py);
    int j;          // exit edge (corner j -> corner j+1)
    int hit = -1;   // corner hit, or -1
    const int mode = w.mode;
    // corners relevant to the decision: apex (entered through an edge), the two far corners
    // (sitting on a corner), or all three (free start)
    float mrel = mode < 3 ? fabsf(sel3(prv(mode), s0, s1, s2))
               : mode < 6 ? fminf(fabsf(sel3(nxt(mode - 3), s0, s1, s2)), fabsf(sel3(prv(mode - 3), s0, s1, s2)))
                          : fminf(fminf(fabsf(s0), fabsf(s1)), fabsf(s2));
    if (ESC && mrel < near) {
        // FP64 re-evaluation of the classification (exact products of the FP32 state)
        w.st |= SG_ST_FP64;
        s0 = f32_keep_sign(sigma64(w.dx, w.dy, 0.f, 0.f, w.px, w.py));
        s1 = f32_keep_sign(sigma64(w.dx, w.dy, R.l01, 0.f, w.px, w.py));
        s2 = f32_keep_sign(sigma64(w.dx, w.dy, R.x2x, R.x2y, w.px, w.py));
    }
    float mflag;    // near-vertex margin, excluding a snapped corner
    if (mode < 3) {
        const int k = mode, a = prv(k);  // apex = corner k+2
        float sa = sel3(a, s0, s1, s2);
        mflag = fabsf(sa);
        if (mflag <= snap) { hit = a; mflag = 3.0e38f; }
        j = sa > 0.f ? nxt(k) : prv(k);
    } else if (mode < 6) {
        const int c = mode - 3, a = nxt(c), b = prv(c);
        j = a;
        float fa = fabsf(sel3(a, s0, s1, s2)), fb = fabsf(sel3(b, s0, s1, s2));
        mflag = fminf(fa, fb);
        if (mflag <= snap) { hit = fa <= fb ? a : b; mflag = fmaxf(fa, fb); }
    } else {
        // forward exit edge: sigma(start corner) < 0 <= sigma(end corner), CCW frame
        if (s0 < 0.f && s1 >= 0.f) j = 0;
        else if (s1 < 0.f && s2 >= 0.f) j = 1;
        else if (s2 < 0.f && s0 >= 0.f) j = 2;
        else { w.st |= SG_ST_INVALID; return true; }
        float fa = fabsf(sel3(j, s0, s1, s2)), fb = fabsf(sel3(nxt(j), s0, s1, s2)), fo = fabsf(sel3(prv(j), s0, s1, s2));
        mflag = fminf(fminf(fa, fb), fo);
        if (fminf(fa, fb) <= snap) { hit = fa <= fb ? j : nxt(j); mflag = fminf(fmaxf(fa, fb), fo); }
    }
    if (mflag < near) w.st |= SG_ST_NEAR_VERTEX;
    hook.on_face(w, s0, s1, s2, mode, hit);
    // exit point on edge j: A = P_j, B = P_{j+1}; s = sigma_A / (sigma_A - sigma_B)
    const int jb = nxt(j);
    float ax = corner_x(R, j), ay = corner_y(R, j);
    float bx = corner_x(R, jb), by = corner_y(R, jb);
    float qx, qy, s;
    if (hit >= 0) {
        qx = corner_x(R, hit); qy = corner_y(R, hit);
        s = (hit == j) ? 0.f : 1.f;
    } else {
        float sa = sel3(j, s0, s1, s2), sb = sel3(jb, s0, s1, s2);
        float den = sa - sb;
        s = den != 0.f ? sa / den : 0.5f;
        s = fminf(fmaxf(s, 0.f), 1.f);
        qx = fmaf(s, bx - ax, ax);
        qy = fmaf(s, by - ay, ay);
    }
    float t = fmaxf(fmaf(qx - w.px, w.dx, (qy - w.py) * w.dy), 0.f);
    float L = w.Lh + w.Ll;
    if (t >= L) {
        // final truncated in-face segment (reading: stop once the length is used up)
        w.px = fmaf(L, w.dx, w.px);
        w.py = fmaf(L, w.dy, w.py);
        w.Lh = 0.f; w.Ll = 0.f;
        // NEAR_EDGE: end point within tau_near*l_ref of an edge line of its face
        float d0 = fabsf(w.py);                                                   // edge 0 (y = 0)
        float d1 = fabsf((R.x2x - R.l01) * (w.py) - R.x2y * (w.px - R.l01)) * R.il1;  // edge 1
        float d2 = fabsf(R.x2x * w.py - R.x2y * w.px) * R.il2;                     // edge 2
        if (fminf(fminf(d0, d1), d2) <= near) w.st |= SG_ST_NEAR_EDGE;
        return true;
    }
    {   // compensated L -= t
        float a = w.Lh, b = -t;
        float sum = a + b;
        float bb = sum - a;
        float err = (a - (sum - bb)) + (b - bb);
        w.Lh = sum;
        w.Ll += err;
    }
    if (hit >= 0) {
        hook.on_vertex(w, hit);
        if (!vertex_transport<HOLE>(w, hit, P)) return true;
        return false;
    }
    const int nb = nbr_of(R, j);
    if (nb < 0) {  // boundary edge: original rule stops (Sec. 4), or hole avoidance
        w.px = qx; w.py = qy;
        if (HOLE) {  // handled by hole_resolve on a later call
            w.mode = SG_MODE_HOLE_EDGE + j;
            return false;
        }
        w.st |= SG_ST_BOUNDARY;
        return true;
    }
    const int g = nb >> 3, kp = nb & 3, fl = (nb >> 2) & 1;
    // into the half-edge frame of (g, kp): x along the crossed edge, the new face on +y
    const float ex = bx - ax, ey = by - ay;
    const float da = fmaf(w.dx, ex, w.dy * ey);
    const float dc = fmaf(w.dx, ey, -w.dy * ex);  // d . (ey, -ex)
    const int hn = 3 * g + kp;
    const FaceRec G = load_rec<true>(MIX ? P.half48 : P.half, hn);
    float ndx = fl ? da : -da, ndy = dc;
    renorm(ndx, ndy);
    if (MIX) {  // a face-frame step (a start on an edge or vertex, a vertex transport) is FP32
        w.dxl = 0.f; w.dyl = 0.f;
    } else {
        hook.on_cross(w, Cross{j, ax, ay, bx, by, qx, qy, w.Lh + w.Ll, g, kp, fl, 0.f, 0.f, hl(G), 0.f, ndx, ndy,
                               1.f, 0.f, hca(G), hsa(G), rsqrtf(fmaf(bx - ax, bx - ax, (by - ay) * (by - ay))), -1, s, da, dc},
                      G);
    }
    w.px = fl ? s : 1.f - s;
    w.py = 0.f;
    w.dx = ndx; w.dy = ndy;
    w.f = g;
    w.h = hn;
    w.R = G;
    w.mode = SG_MODE_HALF;
    if (fl) w.st ^= SG_PARITY_BIT;
    w.ncross++;
    walker_hash(w, g, P.want_hash);
    return false;
}

// query inputs (device pointers; mesh_id/length/w may be NULL)
struct QueryIn {
    int32_t n_mesh;
    const int32_t *__restrict__ mesh_id;
    const int32_t *__restrict__ face;
    const float *__restrict__ bary;
    const float *__restrict__ v;
    const float *__restrict__ length;
    const float *__restrict__ w;
};

// Inputs and outputs of one forward call, handed to the FP64 and double-float walks (exp_map64.cu).
struct SgFwdIO {
    QueryIn in;
    int64_t nq;
    int32_t *out_face;
    float *out_bary, *out_pos, *out_dir, *out_w;
    uint32_t *out_status;
    int32_t *out_ncross;
    uint64_t *out_hash;
    const int32_t *perm;
    int32_t *counter;
};
sg_status sg_geom64_prepare(sg_mesh *m, cudaStream_t s, bool half48);
// Length order of a batch (exp_map.cu): perm[0 .. nq) = the queries longest walk first, in
// buckets of an eighth of an octave of L / l_ref.  Scratch: keys (nq bytes), counts (512 int32).
#define SG_LBUCKETS 256
// With esc_lmax > 0, bucket 0 (the order's head, counts[0] queries) holds the queries longer than
// esc_lmax l_ref.
void sg_length_order(const sg_mesh *m, const QueryIn &in, int64_t nq, uint8_t *keys, int32_t *counts, int32_t *perm,
                     cudaStream_t s, float esc_lmax = 0.f);
cudaError_t sg_launch_walk64(const sg_mesh *m, const SgFwdIO &io, int n_w, const sg_opts &r, cudaStream_t s);

struct Frame3 {
    float ox, oy, oz;  // corner 0
    float e1x, e1y, e1z, e2x, e2y, e2z;
    float x1x, x1y, x1z, x2x, x2y, x2z;  // corners 1, 2
};

// 3-D frame of a face from the vertex positions: e1 along x1-x0, e2 = n x e1.  This is the
// frame in which the intrinsic record was expressed by the mesh builder.
__device__ __forceinline__ Frame3 face_frame(const WalkParams &P, int gf) {
    int4 t = __ldg(P.fv + gf);
    float4 a = __ldg(P.V + t.x), b = __ldg(P.V + t.y), c = __ldg(P.V + t.z);
    Frame3 F;
    F.ox = a.x; F.oy = a.y; F.oz = a.z;
    F.x1x = b.x; F.x1y = b.y; F.x1z = b.z;
    F.x2x = c.x; F.x2y = c.y; F.x2z = c.z;
    float ux = b.x - a.x, uy = b.y - a.y, uz = b.z - a.z;
    float vx = c.x - a.x, vy = c.y - a.y, vz = c.z - a.z;
    float nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    float rn = rsqrtf(nx * nx + ny * ny + nz * nz);
    nx *= rn; ny *= rn; nz *= rn;
    float ru = rsqrtf(ux * ux + uy * uy + uz * uz);
    ux *= ru; uy *= ru; uz *= ru;
    F.e1x = ux; F.e1y = uy; F.e1z = uz;
    F.e2x = ny * uz - nz * uy; F.e2y = nz * ux - nx * uz; F.e2z = nx * uy - ny * ux;
    return F;
}

template <int NW>
struct Carry {
    float c[NW > 0 ? NW : 1], s[NW > 0 ? NW : 1];
};

// initialise_trace (Alg. gpu_parallel): start face, barycentric point, tangent projection,
// length.  Returns false if the query finishes immediately (invalid, zero length).
template <int NW>
__device__ bool walker_init(const WalkParams &P, const QueryIn &a, int64_t q, Walker &w, Carry<NW> &cw) {
    int m = a.mesh_id ? __ldg(a.mesh_id + q) : 0;
    int lf = __ldg(a.face + q);
    w.st = 0; w.steps = 0; w.ncross = 0; w.hash = SG_FNV_OFFSET;
    w.mode = 6; w.Ll = 0.f; w.h = -1;
    bool bad = (m < 0 || m >= a.n_mesh);
    int foff = bad ? 0 : __ldg(P.face_off + m);
    int nfm = bad ? 1 : __ldg(P.face_off + m + 1) - foff;
    bad = bad || lf < 0 || lf >= nfm;
    float lr = bad ? 1.f : __ldg(P.lref + m);
    bad = bad || !(lr > 0.f);  // a mesh moved to a degenerate face carries l_ref = -1
    w.foff = foff;
    w.f = bad ? foff : foff + lf;
    w.lref = bad ? 1.f : lr;
    w.R = load_rec(P.rec, w.f);
    float b0 = __ldg(a.bary + 3 * q), b1 = __ldg(a.bary + 3 * q + 1), b2 = __ldg(a.bary + 3 * q + 2);
    float sb = b0 + b1 + b2;
    if (!(fabsf(sb - 1.f) <= 1e-6f) || b0 < -1e-7f || b1 < -1e-7f || b2 < -1e-7f) bad = true;
    if (bad) {
        w.st |= SG_ST_INVALID;
        w.px = w.py = 0.f; w.dx = w.dy = 0.f;
        w.Lh = 0.f;
        for (int k = 0; k < NW; ++k) { cw.c[k] = 0.f; cw.s[k] = 0.f; }
        return false;
    }
    float rs = 1.f / sb;
    b0 = fmaxf(b0, 0.f) * rs; b1 = fmaxf(b1, 0.f) * rs; b2 = fmaxf(b2, 0.f) * rs;
    w.px = fmaf(b1, w.R.l01, b2 * w.R.x2x);
    w.py = b2 * w.R.x2y;
    Frame3 F = face_frame(P, w.f);
    float vx = __ldg(a.v + 3 * q), vy = __ldg(a.v + 3 * q + 1), vz = __ldg(a.v + 3 * q + 2);
    float v1 = vx * F.e1x + vy * F.e1y + vz * F.e1z;
    float v2 = vx * F.e2x + vy * F.e2y + vz * F.e2z;
    float Lv = sqrtf(v1 * v1 + v2 * v2);
    float L = a.length ? __ldg(a.length + q) : Lv;
    // a non-finite vector or length is invalid input (comparisons with NaN are false)
    if (!(L >= 0.f && L <= 3.0e38f) || !(Lv <= 3.0e38f) || (Lv == 0.f && L > 0.f)) {
        w.st |= SG_ST_INVALID;
        w.dx = w.dy = 0.f; w.Lh = 0.f;
        for (int k = 0; k < NW; ++k) { cw.c[k] = 0.f; cw.s[k] = 0.f; }
        return false;
    }
    if (Lv > 0.f) { w.dx = v1 / Lv; w.dy = v2 / Lv; } else { w.dx = w.dy = 0.f; }
    w.Lh = L;
    // carried vectors as components along d and perp(d) = (-dy, dx); a zero vector v walks
    // nothing and carries them unchanged, measured against e1 instead (reading: transport
    // along an empty path is the identity)
    const float rx = Lv > 0.f ? w.dx : 1.f, ry = Lv > 0.f ? w.dy : 0.f;
    for (int k = 0; k < NW; ++k) {
        const float *wp = a.w + (3 * NW) * q + 3 * k;
        float wx = __ldg(wp), wy = __ldg(wp + 1), wz = __ldg(wp + 2);
        float w1 = wx * F.e1x + wy * F.e1y + wz * F.e1z;
        float w2 = wx * F.e2x + wy * F.e2y + wz * F.e2z;
        cw.c[k] = w1 * rx + w2 * ry;
        cw.s[k] = rx * w2 - ry * w1;
    }
    int zeros = (b0 == 0.f) + (b1 == 0.f) + (b2 == 0.f);
    if (zeros) w.st |= SG_ST_START_ON_EDGE;
    if (zeros == 2 && L > 0.f) {
        // start on a vertex: the direction must point into this face's corner (reading)
        int c = b0 == 1.f ? 0 : (b1 == 1.f ? 1 : 2);
        float cx = corner_x(w.R, c), cy = corner_y(w.R, c);
        float ax = corner_x(w.R, nxt(c)) - cx, ay = corner_y(w.R, nxt(c)) - cy;
        float bx = corner_x(w.R, prv(c)) - cx, by = corner_y(w.R, prv(c)) - cy;
        if (!(ax * w.dy - ay * w.dx > 0.f && w.dx * by - w.dy * bx > 0.f)) {
            w.st |= SG_ST_INVALID;
            w.Lh = 0.f;
            return false;
        }
        w.px = cx; w.py = cy;
        w.mode = 3 + c;
    }
    // the face sequence starts with the start face of every query that walks (L > 0)
    if (L > 0.f) walker_hash(w, w.f, P.want_hash);
    return L > 0.f;
}


// The mixed walk's start, after walker_init placed a free start point: the start direction and
// length in double-float from the FP64 face axes (an FP32 start direction would carry its rounding,
// about 6e-8 rad, over the whole walk), and the walker placed on the edge through which its ray
// enters the start face (behind the start point, the length extended by that distance), so that
// the walk begins in the half-edge mode.  Declined (the FP32 start stays, with no low parts) for a
// start on an edge or vertex, a zero or huge vector, or an entry-edge corner within the near band
// of the ray line.
__device__ __forceinline__ void walker_start_mix(const WalkParams &P, const QueryIn &in, int64_t q, Walker &w) {
    w.dxl = 0.f; w.dyl = 0.f;
    if (w.mode != 6) return;
    const float b0 = __ldg(in.bary + 3 * q), b1 = __ldg(in.bary + 3 * q + 1), b2 = __ldg(in.bary + 3 * q + 2);
    if (!(b0 > 0.f && b1 > 0.f && b2 > 0.f)) return;
    int4 ra, rb;
    ld_rec32<true>(P.half48 + 2 * (3 * w.f), ra, rb);  // half-edge 0 of the face: its frame is the face's
    const DF l01{__int_as_float(ra.x), __int_as_float(ra.y)}, x2x{__int_as_float(ra.z), __int_as_float(ra.w)};
    const DF x2y{__int_as_float(rb.x), __int_as_float(rb.y)};
    const DF sb = df_add(two_sum(b0, b1), DF{b2, 0.f});
    const DF rs = df_div(DF{1.f, 0.f}, sb);
    const DF B1 = df_mul_f(rs, b1), B2 = df_mul_f(rs, b2);
    const DF px = df_add_same_sign(df_mul(B1, l01), df_mul(B2, x2x)), py = df_mul(B2, x2y);
    const double *fr = P.frm64 + 6 * w.f;
    const double vx = __ldg(in.v + 3 * q), vy = __ldg(in.v + 3 * q + 1), vz = __ldg(in.v + 3 * q + 2);
    const DF V1 = df_from(vx * __ldg(fr) + vy * __ldg(fr + 1) + vz * __ldg(fr + 2));
    const DF V2 = df_from(vx * __ldg(fr + 3) + vy * __ldg(fr + 4) + vz * __ldg(fr + 5));
    const DF n2 = df_add_same_sign(df_mul(V1, V1), df_mul(V2, V2));
    if (!(n2.hi > 1e-30f && n2.hi < 1e30f)) return;
    const DF rn = df_rsqrt(n2);
    const DF dx = df_mul(V1, rn), dy = df_mul(V2, rn);
    DF L = df_mul(n2, rn);
    if (in.length) {
        const float Li = __ldg(in.length + q);
        if (!(Li > 0.f && Li < 1e30f)) return;
        L = DF{Li, 0.f};
    }
    // corners' signed distances to the ray line; the ray enters through edge j (corner j on its
    // left, corner j+1 on its right)
    const DF zero{0.f, 0.f};
    const DF s0 = df_sub(df_mul(dy, px), df_mul(dx, py));
    const DF s1 = df_sub(df_mul(dx, df_neg(py)), df_mul(dy, df_sub(l01, px)));
    const DF s2 = df_sub(df_mul(dx, df_sub(x2y, py)), df_mul(dy, df_sub(x2x, px)));
    int j;
    if (s0.hi > 0.f && s1.hi <= 0.f) j = 0;
    else if (s1.hi > 0.f && s2.hi <= 0.f) j = 1;
    else if (s2.hi > 0.f && s0.hi <= 0.f) j = 2;
    else return;
    const float nearf = P.tau_near * w.lref;
    const DF sa = j == 0 ? s0 : (j == 1 ? s1 : s2), sbb = j == 0 ? s1 : (j == 1 ? s2 : s0);
    if (fabsf(sa.hi) < nearf || fabsf(sbb.hi) < nearf) return;
    const DF ax = j == 0 ? zero : (j == 1 ? l01 : x2x), ay = j == 2 ? x2y : zero;
    const DF bx = j == 0 ? l01 : (j == 1 ? x2x : zero), by = j == 1 ? x2y : zero;
    const DF ex = df_sub(bx, ax), ey = df_sub(by, ay);
    const DF se = df_div(sa, df_add_same_sign(sa, df_neg(sbb)));
    const DF qx = df_add(ax, df_mul(se, ex)), qy = df_add(ay, df_mul(se, ey));
    DF tb = df_add(df_mul(df_sub(px, qx), dx), df_mul(df_sub(py, qy), dy));
    if (tb.hi < 0.f) tb = zero;
    const DF il = df_rsqrt(df_add_same_sign(df_mul(ex, ex), df_mul(ey, ey)));
    const DF hx = df_mul(df_add(df_mul(dx, ex), df_mul(dy, ey)), il);
    const DF hy = df_mul(df_sub(df_mul(ex, dy), df_mul(ey, dx)), il);
    if (!(hy.hi > 0.f)) return;
    const DF Lx = df_add_same_sign(L, tb);
    w.h = 3 * w.f + j;
    w.R = load_rec<true>(P.half48, w.h);
    w.px = se.hi; w.py = 0.f;
    w.dx = hx.hi; w.dxl = hx.lo;
    w.dy = hy.hi; w.dyl = hy.lo;
    w.Lh = Lx.hi; w.Ll = Lx.lo;
    w.mode = SG_MODE_HALF;
}

// ------------------------------------------------------------------ persistent driver
// warp-aggregated ticket: the calling lanes get consecutive queue positions
__device__ __forceinline__ int64_t fetch_ticket(int32_t *counter) {
    unsigned mask = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int rank = __popc(mask & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    return (int64_t)base + rank;
}

// Lanes pull task indices t < n from *counter.  A lane whose task has ended keeps its state
// in registers until REFILL lanes of the warp are idle (each kernel sets its own threshold); then all idle lanes finish
// (write results), take new tickets and initialise together, so the long init/finish code
// runs with many lanes active instead of stalling the warp for one lane every few steps.
// Once the counter passes n, lanes finish as soon as they are done and the warp leaves when
// all of its lanes are idle.  Every lane of the warp stays in the loop until then (the
// ballots use the full mask).  Job: bool init(t) (true: a walk to step), bool step()
// (true: done), void finish().  STEPS walk steps run between refill checks (each kernel sets
// its own count).
#define SG_REFILL_LANES 8
#ifndef SG_STEPS_PER_CHECK
#define SG_STEPS_PER_CHECK 2
#endif

template <class Job, int REFILL = SG_REFILL_LANES, int STEPS = SG_STEPS_PER_CHECK>
__device__ __forceinline__ void run_persistent(int32_t *counter, int64_t n, Job &job) {
    if (n <= 0) return;  // an empty list (a count read from device memory): no ticket to take
    bool live = false, pending = false, exhausted = false;
    const unsigned FULL = 0xffffffffu;
    while (true) {
        unsigned idle = __ballot_sync(FULL, !live);
        if (exhausted && idle == FULL) break;
        if (!exhausted && __popc(idle) >= REFILL) {
            bool dry = false;
            if (!live) {
                if (pending) {
                    job.finish();
                    pending = false;
                }
                int64_t t = fetch_ticket(counter);
                if (t >= n) {
                    dry = true;
                } else {
                    live = job.init(t);
                    if (!live) job.finish();
                }
            }
            exhausted = __any_sync(FULL, dry);
        }
        // several steps per refill check divide the loop overhead
#pragma unroll
        for (int k = 0; k < STEPS; ++k) {
            if (live && job.step()) {
                live = false;
                pending = true;
            }
        }
        if (exhausted && pending) {
            job.finish();
            pending = false;
        }
    }
}
