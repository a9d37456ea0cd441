// walk64.cuh -- the FP64, double-float and mixed-precision walkers (device code shared by the
// forward walks of exp_map64.cu and the mixed-precision literal GFD walks of backward.cu).
//
// FP64 walk: the walk of walk.cuh in face frames with every quantity of the walker state and of
// the face geometry in FP64 (Alg. geodesic_step, transport_over_edge, transport_over_vertex).
// Double-float walk: the FP32 walk's half-edge step with every quantity an unevaluated pair of
// FP32 numbers.  Mixed walk: the FP32 walk's orientation tests, exit points and length with the
// direction and the records' edge vectors in double-float.  The rare events of the last two (vertex
// hits, boundary stops, starts on an edge or vertex, MAX_STEPS) run the FP64 face-frame code.
#pragma once
#include <cuda_runtime.h>

#include "sgeo_internal.h"
#include "walk.cuh"

namespace {

struct R64 {
    int n0, n1, n2;
    double l01, x2x, x2y, il1, il2;
};

struct P64 {
    const int4 *__restrict__ rec;     // FP32 records: neighbour links
    const int4 *__restrict__ half48;  // [3 nF][2] double-float half-edge records (precision 48)
    const int4 *__restrict__ half;    // FP32 half-edge records (edge rotation for the outputs)
    const float4 *__restrict__ frm;   // FP32 face frames (3-D axes for the outputs)
    const double *__restrict__ rec64; // [nF][6] l01, x2x, x2y, 1/l12, 1/l20, -
    const double *__restrict__ frm64; // [nF][6] e1, e2
    const double *__restrict__ th64;  // [nV] theta, negated on the boundary
    const int4 *__restrict__ fv;
    const float4 *__restrict__ V;
    const int32_t *__restrict__ face_off;
    const float *__restrict__ lref;
    int max_steps, want_hash;
    double tau_near, tau_snap;
};

__device__ __forceinline__ R64 load64(const P64 &P, int f) {
    const int4 a = __ldg(P.rec + 2 * f);
    const double2 *r = reinterpret_cast<const double2 *>(P.rec64 + 6 * f);
    const double2 u = __ldg(r), v = __ldg(r + 1), w = __ldg(r + 2);
    return R64{a.x, a.y, a.z, u.x, u.y, v.x, v.y, w.x};
}
__device__ __forceinline__ int nb64(const R64 &r, int k) { return sel3(k, r.n0, r.n1, r.n2); }
__device__ __forceinline__ double cx64(const R64 &r, int k) { return sel3(k, 0.0, r.l01, r.x2x); }
__device__ __forceinline__ double cy64(const R64 &r, int k) { return sel3(k, 0.0, 0.0, r.x2y); }

// Walker state.  In the double-float half-edge mode (mode SG48_HALF) the FP64 registers hold
// double-float pairs instead (dpack): f = the half-edge id h, px = the fraction s along the entry
// edge, (dx, dy) = the direction in the edge frame, L = the remaining length, and R = the
// half-edge record (l01 = l, x2x = cx, x2y = cy, n0 = linkR, n1 = linkL).
struct W64 {
    int f, foff, mode, steps, ncross;
    uint32_t st;
    uint64_t hash;
    double px, py, dx, dy, L, lref;
    float nearf, snapf;  // tau_near l_ref, tau_snap l_ref (double-float mode)
    R64 R;
};

__device__ __forceinline__ void hash64(W64 &w, int f, int want) {
    if (want) {
        w.hash ^= (uint64_t)(uint32_t)(f - w.foff);
        w.hash *= SG_FNV_PRIME;
    }
}
__device__ __forceinline__ double sig64(const W64 &w, double cx, double cy) {
    return w.dx * (cy - w.py) - w.dy * (cx - w.px);
}
__device__ __forceinline__ void norm2(double &x, double &y) {
    const double r = 1.0 / sqrt(x * x + y * y);
    x *= r; y *= r;
}
// straightest rule at corner c of w.f (Alg. transport_over_vertex): the outgoing ray splits
// theta in two equal halves with the reversed incoming ray; the fan is walked toward corner c-1
template <int NW>
__device__ bool vertex64(W64 &w, int c, const P64 &P) {
    const int4 t = __ldg(P.fv + w.f);
    const double th = __ldg(P.th64 + sel3(c, t.x, t.y, t.z));
    w.st |= SG_ST_VERTEX_HIT;
    const double cx = cx64(w.R, c), cy = cy64(w.R, c);
    w.px = cx; w.py = cy;
    if (th < 0.0) {
        w.st |= SG_ST_BOUNDARY;
        return false;
    }
    const double half = 0.5 * th;
    const double rx = -w.dx, ry = -w.dy;
    int e = prv(c);
    const double ex = cx64(w.R, prv(c)) - cx, ey = cy64(w.R, prv(c)) - cy;
    double A = atan2(fabs(rx * ey - ry * ex), rx * ex + ry * ey);
    if (A >= half) {
        double hx = ex - (ex * rx + ey * ry) * rx, hy = ey - (ex * rx + ey * ry) * ry;
        norm2(hx, hy);
        double sh, ch;
        sincos(half, &sh, &ch);
        w.dx = ch * rx + sh * hx;
        w.dy = ch * ry + sh * hy;
        norm2(w.dx, w.dy);
        w.mode = 3 + c;
        hash64(w, w.f, P.want_hash);
        return true;
    }
    int cur_c = c;
    R64 Rc = w.R;
    for (int guard = 0; guard < 4096; ++guard) {
        const int nb = nb64(Rc, e);
        if (nb < 0) {
            w.st |= SG_ST_BOUNDARY;
            return false;
        }
        const int g = nb >> 3, kp = nb & 3, fl = (nb >> 2) & 1;
        if (fl) w.st ^= SG_PARITY_BIT;
        const R64 Rg = load64(P, g);
        const bool x_end_cur = (cur_c == nxt(e));
        const bool x_start_g = (x_end_cur != (bool)fl);
        const int cg = x_start_g ? kp : nxt(kp);
        const int yg = x_start_g ? nxt(kp) : kp;
        const int zg = 3 - cg - yg;
        const double gx = cx64(Rg, cg), gy = cy64(Rg, cg);
        double ux = cx64(Rg, yg) - gx, uy = cy64(Rg, yg) - gy;
        const double zx = cx64(Rg, zg) - gx, zy = cy64(Rg, zg) - gy;
        const double gam = atan2(fabs(ux * zy - uy * zx), ux * zx + uy * zy);
        if (A + gam >= half) {
            const double beta = half - A;
            norm2(ux, uy);
            double hx = zx - (zx * ux + zy * uy) * ux, hy = zy - (zx * ux + zy * uy) * uy;
            norm2(hx, hy);
            double sb, cb;
            sincos(beta, &sb, &cb);
            w.dx = cb * ux + sb * hx;
            w.dy = cb * uy + sb * hy;
            norm2(w.dx, w.dy);
            w.f = g;
            w.R = Rg;
            w.px = gx; w.py = gy;
            w.mode = 3 + cg;
            hash64(w, g, P.want_hash);
            return true;
        }
        A += gam;
        e = (nxt(cg) == zg) ? cg : zg;
        cur_c = cg;
        Rc = Rg;
    }
    w.st |= SG_ST_MAX_STEPS;
    return false;
}

// one step of Alg. geodesic_step in FP64 (same decisions as the FP32 general step)
template <int NW>
__device__ bool step64(W64 &w, const P64 &P) {
    if (w.steps >= P.max_steps) {
        w.st |= SG_ST_MAX_STEPS;
        return true;
    }
    w.steps++;
    const R64 &R = w.R;
    const double near = P.tau_near * w.lref, snap = P.tau_snap * w.lref;
    const double s0 = sig64(w, 0.0, 0.0), s1 = sig64(w, R.l01, 0.0), s2 = sig64(w, R.x2x, R.x2y);
    const int mode = w.mode;
    int j, hit = -1;
    double mflag;
    if (mode < 3) {
        const int k = mode, a = prv(k);
        const double sa = sel3(a, s0, s1, s2);
        mflag = fabs(sa);
        if (mflag <= snap) { hit = a; mflag = 3.0e300; }
        j = sa > 0.0 ? nxt(k) : prv(k);
    } else if (mode < 6) {
        const int c = mode - 3, a = nxt(c), b = prv(c);
        j = a;
        const double fa = fabs(sel3(a, s0, s1, s2)), fb = fabs(sel3(b, s0, s1, s2));
        mflag = fmin(fa, fb);
        if (mflag <= snap) { hit = fa <= fb ? a : b; mflag = fmax(fa, fb); }
    } else {
        if (s0 < 0.0 && s1 >= 0.0) j = 0;
        else if (s1 < 0.0 && s2 >= 0.0) j = 1;
        else if (s2 < 0.0 && s0 >= 0.0) j = 2;
        else { w.st |= SG_ST_INVALID; return true; }
        const double fa = fabs(sel3(j, s0, s1, s2)), fb = fabs(sel3(nxt(j), s0, s1, s2)), fo = fabs(sel3(prv(j), s0, s1, s2));
        mflag = fmin(fmin(fa, fb), fo);
        if (fmin(fa, fb) <= snap) { hit = fa <= fb ? j : nxt(j); mflag = fmin(fmax(fa, fb), fo); }
    }
    if (mflag < near) w.st |= SG_ST_NEAR_VERTEX;
    const int jb = nxt(j);
    const double ax = cx64(R, j), ay = cy64(R, j), bx = cx64(R, jb), by = cy64(R, jb);
    double qx, qy, s;
    if (hit >= 0) {
        qx = cx64(R, hit); qy = cy64(R, hit);
        s = (hit == j) ? 0.0 : 1.0;
    } else {
        const double sa = sel3(j, s0, s1, s2), sb = sel3(jb, s0, s1, s2);
        const double den = sa - sb;
        s = den != 0.0 ? sa / den : 0.5;
        s = fmin(fmax(s, 0.0), 1.0);
        qx = ax + s * (bx - ax);
        qy = ay + s * (by - ay);
    }
    const double t = fmax((qx - w.px) * w.dx + (qy - w.py) * w.dy, 0.0);
    if (t >= w.L) {
        w.px += w.L * w.dx;
        w.py += w.L * w.dy;
        w.L = 0.0;
        const double d0 = fabs(w.py);
        const double d1 = fabs((R.x2x - R.l01) * w.py - R.x2y * (w.px - R.l01)) * R.il1;
        const double d2 = fabs(R.x2x * w.py - R.x2y * w.px) * R.il2;
        if (fmin(fmin(d0, d1), d2) <= near) w.st |= SG_ST_NEAR_EDGE;
        return true;
    }
    w.L -= t;
    if (hit >= 0) return !vertex64<NW>(w, hit, P);
    const int nb = nb64(R, j);
    if (nb < 0) {
        w.px = qx; w.py = qy;
        w.st |= SG_ST_BOUNDARY;
        return true;
    }
    // into the frame of g: the shared edge is g's local edge kp (A' -> B'), reversed unless the
    // adjacency is flipped; g lies on the left of A' -> B' in its own frame
    const int g = nb >> 3, kp = nb & 3, fl = (nb >> 2) & 1;
    const R64 G = load64(P, g);
    const double ex = bx - ax, ey = by - ay, le = sqrt(ex * ex + ey * ey);
    const double ux = ex / le, uy = ey / le;
    const double da = w.dx * ux + w.dy * uy;           // along the edge (P_j -> P_j+1)
    const double dn = -w.dx * uy + w.dy * ux;          // along the inward normal of f (< 0 when leaving)
    const double Ax = cx64(G, kp), Ay = cy64(G, kp), Bx = cx64(G, nxt(kp)), By = cy64(G, nxt(kp));
    const double gx = Bx - Ax, gy = By - Ay, lg = sqrt(gx * gx + gy * gy);
    const double vx = gx / lg, vy = gy / lg;           // unit A' -> B'; g's inward normal = (-vy, vx)
    const double sgn = fl ? 1.0 : -1.0;                // image of the edge direction P_j -> P_j+1
    double ndx = sgn * da * vx - dn * -vy, ndy = sgn * da * vy - dn * vx;
    norm2(ndx, ndy);
    const double sp = fl ? s : 1.0 - s;                // fraction along A' -> B'
    w.px = Ax + sp * gx;
    w.py = Ay + sp * gy;
    w.dx = ndx; w.dy = ndy;
    w.f = g;
    w.R = G;
    w.mode = kp;
    if (fl) w.st ^= SG_PARITY_BIT;
    w.ncross++;
    hash64(w, g, P.want_hash);
    return false;
}

// ------------------------------------------------------------------ double-float walk
#define SG48_HALF 7
// the walk ended inside a face in the half-edge mode: px, py hold the end point in the edge frame
#define SG48_END 8

// the double-float half-edge record h into R: one 32-byte sector, one 256-bit load
__device__ __forceinline__ void load48(R64 &R, const P64 &P, int h) {
    int4 a, b;
    ld_rec32<true>(P.half48 + 2 * h, a, b);
    R.l01 = dpack(DF{__int_as_float(a.x), __int_as_float(a.y)});
    R.x2x = dpack(DF{__int_as_float(a.z), __int_as_float(a.w)});
    R.x2y = dpack(DF{__int_as_float(b.x), __int_as_float(b.y)});
    R.n0 = b.z;
    R.n1 = b.w;
}

// Leave the half-edge mode: the point (xe, ye) and direction (ex, ey) of the edge frame of w.f
// (a half-edge id) into the FP64 face frame of its face.
__device__ __forceinline__ void leave48(W64 &w, const P64 &P, DF xe, DF ye, DF ex, DF ey) {
    const int h = w.f, f = h / 3, k = h - 3 * f;
    const R64 F = load64(P, f);
    double ca = 1.0, sa = 0.0;
    if (k == 1) { ca = (F.x2x - F.l01) * F.il1; sa = F.x2y * F.il1; }
    else if (k == 2) { ca = -F.x2x * F.il2; sa = -F.x2y * F.il2; }
    const double x = df_to(xe), y = df_to(ye), dx = df_to(ex), dy = df_to(ey);
    w.px = cx64(F, k) + ca * x - sa * y;
    w.py = cy64(F, k) + sa * x + ca * y;
    w.dx = ca * dx - sa * dy;
    w.dy = sa * dx + ca * dy;
    w.f = f;
    w.R = F;
    w.mode = 6;
}

// Enter the half-edge mode after a face-frame step crossed into w.f through its local edge
// w.mode: the position as a fraction along that edge, the direction in the edge's frame.
__device__ __forceinline__ void enter48(W64 &w, const P64 &P) {
    const int k = w.mode;
    const R64 &G = w.R;
    const double ax = cx64(G, k), ay = cy64(G, k);
    const double ex = cx64(G, nxt(k)) - ax, ey = cy64(G, nxt(k)) - ay;
    const double l2 = ex * ex + ey * ey, il = 1.0 / sqrt(l2);
    const double s = fmin(fmax(((w.px - ax) * ex + (w.py - ay) * ey) / l2, 0.0), 1.0);
    const double hx = (w.dx * ex + w.dy * ey) * il, hy = (ex * w.dy - ey * w.dx) * il;
    const int h = 3 * w.f + k;
    load48(w.R, P, h);
    w.f = h;
    w.px = dpack(df_from(s));
    w.dx = dpack(df_from(hx));
    w.dy = dpack(df_from(hy));
    w.L = dpack(df_from(w.L));
    w.mode = SG48_HALF;
}

// One crossing in double-float arithmetic: the FP32 walk's half-edge step (orientation tests
// sigma_A = dy x, sigma_B = -dy (l - x), sigma_C = dx cy - dy (cx - x); exit B -> C when the apex
// lies left of the ray, else C -> A; the twin's frame has the crossed edge as its x axis).
template <int NW>
__device__ bool half48(W64 &w, const P64 &P) {
    const DF zero{0.f, 0.f}, one{1.f, 0.f};
    const DF L0 = dunpack(w.R.l01), cx = dunpack(w.R.x2x), cy = dunpack(w.R.x2y);
    const DF px = dunpack(w.px), dx = dunpack(w.dx), dy = dunpack(w.dy), Lr = dunpack(w.L);
    const DF x = df_mul(px, L0);
    const DF sA = df_mul(dy, x);
    const DF sB = df_neg(df_mul(dy, df_sub(L0, x)));
    const DF sC = df_sub(df_mul(dx, cy), df_mul(dy, df_sub(cx, x)));
    const float aC = fabsf(sC.hi);
    const bool hit = aC <= w.snapf;
    if (!hit && aC < w.nearf) w.st |= SG_ST_NEAR_VERTEX;
    const bool right = sC.hi > 0.f;
    // exit edge (x0, y0) -> (x0, y0) + (ex, ey): B -> C or C -> A
    const DF x0 = right ? L0 : cx, y0 = right ? zero : cy;
    const DF ex = right ? df_sub(cx, L0) : df_neg(cx), ey = right ? cy : df_neg(cy);
    DF qx, qy, s;
    if (hit) {
        qx = cx; qy = cy;
        s = right ? one : zero;
    } else {
        // s0 and s1 have opposite signs: their difference does not cancel
        const DF s0 = right ? sB : sC, s1 = right ? sC : sA;
        const DF den = df_add_same_sign(s0, df_neg(s1));
        s = den.hi != 0.f ? df_div(s0, den) : DF{0.5f, 0.f};
        if (s.hi < 0.f) s = zero;
        if (df_ge(s, one)) s = one;
        qx = df_add(x0, df_mul(s, ex));
        qy = df_add(y0, df_mul(s, ey));
    }
    DF t = df_add(df_mul(df_sub(qx, x), dx), df_mul(qy, dy));
    if (t.hi < 0.f) t = zero;
    const int k = w.f - 3 * (w.f / 3);
    if (df_ge(t, Lr)) {
        // final truncated in-face segment; the end point stays in the edge frame (SG48_END)
        const DF xe = df_add(x, df_mul(Lr, dx)), ye = df_mul(Lr, dy);
        // distances to the three edges: A -> B is the x axis; B -> C and C -> A by the cross
        // product with the edge vector over its FP32 length (a threshold needs no more)
        const DF bcx = df_sub(cx, L0);
        const DF cB = df_sub(df_mul(bcx, ye), df_mul(cy, df_sub(xe, L0)));
        const DF cA = df_sub(df_mul(cx, ye), df_mul(cy, xe));
        const float nb = sqrtf(fmaf(bcx.hi, bcx.hi, cy.hi * cy.hi)), na = sqrtf(fmaf(cx.hi, cx.hi, cy.hi * cy.hi));
        if (fabsf(ye.hi) <= w.nearf || fabsf(cB.hi) <= w.nearf * nb || fabsf(cA.hi) <= w.nearf * na)
            w.st |= SG_ST_NEAR_EDGE;
        w.px = dpack(xe);
        w.py = dpack(ye);
        w.L = 0.0;
        w.mode = SG48_END;
        return true;
    }
    const DF Ln = df_sub(Lr, t);
    if (hit) {  // the apex is corner k+2 of the face: the straightest rule in FP64
        leave48(w, P, cx, cy, dx, dy);
        w.L = df_to(Ln);
        return !vertex64<NW>(w, prv(k), P);
    }
    const int link = right ? w.R.n0 : w.R.n1;
    if (link < 0) {  // boundary edge: the walk stops (Sec. 4)
        leave48(w, P, qx, qy, dx, dy);
        w.L = df_to(Ln);
        w.st |= SG_ST_BOUNDARY;
        return true;
    }
    const int hn = link >> 1, fl = link & 1;
    const DF da = df_add(df_mul(dx, ex), df_mul(dy, ey));   // |e| (d . e_hat)
    const DF dc = df_sub(df_mul(dx, ey), df_mul(dy, ex));   // |e| (d . n_out)
    const DF re = df_rsqrt(df_add_same_sign(df_mul(da, da), df_mul(dc, dc)));
    const DF ndx = df_mul(fl ? da : df_neg(da), re), ndy = df_mul(dc, re);
    w.px = dpack(fl ? s : df_sub(one, s));
    w.dx = dpack(ndx);
    w.dy = dpack(ndy);
    w.L = dpack(Ln);
    load48(w.R, P, hn);
    w.f = hn;
    if (fl) w.st ^= SG_PARITY_BIT;
    w.ncross++;
    hash64(w, hn / 3, P.want_hash);
    return false;
}

// One step of the double-float walk: the half-edge step, or the FP64 face-frame step (after a
// vertex transport, or from a start the double-float start declined), whose crossings enter the
// half-edge mode.
template <int NW>
__device__ __forceinline__ bool step48(W64 &w, const P64 &P) {
    if (w.mode == SG48_HALF) {
        if (w.steps >= P.max_steps) {
            const DF px = dunpack(w.px), L0 = dunpack(w.R.l01);
            leave48(w, P, df_mul(px, L0), DF{0.f, 0.f}, dunpack(w.dx), dunpack(w.dy));
            w.L = 0.0;
            w.st |= SG_ST_MAX_STEPS;
            return true;
        }
        w.steps++;
        return half48<NW>(w, P);
    }
    const bool done = step64<NW>(w, P);
    if (!done && w.mode < 3) enter48(w, P);
    return done;
}

// ------------------------------------------------------------------ mixed-precision walk
// The error of the FP32 walk that grows with the path is the direction's: each crossing rotates
// the walking direction into the next edge frame with an FP32 edge vector and FP32 products, a
// rounding of about one unit in the last place of the angle, and the rotations' errors add up
// along the path while the position error they cause grows with the distance walked.  The error
// of the position itself does not grow that way: every crossing recomputes the exit point from
// the corners and the direction, so its rounding (about 1e-7 of the face size) enters once per
// crossing and adds up like a random walk.  The mixed walk (precision 40) therefore keeps the
// FP32 walk's arithmetic for the orientation tests, the exit point and the length, and carries
// only the direction in double-float: its rotation into the next frame uses the double-float
// edge vector of the double-float half-edge record (the record of the double-float walk, one
// 32-byte sector) and double-float products.  The start (double-float) and the rare events
// (FP64 face-frame code) are those of the double-float walk.
//
// Walker registers in the mixed half-edge mode: as in the double-float mode (px = the fraction s
// along the entry edge, (dx, dy) the direction, L the remaining length, all packed pairs), with
// only the high word of s and the pair L = Lh + Ll updated by FP32 steps.

template <int NW>
__device__ bool half40(W64 &w, const P64 &P) {
    const DF L0 = dunpack(w.R.l01), cx = dunpack(w.R.x2x), cy = dunpack(w.R.x2y);
    const DF dx = dunpack(w.dx), dy = dunpack(w.dy), Lr = dunpack(w.L);
    const float sp = dunpack(w.px).hi;
    const float l = L0.hi, x = sp * l, ddx = dx.hi, ddy = dy.hi;
    float sA = ddy * x, sB = -ddy * (l - x), sC = fmaf(ddx, cy.hi, -ddy * (cx.hi - x));
    if (fabsf(sC) < w.nearf) {
        // the classification in FP64 from the double-float record and direction
        w.st |= SG_ST_FP64;
        const double X = (double)sp * df_to(L0), DX = df_to(dx), DY = df_to(dy);
        sA = f32_keep_sign(DY * X);
        sB = f32_keep_sign(-DY * (df_to(L0) - X));
        sC = f32_keep_sign(DX * df_to(cy) - DY * (df_to(cx) - X));
    }
    const bool hit = fabsf(sC) <= w.snapf;
    if (!hit && fabsf(sC) < w.nearf) w.st |= SG_ST_NEAR_VERTEX;
    const bool right = sC > 0.f;
    const float x0 = right ? l : cx.hi, y0 = right ? 0.f : cy.hi;
    const float x1 = right ? cx.hi : 0.f, y1 = right ? cy.hi : 0.f;
    float qx, qy, s;
    if (hit) {
        qx = cx.hi; qy = cy.hi;
        s = right ? 1.f : 0.f;
    } else {
        const float s0 = right ? sB : sC, s1 = right ? sC : sA;
        const float den = s0 - s1;
        s = den != 0.f ? __fdividef(s0, den) : 0.5f;
        s = fminf(fmaxf(s, 0.f), 1.f);
        qx = fmaf(s, x1 - x0, x0);
        qy = fmaf(s, y1 - y0, y0);
    }
    const float t = fmaxf(fmaf(qx - x, ddx, qy * ddy), 0.f);
    const float Lf = Lr.hi + Lr.lo;
    const int k = w.f - 3 * (w.f / 3);
    if (t >= Lf) {
        // final truncated in-face segment; the end point stays in the edge frame (SG48_END)
        const float xe = fmaf(Lf, ddx, x), ye = Lf * ddy;
        const float bcx = cx.hi - l;
        const float cB = fabsf(bcx * ye - cy.hi * (xe - l)) * rsqrtf(fmaf(bcx, bcx, cy.hi * cy.hi));
        const float cA = fabsf(cx.hi * ye - cy.hi * xe) * rsqrtf(fmaf(cx.hi, cx.hi, cy.hi * cy.hi));
        if (fminf(fminf(fabsf(ye), cB), cA) <= w.nearf) w.st |= SG_ST_NEAR_EDGE;
        w.px = dpack(DF{xe, 0.f});
        w.py = dpack(DF{ye, 0.f});
        w.L = 0.0;
        w.mode = SG48_END;
        return true;
    }
    // compensated L -= t (t < Lh + Ll: Dekker's fast two-sum gives the exact rounding error)
    const float Lh = Lr.hi - t;
    const DF Ln{Lh, Lr.lo + (-t - (Lh - Lr.hi))};
    if (hit) {  // the apex is corner k+2 of the face: the straightest rule in FP64
        leave48(w, P, cx, cy, dx, dy);
        w.L = df_to(Ln);
        return !vertex64<NW>(w, prv(k), P);
    }
    const int link = right ? w.R.n0 : w.R.n1;
    if (link < 0) {  // boundary edge: the walk stops (Sec. 4)
        leave48(w, P, DF{qx, 0.f}, DF{qy, 0.f}, dx, dy);
        w.L = df_to(Ln);
        w.st |= SG_ST_BOUNDARY;
        return true;
    }
    const int hn = link >> 1, fl = link & 1;
    // the exit edge vector in double-float: B -> C = (cx - l, cy), C -> A = -(cx, cy)
    const DF ex = right ? df_sub(cx, L0) : df_neg(cx), ey = right ? cy : df_neg(cy);
    const DF da = df_dot2(dx, ex, dy, ey);            // |e| (d . e_hat)
    const DF dc = df_dot2(dx, ey, df_neg(dy), ex);    // |e| (d . n_out)
    // one FP32 scale for both components keeps the direction's angle to double-float precision;
    // its norm is 1 to FP32 precision, which only scales the next step's orientation tests
    const float re = rsqrtf(fmaf(da.hi, da.hi, dc.hi * dc.hi));
    w.px = dpack(DF{fl ? s : 1.f - s, 0.f});
    w.dx = dpack(df_mul_f(fl ? da : df_neg(da), re));
    w.dy = dpack(df_mul_f(dc, re));
    w.L = dpack(Ln);
    load48(w.R, P, hn);
    w.f = hn;
    if (fl) w.st ^= SG_PARITY_BIT;
    w.ncross++;
    hash64(w, hn / 3, P.want_hash);
    return false;
}

template <int NW>
__device__ __forceinline__ bool step40(W64 &w, const P64 &P) {
    if (w.mode == SG48_HALF) {
        if (w.steps >= P.max_steps) {
            const DF L0 = dunpack(w.R.l01);
            leave48(w, P, DF{dunpack(w.px).hi * L0.hi, 0.f}, DF{0.f, 0.f}, dunpack(w.dx), dunpack(w.dy));
            w.L = 0.0;
            w.st |= SG_ST_MAX_STEPS;
            return true;
        }
        w.steps++;
        return half40<NW>(w, P);
    }
    const bool done = step64<NW>(w, P);
    if (!done && w.mode < 3) enter48(w, P);
    return done;
}

}  // namespace
