// exp_map64.cu -- the full-precision walk (sg_opts.precision = 64).
//
// The same straightest-geodesic walk as walk.cuh (Alg. geodesic_step, transport_over_edge,
// transport_over_vertex; Sec. 4), with every quantity of the walker state and of the face
// geometry in FP64: the position, direction and remaining length, the face shapes, frames and
// vertex angles.  It serves inputs where the FP32 walk's accumulated error exceeds the
// classification margins (long walks over sliver triangles), at the cost of FP64 arithmetic.
// The walker stays in the face frames (no half-edge records); a crossing maps it into the
// neighbour's frame through the shared edge, the unfolding isometry of Sec. 4.
//
// The FP64 geometry is derived on the device from the mesh's vertex positions (converted to
// FP64) the first time a call asks for it, and again after sg_mesh_update_vertices.
//
// The double-float walk (sg_opts.precision = 48) reaches the same accuracy class on the FP32
// pipes: its hot step is the FP32 walk's half-edge step (one 32-byte record per crossing, in the
// entry edge's frame) with every quantity an unevaluated sum hi + lo of two FP32 numbers, about
// 48 significant bits.  GB300 runs FP64 at a small fraction of its FP32 rate, so the double-float
// step, several times the FP32 step's instructions, is still far faster than the FP64 step.  The
// start and the end are double-float too; rare events (vertex hits, boundary stops, starts on an
// edge or vertex, MAX_STEPS) use the FP64 face-frame code below.
#include <cuda_runtime.h>

#include <algorithm>

#include "sgeo_internal.h"
#include "walk.cuh"

#include "walk64.cuh"

namespace {

struct Fwd64Args {
    P64 P;
    QueryIn in;
    int64_t nq;
    int32_t *out_face;
    float *out_bary, *out_pos, *out_dir, *out_w;
    uint32_t *out_status;
    int32_t *out_ncross;
    uint64_t *out_hash;
    const int32_t *__restrict__ perm;
    int32_t *counter;
};


// PREC 64: the FP64 walk; 48: the double-float walk
template <int NW, int PREC = 64>
struct Job64 {
    static constexpr bool DFW = PREC != 64;
    const Fwd64Args *a;
    W64 w;
    double cc[NW > 0 ? NW : 1], cs[NW > 0 ? NW : 1];
    int64_t q;

    __device__ __forceinline__ bool init(int64_t t) {
        q = a->perm ? (int64_t)__ldg(a->perm + t) : t;
        const P64 &P = a->P;
        const QueryIn &in = a->in;
        const int m = in.mesh_id ? __ldg(in.mesh_id + q) : 0;
        const int lf = __ldg(in.face + q);
        w.st = 0; w.steps = 0; w.ncross = 0; w.hash = SG_FNV_OFFSET; w.mode = 6;
        bool bad = (m < 0 || m >= in.n_mesh);
        const int foff = bad ? 0 : __ldg(P.face_off + m);
        const int nfm = bad ? 1 : __ldg(P.face_off + m + 1) - foff;
        bad = bad || lf < 0 || lf >= nfm;
        const float lr = bad ? 1.f : __ldg(P.lref + m);
        bad = bad || !(lr > 0.f);
        w.foff = foff;
        w.f = bad ? foff : foff + lf;
        w.lref = bad ? 1.0 : (double)lr;
        w.R = load64(P, w.f);
        double b0 = __ldg(in.bary + 3 * q), b1 = __ldg(in.bary + 3 * q + 1), b2 = __ldg(in.bary + 3 * q + 2);
        const double sb = b0 + b1 + b2;
        if (!(fabs(sb - 1.0) <= 1e-6) || b0 < -1e-7 || b1 < -1e-7 || b2 < -1e-7) bad = true;
        for (int k = 0; k < NW; ++k) { cc[k] = 0.0; cs[k] = 0.0; }
        w.px = w.py = w.dx = w.dy = 0.0; w.L = 0.0;
        if (bad) { w.st |= SG_ST_INVALID; return false; }
        w.nearf = (float)(P.tau_near * w.lref);
        w.snapf = (float)(P.tau_snap * w.lref);
        if (DFW) {
            const int r = start48();
            if (r >= 0) return r != 0;
        }
        b0 = fmax(b0, 0.0) / sb; b1 = fmax(b1, 0.0) / sb; b2 = fmax(b2, 0.0) / sb;
        w.px = b1 * w.R.l01 + b2 * w.R.x2x;
        w.py = b2 * w.R.x2y;
        const double *fr = P.frm64 + 6 * w.f;
        const double vx = __ldg(in.v + 3 * q), vy = __ldg(in.v + 3 * q + 1), vz = __ldg(in.v + 3 * q + 2);
        const double v1 = vx * fr[0] + vy * fr[1] + vz * fr[2], v2 = vx * fr[3] + vy * fr[4] + vz * fr[5];
        const double Lv = sqrt(v1 * v1 + v2 * v2);
        const double L = in.length ? (double)__ldg(in.length + q) : Lv;
        if (!(L >= 0.0 && L <= 1.0e300) || !(Lv <= 1.0e300) || (Lv == 0.0 && L > 0.0)) { w.st |= SG_ST_INVALID; return false; }
        if (Lv > 0.0) { w.dx = v1 / Lv; w.dy = v2 / Lv; }
        w.L = L;
        const double rx = Lv > 0.0 ? w.dx : 1.0, ry = Lv > 0.0 ? w.dy : 0.0;  // zero v: against e1
        for (int k = 0; k < NW; ++k) {
            const float *wp = in.w + (3 * NW) * q + 3 * k;
            const double wx = __ldg(wp), wy = __ldg(wp + 1), wz = __ldg(wp + 2);
            const double w1 = wx * fr[0] + wy * fr[1] + wz * fr[2], w2 = wx * fr[3] + wy * fr[4] + wz * fr[5];
            cc[k] = w1 * rx + w2 * ry;
            cs[k] = rx * w2 - ry * w1;
        }
        const int zeros = (b0 == 0.0) + (b1 == 0.0) + (b2 == 0.0);
        if (zeros) w.st |= SG_ST_START_ON_EDGE;
        if (zeros == 2 && L > 0.0) {
            const int c = b0 == 1.0 ? 0 : (b1 == 1.0 ? 1 : 2);
            const double cx = cx64(w.R, c), cy = cy64(w.R, c);
            const double ax = cx64(w.R, nxt(c)) - cx, ay = cy64(w.R, nxt(c)) - cy;
            const double bx = cx64(w.R, prv(c)) - cx, by = cy64(w.R, prv(c)) - cy;
            if (!(ax * w.dy - ay * w.dx > 0.0 && w.dx * by - w.dy * bx > 0.0)) {
                w.st |= SG_ST_INVALID;
                w.L = 0.0;
                return false;
            }
            w.px = cx; w.py = cy;
            w.mode = 3 + c;
        }
        if (L > 0.0) hash64(w, w.f, P.want_hash);
        return L > 0.0;
    }

    // Double-float start: the start point, direction and length in double-float arithmetic, and
    // the walker placed on the edge through which its ray enters the start face (behind the
    // start point, the length extended by that distance), so the walk begins in the half-edge
    // mode with no FP64 division or square root.  Returns 1 (a walk), or -1 for the FP64 start:
    // a start on an edge or a vertex, a zero, huge or non-finite vector or length, or an
    // entry-edge corner within the near band of the ray line (the FP64 step classifies those).
    __device__ __forceinline__ int start48() {
        const P64 &P = a->P;
        const QueryIn &in = a->in;
        const float b0 = __ldg(in.bary + 3 * q), b1 = __ldg(in.bary + 3 * q + 1), b2 = __ldg(in.bary + 3 * q + 2);
        if (!(b0 > 0.f && b1 > 0.f && b2 > 0.f)) return -1;
        R64 H;
        load48(H, P, 3 * w.f);  // the record of edge 0 is the face frame: l01, (x2x, x2y)
        const DF l01 = dunpack(H.l01), x2x = dunpack(H.x2x), x2y = dunpack(H.x2y);
        const DF sb = df_add(two_sum(b0, b1), DF{b2, 0.f});
        const DF rs = df_div(DF{1.f, 0.f}, sb);
        const DF B1 = df_mul_f(rs, b1), B2 = df_mul_f(rs, b2);
        const DF px = df_add_same_sign(df_mul(B1, l01), df_mul(B2, x2x)), py = df_mul(B2, x2y);
        const double *fr = P.frm64 + 6 * w.f;
        const double vx = __ldg(in.v + 3 * q), vy = __ldg(in.v + 3 * q + 1), vz = __ldg(in.v + 3 * q + 2);
        const DF V1 = df_from(vx * fr[0] + vy * fr[1] + vz * fr[2]), V2 = df_from(vx * fr[3] + vy * fr[4] + vz * fr[5]);
        const DF n2 = df_add_same_sign(df_mul(V1, V1), df_mul(V2, V2));
        if (!(n2.hi > 1e-30f && n2.hi < 1e30f)) return -1;
        const DF rn = df_rsqrt(n2);
        const DF dx = df_mul(V1, rn), dy = df_mul(V2, rn);
        DF L = df_mul(n2, rn);
        if (in.length) {
            const float Li = __ldg(in.length + q);
            if (!(Li > 0.f && Li < 1e30f)) return -1;
            L = DF{Li, 0.f};
        }
        // corners' signed distances to the ray line; the ray enters through edge j with corner j
        // on its left and corner j+1 on its right
        const DF zero{0.f, 0.f};
        const DF s0 = df_sub(df_mul(dy, px), df_mul(dx, py));
        const DF s1 = df_sub(df_mul(dx, df_neg(py)), df_mul(dy, df_sub(l01, px)));
        const DF s2 = df_sub(df_mul(dx, df_sub(x2y, py)), df_mul(dy, df_sub(x2x, px)));
        int j;
        if (s0.hi > 0.f && s1.hi <= 0.f) j = 0;
        else if (s1.hi > 0.f && s2.hi <= 0.f) j = 1;
        else if (s2.hi > 0.f && s0.hi <= 0.f) j = 2;
        else return -1;
        const DF sa = j == 0 ? s0 : (j == 1 ? s1 : s2), sbb = j == 0 ? s1 : (j == 1 ? s2 : s0);
        if (fabsf(sa.hi) < w.nearf || fabsf(sbb.hi) < w.nearf) return -1;
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
        if (!(hy.hi > 0.f)) return -1;
        const double rx = df_to(dx), ry = df_to(dy);
        for (int k = 0; k < NW; ++k) {
            const float *wp = in.w + (3 * NW) * q + 3 * k;
            const double wx = __ldg(wp), wy = __ldg(wp + 1), wz = __ldg(wp + 2);
            const double w1 = wx * fr[0] + wy * fr[1] + wz * fr[2], w2 = wx * fr[3] + wy * fr[4] + wz * fr[5];
            cc[k] = w1 * rx + w2 * ry;
            cs[k] = rx * w2 - ry * w1;
        }
        hash64(w, w.f, P.want_hash);
        const int h = 3 * w.f + j;
        load48(w.R, P, h);
        w.f = h;
        w.px = dpack(se);
        w.py = 0.0;
        w.dx = dpack(hx);
        w.dy = dpack(hy);
        w.L = dpack(df_add_same_sign(L, tb));
        w.mode = SG48_HALF;
        return 1;
    }
    __device__ __forceinline__ bool step() {
        return PREC == 48 ? step48<NW>(w, a->P) : step64<NW>(w, a->P);
    }
    // The end of a double-float walk that stopped inside a face in the half-edge mode: the
    // outputs (float32) from the double-float end point, with FP32 rotations and frames.
    __device__ __forceinline__ void finish48() {
        const Fwd64Args &A = *a;
        const int h = w.f, f = h / 3, k = h - 3 * f;
        const DF L0 = dunpack(w.R.l01), cx = dunpack(w.R.x2x), cy = dunpack(w.R.x2y);
        const DF xe = dunpack(w.px), ye = dunpack(w.py);
        const DF bC = df_div(ye, cy);
        const DF bB = df_div(df_sub(xe, df_mul(bC, cx)), L0);
        const DF bA = df_sub(df_sub(DF{1.f, 0.f}, bB), bC);
        float b[3];
        b[k] = bA.hi; b[nxt(k)] = bB.hi; b[prv(k)] = bC.hi;
        const int4 t = __ldg(A.P.fv + f);
        const float4 x0 = __ldg(A.P.V + t.x), x1 = __ldg(A.P.V + t.y), x2 = __ldg(A.P.V + t.z);
        A.out_face[q] = f - w.foff;
        A.out_bary[3 * q] = b[0]; A.out_bary[3 * q + 1] = b[1]; A.out_bary[3 * q + 2] = b[2];
        A.out_pos[3 * q] = fmaf(b[0], x0.x, fmaf(b[1], x1.x, b[2] * x2.x));
        A.out_pos[3 * q + 1] = fmaf(b[0], x0.y, fmaf(b[1], x1.y, b[2] * x2.y));
        A.out_pos[3 * q + 2] = fmaf(b[0], x0.z, fmaf(b[1], x1.z, b[2] * x2.z));
        // direction: edge frame -> face frame (the edge's rotation) -> 3-D (the face axes)
        const int4 hr = __ldg(A.P.half + 2 * h + 1);
        const float ca = __int_as_float(hr.y), sa = __int_as_float(hr.z);
        const float hx = dunpack(w.dx).hi, hy = dunpack(w.dy).hi;
        const float rx = ca * hx - sa * hy, ry = sa * hx + ca * hy;
        const float4 fa = __ldg(A.P.frm + 2 * f), fb = __ldg(A.P.frm + 2 * f + 1);
        A.out_dir[3 * q] = rx * fa.x + ry * fa.w;
        A.out_dir[3 * q + 1] = rx * fa.y + ry * fb.x;
        A.out_dir[3 * q + 2] = rx * fa.z + ry * fb.y;
        if (NW > 0 && A.out_w) {
            const float sg = (w.st & SG_PARITY_BIT) ? -1.f : 1.f;
            for (int i = 0; i < NW; ++i) {
                const float c = (float)cc[i], s = sg * (float)cs[i];
                const float u1 = c * rx - s * ry, u2 = c * ry + s * rx;
                float *o = A.out_w + (3 * NW) * q + 3 * i;
                o[0] = u1 * fa.x + u2 * fa.w;
                o[1] = u1 * fa.y + u2 * fb.x;
                o[2] = u1 * fa.z + u2 * fb.y;
            }
        }
        A.out_status[q] = (w.st & ~SG_PARITY_BIT) | ((w.st & SG_PARITY_BIT) ? SG_ST_FLIPPED : 0u);
        if (A.out_ncross) A.out_ncross[q] = w.ncross;
        if (A.out_hash) A.out_hash[q] = w.hash;
    }

    __device__ __forceinline__ void finish() {
        if (DFW && w.mode == SG48_END) {
            finish48();
            return;
        }
        const Fwd64Args &A = *a;
        const R64 &R = w.R;
        const double b2 = w.py / R.x2y, b1 = (w.px - b2 * R.x2x) / R.l01, b0 = 1.0 - b1 - b2;
        const int4 t = __ldg(A.P.fv + w.f);
        const float4 x0 = __ldg(A.P.V + t.x), x1 = __ldg(A.P.V + t.y), x2 = __ldg(A.P.V + t.z);
        const double *fr = A.P.frm64 + 6 * w.f;
        A.out_face[q] = w.f - w.foff;
        A.out_bary[3 * q] = (float)b0; A.out_bary[3 * q + 1] = (float)b1; A.out_bary[3 * q + 2] = (float)b2;
        A.out_pos[3 * q] = (float)(b0 * x0.x + b1 * x1.x + b2 * x2.x);
        A.out_pos[3 * q + 1] = (float)(b0 * x0.y + b1 * x1.y + b2 * x2.y);
        A.out_pos[3 * q + 2] = (float)(b0 * x0.z + b1 * x1.z + b2 * x2.z);
        A.out_dir[3 * q] = (float)(w.dx * fr[0] + w.dy * fr[3]);
        A.out_dir[3 * q + 1] = (float)(w.dx * fr[1] + w.dy * fr[4]);
        A.out_dir[3 * q + 2] = (float)(w.dx * fr[2] + w.dy * fr[5]);
        if (NW > 0 && A.out_w) {
            const double sg = (w.st & SG_PARITY_BIT) ? -1.0 : 1.0;
            const bool nod = w.dx == 0.0 && w.dy == 0.0;
            const double rx = nod ? 1.0 : w.dx, ry = nod ? 0.0 : w.dy;
            for (int k = 0; k < NW; ++k) {
                const double c = cc[k], s = sg * cs[k];
                const double u1 = c * rx - s * ry, u2 = c * ry + s * rx;
                float *o = A.out_w + (3 * NW) * q + 3 * k;
                o[0] = (float)(u1 * fr[0] + u2 * fr[3]);
                o[1] = (float)(u1 * fr[1] + u2 * fr[4]);
                o[2] = (float)(u1 * fr[2] + u2 * fr[5]);
            }
        }
        A.out_status[q] = (w.st & ~SG_PARITY_BIT) | ((w.st & SG_PARITY_BIT) ? SG_ST_FLIPPED : 0u);
        if (A.out_ncross) A.out_ncross[q] = w.ncross;
        if (A.out_hash) A.out_hash[q] = w.hash;
    }
};

template <int NW>
__global__ void __launch_bounds__(128) k_walk64(Fwd64Args a) {
    Job64<NW> job;
    job.a = &a;
    run_persistent(a.counter, a.nq, job);
}

// resident blocks per SM the double-float walk is compiled for (icosphere s6, 1M queries: 4
// blocks 4.95 ms, 5 blocks 4.59 ms with a few spills, 3 blocks 4.95 ms)
#ifndef SG_WALK48_MINB
#define SG_WALK48_MINB 5
#endif
template <int NW>
__global__ void __launch_bounds__(128, SG_WALK48_MINB) k_walk48(Fwd64Args a) {
    Job64<NW, 48> job;
    job.a = &a;
    run_persistent(a.counter, a.nq, job);
}

// Double-float half-edge records from the FP64 face shapes, in the layout of the FP32 half-edge
// records (origin at corner k, x along edge k, the face on +y): {l, cx} and {cy, linkR, linkL},
// each value split into hi + lo; the links are those of the FP32 records.
__global__ void k_half48(int64_t nH, const int4 *__restrict__ half, const double *__restrict__ rec64, int4 *half48) {
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= nH) return;
    const int64_t f = h / 3;
    const int k = (int)(h - 3 * f), k1 = nxt(k), k2 = prv(k);
    const double *r = rec64 + 6 * f;
    const double Px[3] = {0.0, r[0], r[1]}, Py[3] = {0.0, 0.0, r[2]};
    const double ex = Px[k1] - Px[k], ey = Py[k1] - Py[k];
    const double l = sqrt(ex * ex + ey * ey);
    const double rx = Px[k2] - Px[k], ry = Py[k2] - Py[k];
    const double cx = (rx * ex + ry * ey) / l, cy = (ex * ry - ey * rx) / l;
    const DF L = df_from(l), X = df_from(cx), Y = df_from(cy);
    half48[2 * h] = make_int4(__float_as_int(L.hi), __float_as_int(L.lo), __float_as_int(X.hi), __float_as_int(X.lo));
    half48[2 * h + 1] = make_int4(__float_as_int(Y.hi), __float_as_int(Y.lo), half[2 * h].w, half[2 * h + 1].x);
}

// FP64 geometry from the FP32 vertex positions (converted exactly), the same expressions as
// the host builder: face shape and frame, corner angles summed into theta
__global__ void k_geom64_faces(int64_t nF, const int4 *__restrict__ fv, const float4 *__restrict__ V, double *rec64,
                               double *frm64, double *th64) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nF) return;
    const int4 t = fv[f];
    const float4 a = V[t.x], b = V[t.y], c = V[t.z];
    const double x0[3] = {a.x, a.y, a.z}, x1[3] = {b.x, b.y, b.z}, x2[3] = {c.x, c.y, c.z};
    double e1[3], e2[3], n[3];
    for (int i = 0; i < 3; ++i) { e1[i] = x1[i] - x0[i]; e2[i] = x2[i] - x0[i]; }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const double l01 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    double u[3], nh[3], w[3];
    for (int i = 0; i < 3; ++i) { u[i] = e1[i] * (1.0 / l01); nh[i] = n[i] * (1.0 / nn); }
    w[0] = nh[1] * u[2] - nh[2] * u[1];
    w[1] = nh[2] * u[0] - nh[0] * u[2];
    w[2] = nh[0] * u[1] - nh[1] * u[0];
    const double x2x = e2[0] * u[0] + e2[1] * u[1] + e2[2] * u[2];
    const double x2y = e2[0] * w[0] + e2[1] * w[1] + e2[2] * w[2];
    const double d12[3] = {x2[0] - x1[0], x2[1] - x1[1], x2[2] - x1[2]};
    const double l12 = sqrt(d12[0] * d12[0] + d12[1] * d12[1] + d12[2] * d12[2]);
    const double l20 = sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
    double *r = rec64 + 6 * f;
    r[0] = l01; r[1] = x2x; r[2] = x2y; r[3] = 1.0 / l12; r[4] = 1.0 / l20; r[5] = 0.0;
    double *fr = frm64 + 6 * f;
    fr[0] = u[0]; fr[1] = u[1]; fr[2] = u[2]; fr[3] = w[0]; fr[4] = w[1]; fr[5] = w[2];
    const double *X[3] = {x0, x1, x2};
    const int tv[3] = {t.x, t.y, t.z};
    for (int k = 0; k < 3; ++k) {
        const double *p = X[k], *q1 = X[(k + 1) % 3], *q2 = X[(k + 2) % 3];
        const double ea[3] = {q1[0] - p[0], q1[1] - p[1], q1[2] - p[2]}, eb[3] = {q2[0] - p[0], q2[1] - p[1], q2[2] - p[2]};
        const double cr[3] = {ea[1] * eb[2] - ea[2] * eb[1], ea[2] * eb[0] - ea[0] * eb[2], ea[0] * eb[1] - ea[1] * eb[0]};
        atomicAdd(th64 + tv[k], atan2(sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]),
                                      ea[0] * eb[0] + ea[1] * eb[1] + ea[2] * eb[2]));
    }
}

// boundary vertices carry the sign of the FP32 theta (negative)
__global__ void k_geom64_sign(int64_t nV, const float4 *__restrict__ V, double *th64) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    if (signbit(V[v].w)) th64[v] = -th64[v];
}

}  // namespace

// Builds (first use) or refreshes (after a vertex update) the FP64 geometry, on `s`; with
// half48 also the double-float half-edge records of the double-float walk.
sg_status sg_geom64_prepare(sg_mesh *m, cudaStream_t s, bool half48) {
    if (!m->d_rec64) {
        const size_t b0 = sizeof(double) * 6 * (size_t)m->nF, b1 = b0, b2 = sizeof(double) * (size_t)m->nV;
        if (cudaMalloc((void **)&m->d_rec64, b0) != cudaSuccess || cudaMalloc((void **)&m->d_frm64, b1) != cudaSuccess ||
            cudaMalloc((void **)&m->d_th64, b2) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(m->d_rec64); cudaFree(m->d_frm64); cudaFree(m->d_th64);
            m->d_rec64 = m->d_frm64 = m->d_th64 = nullptr;
            return SG_ERR_OOM;
        }
        m->device_bytes += (int64_t)(b0 + b1 + b2);
        m->geom64_stale = true;
    }
    if (m->geom64_stale) {
        if (cudaMemsetAsync(m->d_th64, 0, sizeof(double) * (size_t)m->nV, s) != cudaSuccess) return SG_ERR_CUDA;
        k_geom64_faces<<<(unsigned)((m->nF + 255) / 256), 256, 0, s>>>(m->nF, m->d_fv, m->d_V, m->d_rec64, m->d_frm64,
                                                                      m->d_th64);
        k_geom64_sign<<<(unsigned)((m->nV + 255) / 256), 256, 0, s>>>(m->nV, m->d_V, m->d_th64);
        if (cudaGetLastError() != cudaSuccess) return SG_ERR_CUDA;
        m->geom64_stale = false;
        m->half48_stale = true;
    }
    if (half48) {
        if (!m->d_half48) {
            const size_t b = sizeof(int4) * 6 * (size_t)m->nF;
            if (cudaMalloc((void **)&m->d_half48, b) != cudaSuccess) {
                cudaGetLastError();
                m->d_half48 = nullptr;
                return SG_ERR_OOM;
            }
            m->device_bytes += (int64_t)b;
            m->half48_stale = true;
        }
        if (m->half48_stale) {
            const int64_t nH = 3 * m->nF;
            k_half48<<<(unsigned)((nH + 255) / 256), 256, 0, s>>>(nH, m->d_half, m->d_rec64, m->d_half48);
            if (cudaGetLastError() != cudaSuccess) return SG_ERR_CUDA;
            m->half48_stale = false;
        }
    }
    return SG_OK;
}

cudaError_t sg_launch_walk64(const sg_mesh *m, const SgFwdIO &io, int n_w, const sg_opts &r, cudaStream_t s) {
    Fwd64Args a{};
    a.P.rec = m->d_rec; a.P.rec64 = m->d_rec64; a.P.frm64 = m->d_frm64; a.P.th64 = m->d_th64;
    a.P.half48 = m->d_half48;
    a.P.half = m->d_half; a.P.frm = m->d_frm;
    a.P.fv = m->d_fv; a.P.V = m->d_V; a.P.face_off = m->d_face_off; a.P.lref = m->d_lref;
    a.P.max_steps = r.max_steps; a.P.want_hash = io.out_hash != nullptr;
    a.P.tau_near = r.tau_near; a.P.tau_snap = r.tau_snap;
    a.in = io.in; a.nq = io.nq;
    a.out_face = io.out_face; a.out_bary = io.out_bary; a.out_pos = io.out_pos; a.out_dir = io.out_dir;
    a.out_w = io.out_w; a.out_status = io.out_status; a.out_ncross = io.out_ncross; a.out_hash = io.out_hash;
    a.perm = io.perm; a.counter = io.counter;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto go = [&](auto kern) {
        int per = r.blocks_per_sm;
        if (per <= 0) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 128, 0);
            per = std::max(per, 1);
        }
        const int64_t grid = std::min<int64_t>((int64_t)sms * per, std::max<int64_t>((io.nq + 127) / 128, 1));
        kern<<<(unsigned)grid, 128, 0, s>>>(a);
    };
    if (r.precision == 48) {
        switch (n_w) {
            case 0: go(k_walk48<0>); break;
            case 1: go(k_walk48<1>); break;
            case 2: go(k_walk48<2>); break;
            case 3: go(k_walk48<3>); break;
            default: go(k_walk48<4>); break;
        }
    } else {
        switch (n_w) {
            case 0: go(k_walk64<0>); break;
            case 1: go(k_walk64<1>); break;
            case 2: go(k_walk64<2>); break;
            case 3: go(k_walk64<3>); break;
            default: go(k_walk64<4>); break;
        }
    }
    return cudaGetLastError();
}
