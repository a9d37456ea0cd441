// backward.cu -- vector-Jacobian products of the exponential map (Sec. 4 "Differentiation").
//
// EP (Eq. "proxy_func"): J^v = R, the rotation taking the start frame [v/|v|, n x v/|v|, n]
// to the same frame transported to the end point; J^p is zeroed.  In the intrinsic 2-D
// frames R maps a start vector x to (x.d0) d' + s (x.perp(d0)) perp(d'), s = -1 when the end
// face is reached through an odd number of orientation flips.  So the VJP is
//   grad_v = F0 gbar0,   gbar0 = a d0 + s b perp(d0),   a = gm.d', b = gm.perp(d'),
// gm = the upstream gradient in the end frame.  No walk is needed (k_ep_backward).
//
// GFD (Eqs. "jv", "jp", two batched rounds in App. "Speed-up GFD and EP through
// batching"): columns (Exp(perturbed) - p') / eps projected on the end plane, for the
// perturbations v+eps e_par (= a short walk eps beyond p'), v+eps e_perp, p+eps e_u and
// p+eps e_v.  In the development of the base ray's face strip the exponential map is
// Exp = p + v, so a perturbed ray that sees the same strip ends at p' + R delta exactly.
// k_rewalk therefore re-walks the base ray once and tests every corner it meets against
// the thin regions swept by the perturbations (a wedge for e_perp, parallelograms for e_u,
// e_v).  A perturbation that sweeps no vertex ("no split") is evaluated as the 3-D chord of
// a short walk from p' along R delta (this keeps the end-face geometry exact and avoids
// cancellation); one that sweeps a vertex, or any perturbation of a walk that stopped on
// the boundary, is evaluated by the literal independent walk, as in the paper.
//
// grad_V (vertex positions; not in the paper): the a.e. derivative of p' with the face
// sequence fixed.  The end point is a chain of rigid 2-D maps T (one per crossing) applied
// to p0 + v; each T depends on the corners of the shared edge in the two faces.  The
// adjoint of T at a crossing needs the end point expressed in the old frame
// (y = q + L_rem d) and the upstream gradient in the new frame, which is the end-frame
// gradient parallel-transported back (gbar_i = a d_i + s_i b perp(d_i)), so one forward
// re-walk accumulates everything (no stored path).  2-D corner gradients map to 3-D by the
// face frame F (in-plane); start and end faces add b_k F gbar0 and b'_k (g.n) n, plus a
// tilt term when v has a normal component.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "sgeo_internal.h"
#include "walk.cuh"

struct BwdArgs {
    WalkParams P;
    QueryIn in;
    int64_t nq;
    const int32_t *__restrict__ end_face;
    const float *__restrict__ end_bary;
    const float *__restrict__ end_dir;
    const uint32_t *__restrict__ end_status;
    const float *__restrict__ g_pos;
    float *grad_v, *grad_p, *grad_bary, *grad_V;
    uint32_t *out_status;
    float eps_v, eps_p;
};

struct F3 {
    float x, y, z;
};
__device__ __forceinline__ F3 f3(float x, float y, float z) { return F3{x, y, z}; }
__device__ __forceinline__ F3 operator+(F3 a, F3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ F3 operator-(F3 a, F3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ F3 operator*(float s, F3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ F3 cross3(F3 a, F3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ F3 e1_of(const Frame3 &F) { return f3(F.e1x, F.e1y, F.e1z); }
__device__ __forceinline__ F3 e2_of(const Frame3 &F) { return f3(F.e2x, F.e2y, F.e2z); }
__device__ __forceinline__ F3 lift(const Frame3 &F, float a, float b) { return a * e1_of(F) + b * e2_of(F); }
__device__ __forceinline__ F3 nrm_of(const Frame3 &F) { return cross3(e1_of(F), e2_of(F)); }
__device__ __forceinline__ F3 vtx(const Frame3 &F, int k) {
    return k == 0 ? f3(F.ox, F.oy, F.oz) : (k == 1 ? f3(F.x1x, F.x1y, F.x1z) : f3(F.x2x, F.x2y, F.x2z));
}
__device__ __forceinline__ void atomic_add3(float *g, int v, F3 a) {
    atomicAdd(g + 3 * v, a.x);
    atomicAdd(g + 3 * v + 1, a.y);
    atomicAdd(g + 3 * v + 2, a.z);
}

// end-frame adjoint of the query: gm (2-D), transported direction d' (2-D), flip sign
struct EndAdj {
    float a, b, sm;   // gbar_i = a d_i + sm * s_i * b perp(d_i)
    float gmx, gmy;
    int gfe;          // global end face
    Frame3 Fm;
    F3 g;
};

__device__ __forceinline__ EndAdj end_adjoint(const BwdArgs &A, int64_t q, int foff) {
    EndAdj E;
    E.gfe = foff + __ldg(A.end_face + q);
    E.Fm = face_frame(A.P, E.gfe);
    E.g = f3(__ldg(A.g_pos + 3 * q), __ldg(A.g_pos + 3 * q + 1), __ldg(A.g_pos + 3 * q + 2));
    F3 dd = f3(__ldg(A.end_dir + 3 * q), __ldg(A.end_dir + 3 * q + 1), __ldg(A.end_dir + 3 * q + 2));
    float dx = dot3(dd, e1_of(E.Fm)), dy = dot3(dd, e2_of(E.Fm));
    float n2 = dx * dx + dy * dy;
    if (n2 > 0.f) { float r = rsqrtf(n2); dx *= r; dy *= r; }
    E.gmx = dot3(E.g, e1_of(E.Fm));
    E.gmy = dot3(E.g, e2_of(E.Fm));
    E.a = E.gmx * dx + E.gmy * dy;
    E.b = -E.gmx * dy + E.gmy * dx;  // gm . perp(d'), perp(d) = (-dy, dx)
    uint32_t est = A.end_status ? __ldg(A.end_status + q) : 0u;
    E.sm = (est & SG_ST_FLIPPED) ? -1.f : 1.f;
    return E;
}

// ------------------------------------------------------------------ EP
__global__ void __launch_bounds__(256) k_ep_backward(BwdArgs A) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.nq) return;
    Walker w;
    Carry<0> cw;
    bool live = walker_init<0>(A.P, A.in, q, w, cw);
    F3 gv = f3(0.f, 0.f, 0.f);
    uint32_t st = w.st & ~SG_PARITY_BIT;
    if (live && !(w.st & SG_ST_INVALID)) {
        EndAdj E = end_adjoint(A, q, w.foff);
        Frame3 F0 = face_frame(A.P, w.f);
        float gx = E.a * w.dx - E.sm * E.b * w.dy;  // gbar0 = a d0 + sm b perp(d0)
        float gy = E.a * w.dy + E.sm * E.b * w.dx;
        gv = lift(F0, gx, gy);
    }
    if (A.grad_v) { A.grad_v[3 * q] = gv.x; A.grad_v[3 * q + 1] = gv.y; A.grad_v[3 * q + 2] = gv.z; }
    if (A.grad_p) { A.grad_p[3 * q] = 0.f; A.grad_p[3 * q + 1] = 0.f; A.grad_p[3 * q + 2] = 0.f; }
    if (A.grad_bary) { A.grad_bary[3 * q] = 0.f; A.grad_bary[3 * q + 1] = 0.f; A.grad_bary[3 * q + 2] = 0.f; }
    if (A.out_status) A.out_status[q] = st;
}

// ------------------------------------------------------------------ re-walk hooks
// Corner positions of a face record in its frame
__device__ __forceinline__ void corner(const FaceRec &R, int k, float &x, float &y) { x = corner_x(R, k); y = corner_y(R, k); }

// Straddle test of the GFD perturbations against the corners the base walk meets.
struct StraddleHook {
    float Ltot, sphi, cphi;      // e_perp wedge: opening angle atan(eps_v / L)
    float ua, ub, va, vb;        // e_u / e_v offsets along and across d0 (start frame)
    float tol;
    unsigned split = 0;
    __device__ __forceinline__ void test(const Walker &w, float sig_loc, int k) {
        float cx = corner_x(w.R, k), cy = corner_y(w.R, k);
        float tau = (Ltot - (w.Lh + w.Ll)) + (cx - w.px) * w.dx + (cy - w.py) * w.dy;
        float sig = (w.st & SG_PARITY_BIT) ? -sig_loc : sig_loc;
        if (tau < -tol || tau > Ltot + tol) return;
        if (sig > -tol && sig * cphi - tau * sphi < tol) split |= 1u;
        if (ub > 0.f ? (sig > -tol && sig < ub + tol) : (sig < tol && sig > ub - tol)) {
            float a = ub != 0.f ? sig / ub : 0.f;
            float s = tau - a * ua;
            if (s > -tol && s < Ltot + tol) split |= 2u;
        }
        if (vb > 0.f ? (sig > -tol && sig < vb + tol) : (sig < tol && sig > vb - tol)) {
            float a = vb != 0.f ? sig / vb : 0.f;
            float s = tau - a * va;
            if (s > -tol && s < Ltot + tol) split |= 4u;
        }
    }
    __device__ __forceinline__ void on_face(const Walker &w, float s0, float s1, float s2, int mode, int) {
        if (mode < 3) {
            int a = prv(mode);
            test(w, sel3(a, s0, s1, s2), a);
        } else if (mode < 6) {
            int c = mode - 3;
            test(w, sel3(nxt(c), s0, s1, s2), nxt(c));
            test(w, sel3(prv(c), s0, s1, s2), prv(c));
        } else {
            test(w, s0, 0); test(w, s1, 1); test(w, s2, 2);
        }
    }
};

// Adjoint of the crossing maps, accumulated into grad_V (see the file header).
struct GradHook {
    bool on;
    float *gV;
    float a, bs;        // gbar_i = a d_i + bs * s_i * perp(d_i)
    int4 fvc;           // vertex ids of the current face
    Frame3 Fc;          // 3-D frame of the current face
    const WalkParams *P;
    __device__ __forceinline__ void on_cross(const Walker &w, int j, float qx, float qy, float Lr, int g,
                                             const FaceRec &G, int kp, int fl, float ndx, float ndy) {
        if (!on) return;
        const FaceRec &R = w.R;
        // old frame: exit edge A = P_j, B = P_{j+1}
        float Ax, Ay, Bx, By;
        corner(R, j, Ax, Ay);
        corner(R, nxt(j), Bx, By);
        float il = inv_len(R, j);
        float ex = (Bx - Ax) * il, ey = (By - Ay) * il, nx = ey, ny = -ex;
        float yx = fmaf(Lr, w.dx, qx), yy = fmaf(Lr, w.dy, qy);  // end point in the old frame
        float ax_ = (yx - Ax) * ex + (yy - Ay) * ey;
        float cc = (yx - Ax) * nx + (yy - Ay) * ny;
        // new frame: A' = P'_kp, B' = P'_{kp+1}
        float Apx, Apy, Bpx, Bpy;
        corner(G, kp, Apx, Apy);
        corner(G, nxt(kp), Bpx, Bpy);
        float ilp = inv_len(G, kp);
        float fx = (Bpx - Apx) * ilp, fy = (Bpy - Apy) * ilp, mx = fy, my = -fx;
        // upstream gradient in the new frame
        uint32_t par = (w.st & SG_PARITY_BIT) ^ (fl ? SG_PARITY_BIT : 0u);
        float sb = par ? -bs : bs;
        float gx = a * ndx - sb * ndy, gy = a * ndy + sb * ndx;
        float sf = fl ? 1.f : -1.f;
        float ge = gx * fx + gy * fy, gn = gx * mx + gy * my;
        float K1 = sf * ge * cc + gn * ax_;
        float K2 = sf * ax_ * gn + cc * ge;
        // dG/dB, dG/dA in the old frame
        float dBx = nx * K1 * il, dBy = ny * K1 * il;
        float dAx = -sf * ge * ex + gn * nx - nx * K1 * il;
        float dAy = -sf * ge * ey + gn * ny - ny * K1 * il;
        // dG/dB', dG/dA' in the new frame
        float dBpx = mx * K2 * ilp + (fl ? 0.f : gx), dBpy = my * K2 * ilp + (fl ? 0.f : gy);
        float dApx = -mx * K2 * ilp + (fl ? gx : 0.f), dApy = -my * K2 * ilp + (fl ? gy : 0.f);
        int4 fvg = __ldg(P->fv + g);
        Frame3 Fg = face_frame(*P, g);
        int vA = sel3(j, fvc.x, fvc.y, fvc.z), vB = sel3(nxt(j), fvc.x, fvc.y, fvc.z);
        int vAp = sel3(kp, fvg.x, fvg.y, fvg.z), vBp = sel3(nxt(kp), fvg.x, fvg.y, fvg.z);
        F3 gA = lift(Fc, dAx, dAy), gB = lift(Fc, dBx, dBy);
        F3 gAp = lift(Fg, dApx, dApy), gBp = lift(Fg, dBpx, dBpy);
        // the shared edge: vA and vB are vAp/vBp in some order
        if (vA == vAp) { gA = gA + gAp; gB = gB + gBp; }
        else { gA = gA + gBp; gB = gB + gAp; }
        atomic_add3(gV, vA, gA);
        atomic_add3(gV, vB, gB);
        fvc = fvg;
        Fc = Fg;
    }
};

template <bool GFD, bool GRADV>
struct BothHook {
    StraddleHook S;
    GradHook G;
    __device__ __forceinline__ void on_face(const Walker &w, float s0, float s1, float s2, int mode, int hit) {
        if (GFD) S.on_face(w, s0, s1, s2, mode, hit);
    }
    __device__ __forceinline__ void on_cross(const Walker &w, int j, float qx, float qy, float Lr, int g,
                                             const FaceRec &R, int kp, int fl, float ndx, float ndy) {
        if (GRADV) G.on_cross(w, j, qx, qy, Lr, g, R, kp, fl, ndx, ndy);
    }
    __device__ __forceinline__ void on_vertex(const Walker &, int) {}
};

// records the crossing point / vertex so a short walk can sum its 3-D segments
struct ChordHook {
    bool moved = false;
    float qx, qy;
    __device__ __forceinline__ void on_face(const Walker &, float, float, float, int, int) {}
    __device__ __forceinline__ void on_cross(const Walker &, int, float x, float y, float, int, const FaceRec &, int,
                                             int, float, float) { moved = true; qx = x; qy = y; }
    __device__ __forceinline__ void on_vertex(const Walker &w, int hit) {
        moved = true; qx = corner_x(w.R, hit); qy = corner_y(w.R, hit);
    }
};

// 3-D chord of a walk of length `len` from the walker's state along unit 2-D direction u,
// summed segment by segment (no cancellation against |p'|)
__device__ F3 short_chord(const WalkParams &P, Walker w, float ux, float uy, float len, uint32_t &st) {
    w.dx = ux; w.dy = uy; w.Lh = len; w.Ll = 0.f; w.mode = 6; w.steps = 0;
    F3 c = f3(0.f, 0.f, 0.f);
    for (int it = 0; it < 64; ++it) {
        int f0 = w.f;
        float px0 = w.px, py0 = w.py;
        ChordHook h;
        bool done = walker_step<true>(w, P, h);
        Frame3 F = face_frame(P, f0);
        if (h.moved) c = c + lift(F, h.qx - px0, h.qy - py0);
        else c = c + lift(F, w.px - px0, w.py - py0);
        if (done) break;
    }
    st |= w.st;
    return c;
}

// 3-D vector from the base end point to a walker's position, evaluated without cancellation
// against |p|: (x0_a - x0_b) + F_a p_a - F_b p_b with face-local 2-D coordinates
__device__ F3 pos_diff(const WalkParams &P, const Walker &a, const Walker &b) {
    Frame3 Fa = face_frame(P, a.f), Fb = face_frame(P, b.f);
    return (vtx(Fa, 0) - vtx(Fb, 0)) + lift(Fa, a.px, a.py) - lift(Fb, b.px, b.py);
}

__device__ void walk_to_end(const WalkParams &P, Walker &w) {
    while (!walker_step<true>(w, P)) {
    }
}

template <bool GFD, bool GRADV>
__global__ void __launch_bounds__(128) k_rewalk(BwdArgs A) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.nq) return;
    const WalkParams &P = A.P;
    Walker w;
    Carry<0> cw;
    bool live = walker_init<0>(P, A.in, q, w, cw);
    uint32_t st = 0;
    if (!live || (w.st & SG_ST_INVALID)) {
        if (GFD) {
            if (A.grad_v) { A.grad_v[3 * q] = 0.f; A.grad_v[3 * q + 1] = 0.f; A.grad_v[3 * q + 2] = 0.f; }
            if (A.grad_p) { A.grad_p[3 * q] = 0.f; A.grad_p[3 * q + 1] = 0.f; A.grad_p[3 * q + 2] = 0.f; }
            if (A.grad_bary) { A.grad_bary[3 * q] = 0.f; A.grad_bary[3 * q + 1] = 0.f; A.grad_bary[3 * q + 2] = 0.f; }
        }
        if (A.out_status) A.out_status[q] = (w.st & ~SG_PARITY_BIT) | SG_ST_NO_GRADV;
        return;
    }
    const Walker w0 = w;  // start state (for literal perturbed walks)
    const float L = w.Lh;
    EndAdj E = end_adjoint(A, q, w.foff);
    Frame3 F0 = face_frame(P, w.f);
    const float d0x = w.dx, d0y = w.dy;
    const float g0x = E.a * d0x - E.sm * E.b * d0y, g0y = E.a * d0y + E.sm * E.b * d0x;  // gbar0
    uint32_t fst = A.end_status ? __ldg(A.end_status + q) : 0u;
    bool gradv = GRADV && !(fst & (SG_ST_VERTEX_HIT | SG_ST_BOUNDARY | SG_ST_MAX_STEPS | SG_ST_INVALID));
    if (GRADV && !gradv) st |= SG_ST_NO_GRADV;
    BothHook<GFD, GRADV> H;
    if (GFD) {
        float ph = atan2f(A.eps_v, L);
        sincosf(ph, &H.S.sphi, &H.S.cphi);
        H.S.Ltot = L;
        H.S.tol = P.tau_near * w.lref;
        // e_u = (1, 0), e_v = P2 / |P2| in the start frame
        float evx = w.R.x2x * w.R.il2, evy = w.R.x2y * w.R.il2;
        H.S.ua = A.eps_p * d0x;  H.S.ub = -A.eps_p * d0y;
        H.S.va = A.eps_p * (evx * d0x + evy * d0y);
        H.S.vb = A.eps_p * (-evx * d0y + evy * d0x);
    }
    if (GRADV) {
        H.G.on = gradv;
        H.G.gV = A.grad_V;
        H.G.a = gradv ? E.a : 0.f;
        H.G.bs = gradv ? E.sm * E.b : 0.f;
        H.G.fvc = __ldg(P.fv + w.f);
        H.G.Fc = F0;
        H.G.P = &P;
        if (gradv) {
            // start face: p0 = sum b_k P_k  ->  grad x_k += b_k F0 gbar0; tilt term if v has a
            // normal component
            float b2 = w.py / w.R.x2y, b1 = (w.px - b2 * w.R.x2x) / w.R.l01, b0 = 1.f - b1 - b2;
            F3 G0 = lift(F0, g0x, g0y);
            F3 vv = f3(__ldg(A.in.v + 3 * q), __ldg(A.in.v + 3 * q + 1), __ldg(A.in.v + 3 * q + 2));
            F3 n0 = nrm_of(F0);
            float vn = dot3(vv, n0);
            F3 u = vtx(F0, 1) - vtx(F0, 0), ww = vtx(F0, 2) - vtx(F0, 0);
            float mlen = sqrtf(dot3(cross3(u, ww), cross3(u, ww)));
            F3 h = (-vn / mlen) * G0;
            F3 t1 = cross3(ww, h), t2 = cross3(h, u);
            atomic_add3(A.grad_V, H.G.fvc.x, b0 * G0 - (t1 + t2));
            atomic_add3(A.grad_V, H.G.fvc.y, b1 * G0 + t1);
            atomic_add3(A.grad_V, H.G.fvc.z, b2 * G0 + t2);
        }
    }
    while (!walker_step<true>(w, P, H)) {
    }
    st |= w.st & ~SG_PARITY_BIT;
    if (GRADV && gradv) {
        // end face: grad x_j += b'_j (g . n) n
        const FaceRec &R = w.R;
        float b2 = w.py / R.x2y, b1 = (w.px - b2 * R.x2x) / R.l01, b0 = 1.f - b1 - b2;
        F3 n = nrm_of(H.G.Fc);
        F3 gn = dot3(E.g, n) * n;
        atomic_add3(A.grad_V, H.G.fvc.x, b0 * gn);
        atomic_add3(A.grad_V, H.G.fvc.y, b1 * gn);
        atomic_add3(A.grad_V, H.G.fvc.z, b2 * gn);
    }
    if (!GFD) {
        if (A.out_status) A.out_status[q] = st;
        return;
    }
    // ---------------- GFD columns
    unsigned split = H.S.split;
    if (w.st & (SG_ST_BOUNDARY | SG_ST_MAX_STEPS)) split = 7u;
    const float ev = A.eps_v, ep = A.eps_p;
    const float sgn = (w.st & SG_PARITY_BIT) ? -1.f : 1.f;  // orientation of the end frame
    F3 nm = nrm_of(face_frame(P, w.f));
    // R delta for a start-frame 2-D vector x: (x.d0) d' + s (x.perp d0) perp d'
    auto Rmap = [&](float x, float y, float &ox, float &oy) {
        float al = x * d0x + y * d0y, be = -x * d0y + y * d0x;
        ox = al * w.dx - sgn * be * w.dy;
        oy = al * w.dy + sgn * be * w.dx;
    };
    // parallel column: continue the walk eps beyond p'
    F3 cpar = short_chord(P, w, w.dx, w.dy, ev, st);
    F3 cprp, cu, cv;
    // perpendicular column
    if (split & 1u) {
        Walker t = w0;
        float vx = L * d0x - ev * d0y, vy = L * d0y + ev * d0x;
        float Lp = sqrtf(vx * vx + vy * vy);
        t.dx = vx / Lp; t.dy = vy / Lp; t.Lh = Lp; t.Ll = 0.f;
        walk_to_end(P, t);
        st |= t.st & ~SG_PARITY_BIT;
        cprp = pos_diff(P, t, w);
    } else {
        float ox, oy;
        Rmap(-d0y, d0x, ox, oy);
        cprp = short_chord(P, w, ox, oy, ev, st);
    }
    // position columns
    for (int c = 0; c < 2; ++c) {
        float ux = c == 0 ? 1.f : w0.R.x2x * w0.R.il2, uy = c == 0 ? 0.f : w0.R.x2y * w0.R.il2;
        F3 col;
        if (split & (2u << c)) {
            // p_u = Exp(p, eps e_u) carrying v, then Exp(p_u, v_u)
            Walker t = w0;
            t.dx = ux; t.dy = uy; t.Lh = ep; t.Ll = 0.f; t.mode = 6;
            walk_to_end(P, t);
            float vc = d0x * ux + d0y * uy, vs = ux * d0y - uy * d0x;  // v/L relative to e_u
            float s_t = (t.st & SG_PARITY_BIT) ? -1.f : 1.f;
            float nx = vc * t.dx - s_t * vs * t.dy, ny = vc * t.dy + s_t * vs * t.dx;
            t.dx = nx; t.dy = ny; t.Lh = L; t.Ll = 0.f; t.mode = 6; t.steps = 0;
            walk_to_end(P, t);
            st |= t.st & ~SG_PARITY_BIT;
            col = pos_diff(P, t, w);
        } else {
            float ox, oy;
            Rmap(ux, uy, ox, oy);
            col = short_chord(P, w, ox, oy, ep, st);
        }
        if (c == 0) cu = col; else cv = col;
    }
    if (split) st |= SG_ST_GFD_SPLIT;
    // project on the end plane and contract with g
    auto colg = [&](F3 c, float eps) { return dot3(c - dot3(c, nm) * nm, E.g) / eps; };
    float gp = colg(cpar, ev), gq = colg(cprp, ev), gu = colg(cu, ep), gw = colg(cv, ep);
    F3 epar = lift(F0, d0x, d0y), eprp = lift(F0, -d0y, d0x);
    F3 gv = gp * epar + gq * eprp;
    F3 eu = lift(F0, 1.f, 0.f), evv = lift(F0, w0.R.x2x * w0.R.il2, w0.R.x2y * w0.R.il2);
    float a11 = dot3(eu, eu), a12 = dot3(eu, evv), a22 = dot3(evv, evv);
    float det = a11 * a22 - a12 * a12;
    float c0 = (a22 * gu - a12 * gw) / det, c1 = (-a12 * gu + a11 * gw) / det;
    F3 gpv = c0 * eu + c1 * evv;
    if (A.grad_v) { A.grad_v[3 * q] = gv.x; A.grad_v[3 * q + 1] = gv.y; A.grad_v[3 * q + 2] = gv.z; }
    if (A.grad_p) { A.grad_p[3 * q] = gpv.x; A.grad_p[3 * q + 1] = gpv.y; A.grad_p[3 * q + 2] = gpv.z; }
    if (A.grad_bary) {
        for (int k = 0; k < 3; ++k) A.grad_bary[3 * q + k] = dot3(gpv, vtx(F0, k));
    }
    if (A.out_status) A.out_status[q] = st;
}

extern "C" sg_status sg_exp_map_backward(const sg_mesh *m, int32_t estimator, float eps_v, float eps_p, int64_t nq,
                                         const int32_t *mesh_id, const int32_t *face, const float *bary,
                                         const float *v, const int32_t *end_face, const float *end_bary,
                                         const float *end_dir, const uint32_t *end_status, const float *g_pos,
                                         float *grad_v, float *grad_p, float *grad_bary, float *grad_V,
                                         uint32_t *out_status, const sg_opts *o, void *stream) {
    if (!m || nq < 0) return SG_ERR_INVALID_ARG;
    if (estimator != SG_EST_EP && estimator != SG_EST_GFD) return SG_ERR_INVALID_ARG;
    if (nq == 0) return SG_OK;
    if (nq > (int64_t)INT32_MAX - 1024) return SG_ERR_INVALID_ARG;
    if (!face || !bary || !v || !end_face || !end_dir || !g_pos) return SG_ERR_INVALID_ARG;
    if (grad_V && !end_status) return SG_ERR_INVALID_ARG;
    if (estimator == SG_EST_GFD && !(eps_v > 0.f && eps_p > 0.f)) return SG_ERR_INVALID_ARG;
    (void)end_bary;
    sg_opts r;
    sg_opts_default(&r);
    if (o) r = *o;
    if (r.max_steps <= 0) r.max_steps = 1 << 20;
    if (r.tau_near <= 0.f) r.tau_near = 1e-4f;
    if (r.tau_snap <= 0.f) r.tau_snap = 1e-6f;
    cudaStream_t s = (cudaStream_t)stream;
    BwdArgs A{};
    A.P.rec = m->d_rec; A.P.fv = m->d_fv; A.P.V = m->d_V; A.P.face_off = m->d_face_off; A.P.lref = m->d_lref;
    A.P.max_steps = r.max_steps; A.P.tau_near = r.tau_near; A.P.tau_snap = r.tau_snap; A.P.want_hash = 0;
    A.in.n_mesh = m->n_mesh; A.in.mesh_id = mesh_id; A.in.face = face; A.in.bary = bary; A.in.v = v;
    A.in.length = nullptr; A.in.w = nullptr;
    A.nq = nq;
    A.end_face = end_face; A.end_bary = end_bary; A.end_dir = end_dir; A.end_status = end_status; A.g_pos = g_pos;
    A.grad_v = grad_v; A.grad_p = grad_p; A.grad_bary = grad_bary; A.grad_V = grad_V; A.out_status = out_status;
    A.eps_v = eps_v; A.eps_p = eps_p;
    if (estimator == SG_EST_EP) {
        k_ep_backward<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(A);
        if (cudaGetLastError() != cudaSuccess) return SG_ERR_CUDA;
        if (grad_V) {
            BwdArgs B = A;
            B.grad_v = nullptr; B.grad_p = nullptr; B.grad_bary = nullptr; B.out_status = nullptr;
            k_rewalk<false, true><<<(unsigned)((nq + 127) / 128), 128, 0, s>>>(B);
        }
    } else {
        if (grad_V)
            k_rewalk<true, true><<<(unsigned)((nq + 127) / 128), 128, 0, s>>>(A);
        else
            k_rewalk<true, false><<<(unsigned)((nq + 127) / 128), 128, 0, s>>>(A);
    }
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}
