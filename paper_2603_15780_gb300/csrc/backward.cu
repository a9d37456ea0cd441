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
// Exp = p + v, so a perturbed ray that sweeps no vertex ends at p' + R delta.  The work is
// split into uniform launches:
//   k_bwd_rewalk   re-walks the base ray and tests every corner it meets against the thin
//                  regions swept by the perturbations (a wedge for e_perp, parallelograms for
//                  e_u, e_v); a perturbation that sweeps a vertex (or any perturbation of a
//                  walk that stopped on the boundary) is appended to a task list.  The same
//                  re-walk accumulates grad_V (below).
//   k_bwd_literal  evaluates the swept columns by the paper's literal walk
//                  (Exp(p, v + eps e_perp), or Exp(p_u, v_u) after Exp(p, eps e_u) carrying v),
//                  restarted on the entry edge of the face where the re-walk met the first
//                  swept corner, differences taken in face-local coordinates;
//   k_bwd_assemble evaluates every other column as the 3-D chord of a short walk from p'
//                  along R delta, summed segment by segment (exact for unswept
//                  perturbations, no cancellation against |p'|), and contracts the columns
//                  into grad_v, grad_p, grad_bary.  A chord that stays in the end face needs
//                  no walk; the few queries with one that leaves it are finished by
//                  k_bwd_assemble_walk.
//
// grad_V (vertex positions; not in the paper): the a.e. derivative of p' with the face
// sequence fixed.  The end point is a chain of rigid 2-D maps T (one per crossing) applied
// to p0 + v; each T depends on the corners of the shared edge in the two faces.  The
// adjoint of T at a crossing needs the end point expressed in the old frame
// (y = q + L_rem d) and the upstream gradient in the new frame, which is the end-frame
// gradient parallel-transported back (gbar_i = a d_i + s_i b perp(d_i)), so one forward
// re-walk accumulates everything (no stored path).  2-D corner gradients map to 3-D by the
// face frame F (in-plane); start and end faces add b_k F gbar0 and b'_k (g.n) n, plus a
// tilt term when v has a normal component.  Each crossing yields two scalars for its interior
// edge.  Two consecutive crossings of a walk share a face, so they are added together with one
// 16-byte atomic into that face's accumulator window for the pair of edges (GradHook below);
// k_gradv_edges sums each edge's windows in its two faces and expands them into vertex
// gradients once per edge, the start and end terms go into a float4 accumulator per vertex,
// and k_gradv_flush adds it to the caller's grad_V.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "sgeo_internal.h"
#include "walk.cuh"
#include "walk64.cuh"

#define SG_BWD_MAX_W 4
// lanes of a warp that must be idle before the re-walk refills them together (swept under the
// length order with the paired grad_V reductions: 16 0.706, 20 0.686, 24 0.648, 28 0.631,
// 32 0.633 ms)
#ifndef SG_REWALK_REFILL
#define SG_REWALK_REFILL 28
#endif
// minimum resident blocks per SM the assemble and literal kernels are compiled for (the assemble
// pass holds no walk since its chord walks moved to a second pass)
#ifndef SG_ASSEMBLE_MINB
#define SG_ASSEMBLE_MINB 8
#endif
// literal walks: 7 blocks/SM (72 registers) took the GFD phase from 1.008 to 0.998 ms against
// the registers the compiler picks unbounded (78-80, 6 blocks)
#ifndef SG_LITERAL_MINB
#define SG_LITERAL_MINB 7
#endif
// walk steps between the re-walk's and the literal walks' refill checks (re-walk: 1 step 0.600 ms,
// 2 steps 0.619, 3 steps 0.651; refill at 28 idle lanes with one step: 20 0.665, 24 0.619,
// 30 0.601, 32 0.610 ms; the forward walk keeps 2: 0.389 ms against 0.522 with one)
#ifndef SG_REWALK_STEPS
#define SG_REWALK_STEPS 1
#endif
#ifndef SG_LITERAL_STEPS
#define SG_LITERAL_STEPS 2
#endif
// minimum resident blocks per SM of the re-walk (69 registers at 7 without spills, with the
// straddle test's rare constants, the query id and the face offset in shared memory; 6 blocks
// time the same)
#ifndef SG_REWALK_MINB
#define SG_REWALK_MINB 7
#endif
// the same for the literal GFD walks
#ifndef SG_LITERAL_REFILL
#define SG_LITERAL_REFILL 24
#endif

struct BwdArgs {
    WalkParams P;
    QueryIn in;
    int64_t nq;
    const int32_t *__restrict__ end_face;
    const float *__restrict__ end_bary;
    const float *__restrict__ end_dir;
    const uint32_t *__restrict__ end_status;
    const float *__restrict__ g_pos;
    const float *__restrict__ g_bary;  // [nq][3] upstream gradient of end_bary, or NULL
    const float *__restrict__ g_dir;   // [nq][3] upstream gradient of end_dir, or NULL
    const float *__restrict__ g_w;     // [nq][n_w][3] upstream gradients of the carried vectors, or NULL
    int32_t n_w;
    float *grad_v, *grad_p, *grad_bary, *grad_V, *grad_w;
    uint32_t *out_status;
    float eps_v, eps_p;
    float4 *gacc;       // [nV] vertex-gradient accumulator (scratch)
    float4 *wacc;       // [3 nF] per face f, window k = the (start, end) coefficients of its edges k
                        // and k+1, each in f's orientation of the edge (corner k -> k+1) (scratch)
    float *cols;        // [nq][4] column contractions: par, perp, u, v; until the chords are
                        // evaluated the par slot holds the re-walk's swept-column mask (scratch)
    int32_t *tasks;     // [3 nq] (q << 2 | k) columns recomputed by literal walks (scratch)
    int32_t *ntask;     // counters (scratch): [0] tasks, [1] re-walk and [2] literal-walk tickets,
                        // [3] queries the assemble pass deferred (their ids reuse `tasks`),
                        // [4] mixed-walk tasks and [5] their tickets
    int4 *rst;          // [nq][2] where the literal walks of a split query restart (scratch):
                        // {half-edge | parity << 30 (-1: from the start), s, dx, dy}, {Lh, Ll, -, -}
    const int32_t *perm;  // re-walk queue position -> query (length order), or NULL
    // the literal walks of the queries whose forward walk was the mixed walk (SG_ST_MIXED): their
    // task list [3 nq] (count ntask[4], tickets ntask[5]) and the mesh's wide-precision geometry
    int32_t *tasks40;
    P64 P4;
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

// 3-D axes of a face's 2-D frame (precomputed per face)
struct Fr2 {
    float e1x, e1y, e1z, e2x, e2y, e2z;
};
__device__ __forceinline__ Fr2 load_frm(const WalkParams &P, int f) {
    float4 a = __ldg(P.frm + 2 * f), b = __ldg(P.frm + 2 * f + 1);
    return Fr2{a.x, a.y, a.z, a.w, b.x, b.y};
}
__device__ __forceinline__ F3 lift(const Fr2 &F, float a, float b) {
    return f3(a * F.e1x + b * F.e2x, a * F.e1y + b * F.e2y, a * F.e1z + b * F.e2z);
}
__device__ __forceinline__ F3 nrm_of(const Fr2 &F) {
    return cross3(f3(F.e1x, F.e1y, F.e1z), f3(F.e2x, F.e2y, F.e2z));
}
__device__ __forceinline__ F3 vpos(const WalkParams &P, int v) {
    float4 a = __ldg(P.V + v);
    return f3(a.x, a.y, a.z);
}
__device__ __forceinline__ void atomic_add3(float4 *g, int v, F3 a) {
    atomicAdd(g + v, make_float4(a.x, a.y, a.z, 0.f));
}
__device__ __forceinline__ F3 ld3(const float *p, int64_t q) {
    return f3(__ldg(p + 3 * q), __ldg(p + 3 * q + 1), __ldg(p + 3 * q + 2));
}
__device__ __forceinline__ void st3(float *p, int64_t q, F3 a) {
    p[3 * q] = a.x; p[3 * q + 1] = a.y; p[3 * q + 2] = a.z;
}

// end-frame adjoint of a query: gbar_i = a d_i + sm * s_i * b perp(d_i)
struct EndAdj {
    float a, b, sm;
    float dmx, dmy;     // transported direction in the end frame
    F3 g, nm;           // upstream gradient, end-face normal
    int gfe;            // global end face
};

// Tangent gradient equivalent to an upstream gradient gb on the barycentrics of a point of face
// f (Sec. 4: points are (face, b) pairs): g_t = sum_k gb_k grad(b_k), with grad b_1 =
// (1/l01, -x2x/(l01 x2y)) and grad b_2 = (0, 1/x2y) in the face frame (grad b_0 = -grad b_1 -
// grad b_2), so g_t . dp = sum_k gb_k db_k for every displacement dp in the face plane.
__device__ __forceinline__ F3 bary_grad_to_tangent(const WalkParams &P, int f, F3 gb) {
    const FaceRec R = load_rec(P.rec, f);
    const float g1 = gb.y - gb.x, g2 = gb.z - gb.x;
    const float tx = g1 / R.l01;
    const float ty = (g2 - g1 * R.x2x / R.l01) / R.x2y;
    return lift(load_frm(P, f), tx, ty);
}

__device__ __forceinline__ EndAdj end_adjoint(const BwdArgs &A, int64_t q, int foff) {
    EndAdj E;
    E.gfe = foff + __ldg(A.end_face + q);
    Fr2 Fm = load_frm(A.P, E.gfe);
    E.g = ld3(A.g_pos, q);
    F3 dd = ld3(A.end_dir, q);
    float dx = dd.x * Fm.e1x + dd.y * Fm.e1y + dd.z * Fm.e1z;
    float dy = dd.x * Fm.e2x + dd.y * Fm.e2y + dd.z * Fm.e2z;
    float n2 = dx * dx + dy * dy;
    if (n2 > 0.f) { float r = rsqrtf(n2); dx *= r; dy *= r; }
    E.dmx = dx; E.dmy = dy;
    float gmx = E.g.x * Fm.e1x + E.g.y * Fm.e1y + E.g.z * Fm.e1z;
    float gmy = E.g.x * Fm.e2x + E.g.y * Fm.e2y + E.g.z * Fm.e2z;
    E.a = gmx * dx + gmy * dy;
    E.b = -gmx * dy + gmy * dx;  // gm . perp(d'), perp(d) = (-dy, dx)
    uint32_t est = A.end_status ? __ldg(A.end_status + q) : 0u;
    E.sm = (est & SG_ST_FLIPPED) ? -1.f : 1.f;
    E.nm = nrm_of(Fm);
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
        Fr2 F0 = load_frm(A.P, w.f);
        float gx = E.a * w.dx - E.sm * E.b * w.dy;  // gbar0 = a d0 + sm b perp(d0)
        float gy = E.a * w.dy + E.sm * E.b * w.dx;
        gv = lift(F0, gx, gy);
    }
    if (A.grad_v) st3(A.grad_v, q, gv);
    if (A.grad_p) st3(A.grad_p, q, f3(0.f, 0.f, 0.f));
    if (A.grad_bary) st3(A.grad_bary, q, f3(0.f, 0.f, 0.f));
    if (A.out_status) A.out_status[q] = st;
}

// ------------------------------------------------------------------ re-walk hooks
// Straddle test of the GFD perturbations against the corners the base walk meets.
// The perturbed rays run in the base ray's face strip until the first corner they sweep, so the
// literal walks of a split query can restart on the entry edge of the face where the first such
// corner was met; the hook stores the base walker's state there (bit 3 of `split`).
#define SG_SPLIT_RESTART 8u
// The constants of the full test are read only after the |sig| <= sbound rejection, about once
// per hundred corners, so they live in shared memory (one column per thread of the re-walk's
// 128-thread blocks), not in registers:
//   Ltot, tphi   e_perp wedge: the walk's length, tan of its opening angle eps_v / L
//   ub, vb       e_u / e_v offsets across d0 (start frame)
//   uq, vq       offsets along d0 over those across (0 when ub, vb = 0)
//   tol          tau_near l_ref (1 + tphi^2), at least tau_near l_ref / cos(phi)
#define SG_STR_LTOT 0
#define SG_STR_TPHI 1
#define SG_STR_TOL 2
#define SG_STR_UB 3
#define SG_STR_VB 4
#define SG_STR_UQ 5
#define SG_STR_VQ 6
__shared__ float s_straddle[7][128];
// the re-walk's query and its mesh's face offset, read only when a swept corner is recorded and
// at the end of the walk (shared memory, one slot per thread, instead of two registers).  These
// arrays are sized for the re-walk's 128-thread blocks: its __launch_bounds__(128, ...) makes a
// launch with larger blocks fail instead of indexing past them.
__shared__ int32_t s_rewalk_q[128], s_rewalk_foff[128];
struct StraddleHook {
    const BwdArgs *A;
    float sbound;                // every region below lies within |sig| <= sbound
    unsigned split;
    // RECORD: the walker sits on a half-edge (the apex test of the hot step), where a first
    // swept corner stores the restart state
    template <bool RECORD>
    __device__ __forceinline__ void test_at(const Walker &w, float sig_loc, float cx, float cy, float px, float py) {
        // nearly every vertex passed lies far from the eps-wide regions: reject on |sig| first
        if (fabsf(sig_loc) > sbound) return;
        const int th = threadIdx.x;
        const float Ltot = s_straddle[SG_STR_LTOT][th], tphi = s_straddle[SG_STR_TPHI][th];
        const float tol = s_straddle[SG_STR_TOL][th], ub = s_straddle[SG_STR_UB][th], vb = s_straddle[SG_STR_VB][th];
        const float uq = s_straddle[SG_STR_UQ][th], vq = s_straddle[SG_STR_VQ][th];
        float tau = (Ltot - (w.Lh + w.Ll)) + (cx - px) * w.dx + (cy - py) * w.dy;
        float sig = (w.st & SG_PARITY_BIT) ? -sig_loc : sig_loc;
        if (tau < -tol || tau > Ltot + tol) return;
        unsigned nb = 0u;
        if (sig > -tol && sig - tau * tphi < tol) nb |= 1u;
        if (ub > 0.f ? (sig > -tol && sig < ub + tol) : (sig < tol && sig > ub - tol)) {
            float s = tau - sig * uq;
            if (s > -tol && s < Ltot + tol) nb |= 2u;
        }
        if (vb > 0.f ? (sig > -tol && sig < vb + tol) : (sig < tol && sig > vb - tol)) {
            float s = tau - sig * vq;
            if (s > -tol && s < Ltot + tol) nb |= 4u;
        }
        if (RECORD && nb && !split) {
            // first swept corner, met on a half-edge: the state on its entry edge
            const int hp = w.h | ((w.st & SG_PARITY_BIT) ? (1 << 30) : 0);
            int4 *r = A->rst + 2 * (int64_t)s_rewalk_q[threadIdx.x];
            r[0] = make_int4(hp, __float_as_int(w.px), __float_as_int(w.dx), __float_as_int(w.dy));
            *reinterpret_cast<float2 *>(r + 1) = make_float2(w.Lh, w.Ll);
            nb |= SG_SPLIT_RESTART;
        }
        split |= nb;
    }
    __device__ __forceinline__ void test(const Walker &w, float sig_loc, int k) {
        test_at<false>(w, sig_loc, corner_x(w.R, k), corner_y(w.R, k), w.px, w.py);
    }
    __device__ __forceinline__ void on_face(const Walker &w, float s0, float s1, float s2, int mode) {
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

// Adjoint of the crossing maps.  For a crossing of edge A -> B (the exit edge, unit e, outward
// unit normal n in the old frame) with end point y (old frame) and upstream gradient gbar in
// the old frame (g_e = gbar.e, g_n = gbar.n), the transition's linear part gives the same
// scalar K = g_e ((y-A).n) - g_n ((y-A).e) for both faces' corner gradients, and the jump of
// the lifted adjoint across the edge is -g_n (N_old + N_new).  Lifted to 3-D the two shared
// vertices receive
//   g_B = (K / l) (N_old + N_new),   g_A = -(g_n + K / l) (N_old + N_new),
// N_old / N_new = the in-plane unit normals of the edge pointing out of the old / new face.
// N_old + N_new is a constant of the edge, so the walk only adds the two scalar
// coefficients (kA, kB) to an accumulator of the edge; k_gradv_edges turns them into vertex
// gradients once.  For coplanar faces N_old + N_new = 0.
//
// Accumulation: a crossing leaves face f through its edge j (A = corner j, B = corner j+1)
// and enters g through g's edge kp.  The next crossing leaves g, so the two meet in g: the
// first is held in registers (in g's orientation of edge kp) and the pair goes to g's window
// for edges {kp, j'} as one 16-byte atomic.  Window k of a face holds edges k and k+1, so the
// three windows cover the three pairs.  A crossing with no successor in its face (the walk
// ends, or the next step is a vertex transport) is added alone to the first half of its
// edge's window.  This halves the atomics, which share the L2 with the record reads.
struct GradHook {
    float a, bs;        // gbar_i = a d_i + bs * s_i * perp(d_i)
    // The held crossing: its coefficients in g's orientation of edge kp (corner kp -> kp+1).
    // Its half-edge 3g + kp is the walker's w.h from that crossing until the walk's next
    // crossing, vertex transport or end (none of which happens without a flush or a pairing).
    bool held;
    float pa, pb;
    __device__ __forceinline__ void flush(float4 *wacc, int h) {
        if (held) atomicAdd(reinterpret_cast<float2 *>(wacc + h), make_float2(pa, pb));
        held = false;
    }
    __device__ __forceinline__ void on_cross(const Walker &w, const Cross &c, float4 *wacc) {
        // With e = B - A, q - A = s e and y - A = s e + L_rem d, and g = a d + sb perp(d):
        // g x e = a (d x e) - sb (d . e) = m, g x (y - A) = s m - sb L_rem, so
        // K = -il (g x (y - A)) = il (sb L_rem - s m) and g_n = il m
        const float sb = (w.st & SG_PARITY_BIT) ? -bs : bs;             // old-frame parity
        const float m = fmaf(a, c.dc, -sb * c.da);
        const float sl = sb * c.Lr;
        const float kB = c.il * fmaf(-c.s, m, sl);
        const float kA = -c.il * (m + fmaf(-c.s, m, sl));               // -(g_n + K)
        if (held && c.ke >= 0) {
            // the held crossing entered this face through edge ke (a half-edge step, w.h = 3f +
            // ke): window ke holds (ke, ke+1) when the walk leaves through j = ke+1, window j
            // holds (j, ke) when it leaves through j = ke-1
            if (c.j == nxt(c.ke)) atomicAdd(wacc + w.h, make_float4(pa, pb, kA, kB));
            else atomicAdd(wacc + (w.h - c.ke + c.j), make_float4(kA, kB, pa, pb));
            held = false;
        } else {
            flush(wacc, w.h);
            // held in g's orientation of edge kp: corner kp of g is B, kp+1 is A, unless the
            // adjacency is flipped (the two faces list the edge in the same direction)
            held = true;
            pa = c.fl ? kA : kB;
            pb = c.fl ? kB : kA;
        }
    }
};

template <bool GFD, bool GRADV>
struct RewalkHook {
    const BwdArgs *A;   // the kernel's arguments (parameter space, not a register)
    StraddleHook S;
    GradHook G;
    bool gradv;
    __device__ __forceinline__ void on_face(const Walker &w, float s0, float s1, float s2, int mode, int) {
        if (GFD) S.on_face(w, s0, s1, s2, mode);
    }
    __device__ __forceinline__ void on_apex(const Walker &w, float sC, float cx, float cy, float px, float py) {
        if (GFD) S.template test_at<true>(w, sC, cx, cy, px, py);
    }
    __device__ __forceinline__ void on_cross(const Walker &w, const Cross &c, const FaceRec &) {
        if (GRADV && gradv) G.on_cross(w, c, A->wacc);
    }
    __device__ __forceinline__ void on_vertex(const Walker &w, int) {
        if (GRADV && gradv) G.flush(A->wacc, w.h);
    }
};

// ------------------------------------------------------------------ kernel 1: re-walk
template <bool GFD, bool GRADV>
struct RewalkJob {
    const BwdArgs *A;
    Walker w;
    RewalkHook<GFD, GRADV> H;
    bool valid;

    __device__ __forceinline__ bool init(int64_t t) {
        // the query (nq < 2^29, checked at the entry point); an order entry out of range (a
        // caller's order that is not a permutation) is skipped
        const int32_t q = A->perm ? __ldg(A->perm + t) : (int32_t)t;
        if ((uint32_t)q >= (uint32_t)A->nq) {
            s_rewalk_q[threadIdx.x] = -1;
            valid = false;
            return false;
        }
        s_rewalk_q[threadIdx.x] = q;
        H.A = A;
        const WalkParams &P = A->P;
        Carry<0> cw;
        bool live = walker_init<0>(P, A->in, q, w, cw);
        valid = live && !(w.st & SG_ST_INVALID);
        if (!valid) return false;
        s_rewalk_foff[threadIdx.x] = w.foff;
        uint32_t fst = A->end_status ? __ldg(A->end_status + q) : 0u;
        H.gradv = GRADV && !(fst & (SG_ST_VERTEX_HIT | SG_ST_BOUNDARY | SG_ST_MAX_STEPS | SG_ST_INVALID | SG_ST_HOLE));
        if (GRADV && !H.gradv) w.st |= SG_ST_NO_GRADV;  // the walker never touches this bit
        if (GRADV) H.G.held = false;
        const float L = w.Lh, d0x = w.dx, d0y = w.dy;
        if (GFD) {
            H.S.A = A;
            const float tphi = A->eps_v / L;
            const float tol = P.tau_near * w.lref * (1.f + tphi * tphi);
            // a walk that slid along the boundary (hole avoidance) takes literal walks
            H.S.split = (fst & SG_ST_HOLE) ? 7u : 0u;
            float evx = w.R.x2x * w.R.il2, evy = w.R.x2y * w.R.il2;  // e_u = (1,0), e_v = P2/|P2|
            const float ua = A->eps_p * d0x, va = A->eps_p * (evx * d0x + evy * d0y);
            const float ub = -A->eps_p * d0y;
            const float vb = A->eps_p * (-evx * d0y + evy * d0x);
            const int th = threadIdx.x;
            s_straddle[SG_STR_LTOT][th] = L;
            s_straddle[SG_STR_TPHI][th] = tphi;
            s_straddle[SG_STR_TOL][th] = tol;
            s_straddle[SG_STR_UB][th] = ub;
            s_straddle[SG_STR_VB][th] = vb;
            s_straddle[SG_STR_UQ][th] = ub != 0.f ? ua / ub : 0.f;
            s_straddle[SG_STR_VQ][th] = vb != 0.f ? va / vb : 0.f;
            // the wedge needs sig < tau tphi + tol with tau <= Ltot + tol; the parallelograms
            // |sig| < |ub| + tol, |vb| + tol (with a margin for the bound's own rounding)
            H.S.sbound = 1.0001f * (fmaxf(fmaxf(fabsf(ub), fabsf(vb)), (L + tol) * tphi) + tol);
        }
        if (GRADV && H.gradv) {
            EndAdj E = end_adjoint(*A, q, w.foff);
            H.G.a = E.a;
            H.G.bs = E.sm * E.b;
            // start face: p0 = sum b_k P_k -> grad x_k += b_k F0 gbar0; tilt term if v has a
            // normal component (moving the plane changes the projection of v)
            const int4 fv0 = __ldg(P.fv + w.f);
            const Fr2 F0 = load_frm(P, w.f);
            const float g0x = E.a * d0x - E.sm * E.b * d0y, g0y = E.a * d0y + E.sm * E.b * d0x;
            float b2 = w.py / w.R.x2y, b1 = (w.px - b2 * w.R.x2x) / w.R.l01, b0 = 1.f - b1 - b2;
            F3 G0 = lift(F0, g0x, g0y);
            F3 n0 = nrm_of(F0);
            float vn = dot3(ld3(A->in.v, q), n0);
            F3 x0 = vpos(P, fv0.x), u = vpos(P, fv0.y) - x0, ww = vpos(P, fv0.z) - x0;
            F3 m = cross3(u, ww);
            F3 h = (-vn * rsqrtf(dot3(m, m))) * G0;
            F3 t1 = cross3(ww, h), t2 = cross3(h, u);
            atomic_add3(A->gacc, fv0.x, b0 * G0 - (t1 + t2));
            atomic_add3(A->gacc, fv0.y, b1 * G0 + t1);
            atomic_add3(A->gacc, fv0.z, b2 * G0 + t2);
        }
        return true;
    }
    __device__ __forceinline__ bool step() { return walker_step<true>(w, A->P, H); }
    __device__ __forceinline__ void finish() {
        const int32_t q = s_rewalk_q[threadIdx.x];
        if (q < 0) return;
        if (!valid) {
            if (A->out_status) A->out_status[q] = (w.st & ~SG_PARITY_BIT) | (GRADV ? SG_ST_NO_GRADV : 0u);
            return;
        }
        uint32_t st = w.st & ~SG_PARITY_BIT;
        if (GRADV && H.gradv) {
            H.G.flush(A->wacc, w.h);
            // end face: grad x_j += b'_j (g . n) n
            const FaceRec &R = w.R;
            const int4 fve = __ldg(A->P.fv + w.f);
            float b2 = w.py / R.x2y, b1 = (w.px - b2 * R.x2x) / R.l01, b0 = 1.f - b1 - b2;
            F3 n = nrm_of(load_frm(A->P, w.f));
            F3 gn = dot3(ld3(A->g_pos, q), n) * n;  // g (reloaded rather than kept through the walk)
            atomic_add3(A->gacc, fve.x, b0 * gn);
            atomic_add3(A->gacc, fve.y, b1 * gn);
            atomic_add3(A->gacc, fve.z, b2 * gn);
        }
        // A forward walk beyond the FP32 walk's range ran in the mixed walk; this FP32 re-walk
        // may then pass a vertex on the other side: reported when it ends in another face.
        const bool mixed = A->end_status && (__ldg(A->end_status + q) & SG_ST_MIXED);
        const bool diverged = mixed && w.f - s_rewalk_foff[threadIdx.x] != __ldg(A->end_face + q);
        if (diverged) st |= SG_ST_REWALK_DIVERGED;
        if (GFD) {
            // A walk that stopped at the boundary or at MAX_STEPS, or slid along the boundary
            // (hole avoidance), takes literal walks for all perturbed columns; the par column
            // is the chord from p' in every case (Round 2 of the paper's batching).  So does a
            // re-walk that left the forward's path.  The literal walks of a query the forward
            // walked in the mixed walk are the mixed walk too (k_bwd_literal40, from the start).
            unsigned split = H.S.split & 7u;
            if (w.st & (SG_ST_BOUNDARY | SG_ST_MAX_STEPS) || diverged) split = 7u;
            A->cols[4 * (int64_t)q] = __uint_as_float(split);  // read by k_bwd_assemble
            if (split && !mixed && !(H.S.split & SG_SPLIT_RESTART)) A->rst[2 * (int64_t)q] = make_int4(-1, 0, 0, 0);
            if (split) {
                st |= SG_ST_GFD_SPLIT;
                int32_t *list = mixed ? A->tasks40 : A->tasks;
                int base = atomicAdd(A->ntask + (mixed ? 4 : 0), __popc(split));
                for (int k = 0; k < 3; ++k)
                    if (split & (1u << k)) list[base++] = (int32_t)((q << 2) | (k + 1));
            }
        }
        if (A->out_status) A->out_status[q] = st;
    }
};

template <bool GFD, bool GRADV>
__global__ void __launch_bounds__(128, SG_REWALK_MINB) k_bwd_rewalk(BwdArgs A) {
    RewalkJob<GFD, GRADV> job;
    job.A = &A;
    run_persistent<RewalkJob<GFD, GRADV>, SG_REWALK_REFILL, SG_REWALK_STEPS>(A.ntask + 1, A.nq, job);
}

// ------------------------------------------------------------------ chord / literal walks
// the forward end state (face, 2-D point, transported direction, parity) of query q
__device__ __forceinline__ void end_walker(const BwdArgs &A, int64_t q, const Walker &start, const EndAdj &E,
                                           Walker &w) {
    w = start;
    w.f = E.gfe;
    w.R = load_rec(A.P.rec, w.f);
    float b1 = __ldg(A.end_bary + 3 * q + 1), b2 = __ldg(A.end_bary + 3 * q + 2);
    w.px = fmaf(b1, w.R.l01, b2 * w.R.x2x);
    w.py = b2 * w.R.x2y;
    w.dx = E.dmx; w.dy = E.dmy;
    w.st = (E.sm < 0.f) ? SG_PARITY_BIT : 0u;
    w.mode = 6; w.steps = 0;
}

// 3-D vector from walker b's position to walker a's, without cancellation against |p|:
// (x0_a - x0_b) + F_a p_a - F_b p_b with face-local 2-D coordinates
__device__ F3 pos_diff(const WalkParams &P, const Walker &a, const Walker &b) {
    int4 ta = __ldg(P.fv + a.f), tb = __ldg(P.fv + b.f);
    Fr2 Fa = load_frm(P, a.f), Fb = load_frm(P, b.f);
    return (vpos(P, ta.x) - vpos(P, tb.x)) + lift(Fa, a.px, a.py) - lift(Fb, b.px, b.py);
}

__device__ __forceinline__ float contract(F3 c, const EndAdj &E, float eps) {
    return dot3(c - dot3(c, E.nm) * E.nm, E.g) / eps;
}

// A walk of length `len` from the end state w0 along unit 2-D direction u (face frame); its
// 3-D chord is the cancellation-free difference of its end and start positions, contracted.
template <bool HOLE>
__device__ __noinline__ float chord_walk(const WalkParams &P, const Walker &w0, const EndAdj &E, float ux, float uy,
                                         float len) {
    Walker w = w0;
    w.dx = ux; w.dy = uy; w.Lh = len; w.Ll = 0.f; w.mode = 6; w.steps = 0;
    while (!walker_step<true, HOLE>(w, P)) {
    }
    return contract(pos_diff(P, w, w0), E, len);
}

// Contracted chord (p'' - p') / len of a walk of length `len` from the end state along u.  A
// chord that ends inside the end face, farther than tau_near l_ref from its edges, is the step
// len u itself, and its contraction u . gm = (u.d') a + (u.perp d') b needs no walk.  Other
// chords are walked when WALK, else `ok` is cleared.
template <bool HOLE, bool WALK>
__device__ __forceinline__ float chord_col(const WalkParams &P, const Walker &w0, const EndAdj &E, float ux, float uy,
                                           float len, bool &ok) {
    const FaceRec &R = w0.R;
    const float x = fmaf(len, ux, w0.px), y = fmaf(len, uy, w0.py);
    const float tol = P.tau_near * w0.lref;
    const float e1 = ((R.x2x - R.l01) * y - R.x2y * (x - R.l01)) * R.il1;
    const float e2 = (R.x2y * x - R.x2x * y) * R.il2;
    if (y > tol && e1 > tol && e2 > tol)
        return fmaf(fmaf(ux, E.dmx, uy * E.dmy), E.a, fmaf(uy, E.dmx, -ux * E.dmy) * E.b);
    if (WALK) return chord_walk<HOLE>(P, w0, E, ux, uy, len);
    ok = false;
    return 0.f;
}

// R x for a start-frame 2-D vector x: (x.d0) d' + s (x.perp d0) perp d'
__device__ __forceinline__ void rmap(float x, float y, float d0x, float d0y, const EndAdj &E, float &ox, float &oy) {
    float al = x * d0x + y * d0y, be = -x * d0y + y * d0x;
    ox = al * E.dmx - E.sm * be * E.dmy;
    oy = al * E.dmy + E.sm * be * E.dmx;
}

// literal walk of one swept perturbation (task = q << 2 | k): k = 1 walks Exp(p, v + eps e_perp);
// k = 2, 3 walk p_u = Exp(p, eps e_u) carrying v, then Exp(p_u, v_u) (two phases)
template <bool HOLE>
struct LiteralJob {
    const BwdArgs *A;
    Walker w;
    int64_t q;
    int k, phase;
    float L, d0x, d0y, ux, uy;

    // Restart on the entry edge (half-edge h, fraction s, base direction d, remaining length
    // Lrem) of the face where the base walk met its first swept corner.  Up to there the
    // perturbed ray ran in the base ray's development, where it is a rigid image of the
    // perturbed start ray: for e_perp the ray turned by phi (sin phi = eps_v / L', L' = |v +
    // eps_v e_perp|), for e_u / e_v the ray shifted by delta = a d0 + b perp(d0).  With tau = L
    // - Lrem the base distance walked and sm the parity, it crosses the entry edge at
    //   e_perp: x' = x - tau sm sin(phi) / d'_y,  Lrem' = Lrem + (L' - L) - tau (d_y - d'_y) / d'_y
    //   shift:  x' = x - sm b / d_y,              Lrem' = Lrem + a + sm b d_x / d_y
    // (no cancellation: every correction is formed from the small quantities themselves).
    // Returns false when the record says "from the start" or the crossing leaves the edge.
    __device__ __forceinline__ bool restart(int kk) {
        const int4 r0 = __ldg(A->rst + 2 * q);
        if (r0.x < 0) return false;
        const float2 r1 = __ldg(reinterpret_cast<const float2 *>(A->rst + 2 * q + 1));
        const int h = r0.x & ((1 << 30) - 1);
        const float sm = (r0.x & (1 << 30)) ? -1.f : 1.f;
        const float bdx = __int_as_float(r0.z), bdy = __int_as_float(r0.w);
        const float Lh0 = r1.x, Ll0 = r1.y;
        const FaceRec G = load_rec(A->P.half, h);
        const float l = hl(G), x = __int_as_float(r0.y) * l;
        float ndx = bdx, ndy = bdy, xp, dl;
        if (kk == 1) {
            const float ev = A->eps_v;
            const float Lp = sqrtf(fmaf(L, L, ev * ev));
            const float sn = ev / Lp, cs = L / Lp, dL = ev * ev / (Lp + L);
            const float tau = L - (Lh0 + Ll0);
            ndx = cs * bdx - sm * sn * bdy;
            ndy = cs * bdy + sm * sn * bdx;
            if (!(ndy > 0.f)) return false;
            xp = x - tau * sm * sn / ndy;
            dl = dL - tau * (bdy * dL / Lp - sm * sn * bdx) / ndy;
        } else {
            const float ex = kk == 2 ? 1.f : w.R.x2x * w.R.il2, ey = kk == 2 ? 0.f : w.R.x2y * w.R.il2;
            const float a = A->eps_p * (ex * d0x + ey * d0y), b = A->eps_p * (ey * d0x - ex * d0y);
            if (!(bdy > 0.f)) return false;
            xp = x - sm * b / bdy;
            dl = a + sm * b * bdx / bdy;
        }
        const float sp = xp / l;
        if (!(sp >= 0.f && sp <= 1.f)) return false;
        w.h = h; w.R = G; w.mode = SG_MODE_HALF;
        w.px = sp; w.py = 0.f; w.dx = ndx; w.dy = ndy;
        {   // Lh + Ll += dl, compensated
            const float sum = Lh0 + dl, bb = sum - Lh0;
            w.Lh = sum;
            w.Ll = Ll0 + ((Lh0 - (sum - bb)) + (dl - bb));
        }
        w.st = sm < 0.f ? SG_PARITY_BIT : 0u;
        w.steps = 0;
        return true;
    }

    __device__ __forceinline__ bool init(int64_t t) {
        const int32_t task = A->tasks[t];
        q = task >> 2;
        k = task & 3;
        Carry<0> cw;
        walker_init<0>(A->P, A->in, q, w, cw);
        L = w.Lh; d0x = w.dx; d0y = w.dy;
        if (restart(k)) {
            phase = 1;
            return true;
        }
        if (k == 1) {
            float vx = L * d0x - A->eps_v * d0y, vy = L * d0y + A->eps_v * d0x;
            float Lp = sqrtf(vx * vx + vy * vy);
            w.dx = vx / Lp; w.dy = vy / Lp; w.Lh = Lp; w.Ll = 0.f;
            phase = 1;
        } else {
            ux = k == 2 ? 1.f : w.R.x2x * w.R.il2;
            uy = k == 2 ? 0.f : w.R.x2y * w.R.il2;
            w.dx = ux; w.dy = uy; w.Lh = A->eps_p; w.Ll = 0.f; w.mode = 6;
            phase = 0;
        }
        return true;
    }
    __device__ __forceinline__ bool step() {
        if (!walker_step<true, HOLE>(w, A->P)) return false;
        if (phase == 1) return true;
        // end of p -> p_u: continue with v transported along the short walk
        float vc = d0x * ux + d0y * uy, vs = ux * d0y - uy * d0x;  // v/L relative to e_u
        float s_t = (w.st & SG_PARITY_BIT) ? -1.f : 1.f;
        float nx = vc * w.dx - s_t * vs * w.dy, ny = vc * w.dy + s_t * vs * w.dx;
        w.dx = nx; w.dy = ny; w.Lh = L; w.Ll = 0.f; w.mode = 6; w.steps = 0;
        phase = 1;
        return false;
    }
    __device__ __forceinline__ void finish() {
        // the forward's end state (the task's own walker supplies the per-query fields)
        EndAdj E = end_adjoint(*A, q, w.foff);
        Walker we;
        end_walker(*A, q, w, E, we);
        const float eps = k == 1 ? A->eps_v : A->eps_p;
        A->cols[4 * q + k] = contract(pos_diff(A->P, w, we), E, eps);
        if (A->out_status) atomicOr(A->out_status + q, w.st & (SG_ST_BOUNDARY | SG_ST_MAX_STEPS | SG_ST_NEAR_VERTEX));
    }
};

template <bool HOLE>
__global__ void __launch_bounds__(128, SG_LITERAL_MINB) k_bwd_literal(BwdArgs A) {
    LiteralJob<HOLE> job;
    job.A = &A;
    run_persistent<LiteralJob<HOLE>, SG_LITERAL_REFILL, SG_LITERAL_STEPS>(A.ntask + 2, (int64_t)*A.ntask, job);
}

// The literal walks of the swept columns of a query whose forward walk was the mixed walk (a walk
// beyond the FP32 walk's range): the same two perturbed walks as LiteralJob, from the start, on
// the mixed walk (walk64.cuh).  The start and the perturbation are FP64 (the perturbed vector
// v + eps e_perp or the shift eps e_u, e_v is formed exactly, not rounded to FP32), and the
// column's difference p'' - p' is taken in FP64 face-local coordinates: an FP32 end point would
// carry an error of the order of 1e-7 of the mesh size into a difference divided by eps.
struct Literal40Job {
    const BwdArgs *A;
    W64 w;
    int64_t q;
    int k, phase;
    double L, d0x, d0y, ux, uy;

    // a walk that ended in the half-edge mode: into its face's frame (FP64)
    __device__ __forceinline__ void to_face() {
        if (w.mode == SG48_END) leave48(w, A->P4, dunpack(w.px), dunpack(w.py), dunpack(w.dx), dunpack(w.dy));
    }
    __device__ __forceinline__ bool init(int64_t t) {
        const P64 &P = A->P4;
        const QueryIn &in = A->in;
        const int32_t task = A->tasks40[t];
        q = task >> 2;
        k = task & 3;
        const int m = in.mesh_id ? __ldg(in.mesh_id + q) : 0;
        w.foff = __ldg(P.face_off + m);
        w.f = w.foff + __ldg(in.face + q);
        w.lref = (double)__ldg(P.lref + m);
        w.nearf = (float)(P.tau_near * w.lref);
        w.snapf = (float)(P.tau_snap * w.lref);
        w.R = load64(P, w.f);
        double b0 = __ldg(in.bary + 3 * q), b1 = __ldg(in.bary + 3 * q + 1), b2 = __ldg(in.bary + 3 * q + 2);
        const double sb = b0 + b1 + b2;
        b1 = fmax(b1, 0.0) / sb; b2 = fmax(b2, 0.0) / sb;
        w.px = b1 * w.R.l01 + b2 * w.R.x2x;
        w.py = b2 * w.R.x2y;
        const double *fr = P.frm64 + 6 * w.f;
        const double vx = __ldg(in.v + 3 * q), vy = __ldg(in.v + 3 * q + 1), vz = __ldg(in.v + 3 * q + 2);
        const double v1 = vx * fr[0] + vy * fr[1] + vz * fr[2], v2 = vx * fr[3] + vy * fr[4] + vz * fr[5];
        L = sqrt(v1 * v1 + v2 * v2);
        d0x = v1 / L; d0y = v2 / L;
        w.st = 0; w.steps = 0; w.ncross = 0; w.hash = SG_FNV_OFFSET; w.mode = 6;
        if (k == 1) {  // v + eps e_perp, e_perp = perp(d0)
            const double ev = A->eps_v;
            const double px = L * d0x - ev * d0y, py = L * d0y + ev * d0x, Lp = sqrt(px * px + py * py);
            w.dx = px / Lp; w.dy = py / Lp; w.L = Lp;
            phase = 1;
        } else {        // p -> p_u = Exp(p, eps e_u) (e_u = corner 0 -> 1, e_v = corner 0 -> 2)
            ux = k == 2 ? 1.0 : w.R.x2x * w.R.il2;
            uy = k == 2 ? 0.0 : w.R.x2y * w.R.il2;
            w.dx = ux; w.dy = uy; w.L = A->eps_p;
            phase = 0;
        }
        return true;
    }
    __device__ __forceinline__ bool step() {
        if (!step40<0>(w, A->P4)) return false;
        if (phase == 1) return true;
        // end of p -> p_u: continue with v transported along the short walk (its angle to the
        // walking direction kept)
        to_face();
        const double vc = d0x * ux + d0y * uy, vs = ux * d0y - uy * d0x;
        const double s_t = (w.st & SG_PARITY_BIT) ? -1.0 : 1.0;
        const double nx = vc * w.dx - s_t * vs * w.dy, ny = vc * w.dy + s_t * vs * w.dx;
        w.dx = nx; w.dy = ny; w.L = L; w.mode = 6; w.steps = 0;
        phase = 1;
        return false;
    }
    __device__ __forceinline__ void finish() {
        to_face();
        const P64 &P = A->P4;
        const EndAdj E = end_adjoint(*A, q, w.foff);
        // p'' - p' = (x0_a - x0_b) + (px e1_a + py e2_a) - (b1 (x1_b - x0_b) + b2 (x2_b - x0_b))
        const int4 ta = __ldg(P.fv + w.f), tb = __ldg(P.fv + E.gfe);
        const float4 a0 = __ldg(P.V + ta.x), c0 = __ldg(P.V + tb.x), c1 = __ldg(P.V + tb.y), c2 = __ldg(P.V + tb.z);
        const double *fr = P.frm64 + 6 * w.f;
        const double b1 = __ldg(A->end_bary + 3 * q + 1), b2 = __ldg(A->end_bary + 3 * q + 2);
        double d[3];
        const double ax[3] = {a0.x, a0.y, a0.z}, x0[3] = {c0.x, c0.y, c0.z}, x1[3] = {c1.x, c1.y, c1.z},
                     x2[3] = {c2.x, c2.y, c2.z};
        for (int i = 0; i < 3; ++i)
            d[i] = (ax[i] - x0[i]) + (w.px * fr[i] + w.py * fr[3 + i]) - (b1 * (x1[i] - x0[i]) + b2 * (x2[i] - x0[i]));
        const double dn = d[0] * E.nm.x + d[1] * E.nm.y + d[2] * E.nm.z;
        const double c = ((d[0] - dn * E.nm.x) * E.g.x + (d[1] - dn * E.nm.y) * E.g.y + (d[2] - dn * E.nm.z) * E.g.z);
        A->cols[4 * q + k] = (float)(c / (k == 1 ? A->eps_v : A->eps_p));
        if (A->out_status) atomicOr(A->out_status + q, w.st & (SG_ST_BOUNDARY | SG_ST_MAX_STEPS | SG_ST_NEAR_VERTEX));
    }
};

// resident blocks per SM of the mixed literal walks (the mixed forward walk's residency)
#ifndef SG_LITERAL40_MINB
#define SG_LITERAL40_MINB 5
#endif
__global__ void __launch_bounds__(128, SG_LITERAL40_MINB) k_bwd_literal40(BwdArgs A) {
    Literal40Job job;
    job.A = &A;
    run_persistent<Literal40Job, SG_LITERAL_REFILL>(A.ntask + 5, (int64_t)A.ntask[4], job);
}

// Columns the re-walk found unswept are chords from p' (the par column always is); the swept
// ones were written by k_bwd_literal.  Then the columns are contracted into the gradients.
// Without WALK a query whose chord leaves the end face is left for a second pass (false).
template <bool HOLE, bool WALK>
__device__ __forceinline__ bool assemble_query(const BwdArgs &A, int64_t q) {
    const WalkParams &P = A.P;
    Walker w;
    Carry<0> cw;
    bool live = walker_init<0>(P, A.in, q, w, cw);
    F3 gv = f3(0.f, 0.f, 0.f), gp = gv, gb = gv;
    if (live && !(w.st & SG_ST_INVALID)) {
        float4 c = *reinterpret_cast<const float4 *>(A.cols + 4 * q);
        const unsigned split = __float_as_uint(c.x);
        bool ok = true;
        {
            const float d0x = w.dx, d0y = w.dy;
            EndAdj E = end_adjoint(A, q, w.foff);
            Walker we;
            end_walker(A, q, w, E, we);
            float ux, uy;
            c.x = chord_col<HOLE, WALK>(P, we, E, E.dmx, E.dmy, A.eps_v, ok);
            if (!(split & 1u)) {
                rmap(-d0y, d0x, d0x, d0y, E, ux, uy);
                c.y = chord_col<HOLE, WALK>(P, we, E, ux, uy, A.eps_v, ok);
            }
            if (!(split & 2u)) {
                rmap(1.f, 0.f, d0x, d0y, E, ux, uy);
                c.z = chord_col<HOLE, WALK>(P, we, E, ux, uy, A.eps_p, ok);
            }
            if (!(split & 4u)) {
                rmap(w.R.x2x * w.R.il2, w.R.x2y * w.R.il2, d0x, d0y, E, ux, uy);
                c.w = chord_col<HOLE, WALK>(P, we, E, ux, uy, A.eps_p, ok);
            }
        }
        if (!WALK && !ok) return false;
        Fr2 F0 = load_frm(P, w.f);
        gv = c.x * lift(F0, w.dx, w.dy) + c.y * lift(F0, -w.dy, w.dx);
        F3 eu = lift(F0, 1.f, 0.f), ev = lift(F0, w.R.x2x * w.R.il2, w.R.x2y * w.R.il2);
        float a11 = dot3(eu, eu), a12 = dot3(eu, ev), a22 = dot3(ev, ev);
        float det = a11 * a22 - a12 * a12;
        float c0 = (a22 * c.z - a12 * c.w) / det, c1 = (-a12 * c.z + a11 * c.w) / det;
        gp = c0 * eu + c1 * ev;
        int4 t = __ldg(P.fv + w.f);
        gb = f3(dot3(gp, vpos(P, t.x)), dot3(gp, vpos(P, t.y)), dot3(gp, vpos(P, t.z)));
    }
    if (A.grad_v) st3(A.grad_v, q, gv);
    if (A.grad_p) st3(A.grad_p, q, gp);
    if (A.grad_bary) st3(A.grad_bary, q, gb);
    return true;
}

// One thread per query; the few queries with a chord that leaves the end face (a few percent)
// go to a list for k_bwd_assemble_walk, which keeps the walk's registers out of this kernel.
template <bool HOLE>
__global__ void __launch_bounds__(128, SG_ASSEMBLE_MINB) k_bwd_assemble(BwdArgs A) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.nq) return;
    if (!assemble_query<HOLE, false>(A, q)) A.tasks[atomicAdd(A.ntask + 3, 1)] = (int32_t)q;
}

template <bool HOLE>
__global__ void __launch_bounds__(128) k_bwd_assemble_walk(BwdArgs A) {
    const int n = A.ntask[3];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        assemble_query<HOLE, true>(A, A.tasks[i]);
}

// ------------------------------------------------------------------ end-barycentric upstream
// An upstream gradient on the end barycentrics b' enters every estimator as its tangent
// equivalent g_t (bary_grad_to_tangent), added to g_pos once before the other kernels run.
__global__ void __launch_bounds__(256) k_fold_gbary(BwdArgs A, const float *g_pos, float *g_eff) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.nq) return;
    F3 g = ld3(g_pos, q);
    const int m = A.in.mesh_id ? __ldg(A.in.mesh_id + q) : 0;
    const int lf = __ldg(A.end_face + q);
    if (m >= 0 && m < A.in.n_mesh) {
        const int foff = __ldg(A.P.face_off + m);
        if (lf >= 0 && lf < __ldg(A.P.face_off + m + 1) - foff)
            g = g + bary_grad_to_tangent(A.P, foff + lf, ld3(A.g_bary, q));
    }
    st3(g_eff, q, g);
}

// For grad_V: b' also moves with the end vertices at a fixed end point (sum_k x_k db'_k =
// dp' - sum_k b'_k dx_k), which takes b'_k g_t off each end vertex of a query the re-walk
// differentiated.
__global__ void __launch_bounds__(256) k_gradv_gbary(BwdArgs A) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.nq) return;
    Walker w;
    Carry<0> cw;
    if (!walker_init<0>(A.P, A.in, q, w, cw) || (w.st & SG_ST_INVALID)) return;
    const uint32_t fst = __ldg(A.end_status + q);
    if (fst & (SG_ST_VERTEX_HIT | SG_ST_BOUNDARY | SG_ST_MAX_STEPS | SG_ST_INVALID | SG_ST_HOLE)) return;
    const int gfe = w.foff + __ldg(A.end_face + q);
    const F3 gt = bary_grad_to_tangent(A.P, gfe, ld3(A.g_bary, q));
    const F3 b = ld3(A.end_bary, q);
    const int4 t = __ldg(A.P.fv + gfe);
    atomic_add3(A.gacc, t.x, (-b.x) * gt);
    atomic_add3(A.gacc, t.y, (-b.y) * gt);
    atomic_add3(A.gacc, t.z, (-b.z) * gt);
}

// ------------------------------------------------------------------ direction and carried vectors
// Sec. 4 "Parallel Transport": along the walk the direction and every carried vector keep their
// angle to each other, so for a fixed face sequence w' = R w with R = M_p' M_p^T the rotation of
// Eq. proxy_func, and grad_w = R^T g_w (exact).  The direction d' = R v/|v| is differentiated
// with R held fixed, as EP does for the end point (under both estimators: GFD's differences
// are taken of end points only): grad_v += (I - d0 d0^T) R^T g_dir / |v|.
__global__ void __launch_bounds__(256) k_bwd_transport(BwdArgs A) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= A.nq) return;
    const WalkParams &P = A.P;
    Walker w;
    Carry<0> cw;
    walker_init<0>(P, A.in, q, w, cw);
    // zero-length queries included: their transport is the identity in the start face
    const bool valid = !(w.st & SG_ST_INVALID);
    F3 gw[SG_BWD_MAX_W];
    for (int k = 0; k < A.n_w; ++k) gw[k] = f3(0.f, 0.f, 0.f);
    if (valid) {
        const int gfe = w.foff + __ldg(A.end_face + q);
        const Fr2 Fm = load_frm(P, gfe), F0 = load_frm(P, w.f);
        F3 dd = ld3(A.end_dir, q);
        float dmx = dd.x * Fm.e1x + dd.y * Fm.e1y + dd.z * Fm.e1z;
        float dmy = dd.x * Fm.e2x + dd.y * Fm.e2y + dd.z * Fm.e2z;
        const float n2 = dmx * dmx + dmy * dmy;
        if (n2 > 0.f) { const float r = rsqrtf(n2); dmx *= r; dmy *= r; }
        const uint32_t est = A.end_status ? __ldg(A.end_status + q) : 0u;
        const float sm = (est & SG_ST_FLIPPED) ? -1.f : 1.f;
        // a zero vector v has no direction: the forward measured carried vectors against e1
        // at both ends of its empty path
        const bool nod = w.dx == 0.f && w.dy == 0.f;
        const float d0x = nod ? 1.f : w.dx, d0y = nod ? 0.f : w.dy;
        if (nod) { dmx = 1.f; dmy = 0.f; }
        // R^T g for a tangent g at the end, as a start-frame 2-vector (along, across d0)
        auto back = [&](F3 g, float &al, float &ac) {
            const float gx = g.x * Fm.e1x + g.y * Fm.e1y + g.z * Fm.e1z;
            const float gy = g.x * Fm.e2x + g.y * Fm.e2y + g.z * Fm.e2z;
            al = gx * dmx + gy * dmy;
            ac = sm * (-gx * dmy + gy * dmx);
        };
        if (A.g_dir && A.grad_v) {
            const F3 v = ld3(A.in.v, q);
            const float v1 = v.x * F0.e1x + v.y * F0.e1y + v.z * F0.e1z, v2 = v.x * F0.e2x + v.y * F0.e2y + v.z * F0.e2z;
            const float Lv = sqrtf(v1 * v1 + v2 * v2);
            if (Lv > 0.f) {
                float al, ac;
                back(ld3(A.g_dir, q), al, ac);
                const F3 add = (ac / Lv) * lift(F0, -d0y, d0x);
                A.grad_v[3 * q] += add.x; A.grad_v[3 * q + 1] += add.y; A.grad_v[3 * q + 2] += add.z;
            }
        }
        if (A.g_w) {
            for (int k = 0; k < A.n_w; ++k) {
                float al, ac;
                back(ld3(A.g_w, (int64_t)A.n_w * q + k), al, ac);
                gw[k] = lift(F0, al * d0x - ac * d0y, al * d0y + ac * d0x);
            }
        }
    }
    if (A.grad_w)
        for (int k = 0; k < A.n_w; ++k) st3(A.grad_w, (int64_t)A.n_w * q + k, gw[k]);
}

// the coefficients of edge k of face f in f's orientation: windows k (first half) and k-1
// (second half)
__device__ __forceinline__ float2 window_sum(const float4 *__restrict__ wacc, int f, int k) {
    const float4 a = wacc[3 * f + k], b = wacc[3 * f + prv(k)];
    return make_float2(a.x + b.z, a.y + b.w);
}

// per interior edge: its coefficients (summed over the windows of its two faces, in the
// canonical half-edge's orientation) times N_a + N_b (the outward in-plane normals of the edge
// in its two faces, N = F_f (sa, -ca) of each half-edge), added to the canonical half-edge's
// start and end vertices
__global__ void k_gradv_edges(int64_t nE, WalkParams P, const int2 *__restrict__ edges, const float4 *__restrict__ wacc,
                              float4 *gacc) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nE) return;
    const int2 hh = __ldg(edges + e);
    const int fa = hh.x / 3, ka = hh.x - 3 * fa, fb = hh.y / 3, kb = hh.y - 3 * fb;
    const float2 ca = window_sum(wacc, fa, ka), cb = window_sum(wacc, fb, kb);
    // fb lists the edge in the opposite direction unless the adjacency is flipped
    const int4 na = __ldg(P.rec + 2 * fa);
    const bool flip = (sel3(ka, na.x, na.y, na.z) >> 2) & 1;
    const float2 c = flip ? make_float2(ca.x + cb.x, ca.y + cb.y) : make_float2(ca.x + cb.y, ca.y + cb.x);
    if (c.x == 0.f && c.y == 0.f) return;
    const FaceRec Ha = load_rec(P.half, hh.x), Hb = load_rec(P.half, hh.y);
    const F3 N = lift(load_frm(P, fa), hsa(Ha), -hca(Ha)) + lift(load_frm(P, fb), hsa(Hb), -hca(Hb));
    const int4 t = __ldg(P.fv + fa);
    atomic_add3(gacc, sel3(ka, t.x, t.y, t.z), c.x * N);
    atomic_add3(gacc, sel3(nxt(ka), t.x, t.y, t.z), c.y * N);
}

__global__ void k_gradv_flush(int64_t nV, const float4 *__restrict__ gacc, float *grad_V) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nV) return;
    float4 a = gacc[v];
    grad_V[3 * v] += a.x;
    grad_V[3 * v + 1] += a.y;
    grad_V[3 * v + 2] += a.z;
}

// ------------------------------------------------------------------ host
namespace {
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// SM-filling grid of 128-thread blocks for a persistent kernel over n tasks
template <class K>
unsigned persistent_grid(K kernel, int64_t n) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 128, 0);
    int64_t need = (n + 127) / 128;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * std::max(per, 1), need));
}
struct BwdLayout {
    size_t gacc, wacc, cols, tasks, tasks40, rst, ntask, gpos, lcounts, lkeys, perm, total;
};
// The re-walk takes its queries longest first (the forward's length order, rebuilt here) for
// batches of at least this many queries, unless opts.sort is 0.
#define SG_BWD_LORDER_MIN 65536
bool bwd_lorder(const sg_opts &r, int64_t nq) { return r.sort == 2 || (r.sort < 0 && nq >= SG_BWD_LORDER_MIN); }

BwdLayout bwd_layout(int64_t nV, int64_t nF, int64_t nq, int32_t estimator, bool grad_V, bool lorder) {
    BwdLayout L{};
    size_t o = 0;
    L.ntask = o; o = align_up(o + 64, 256);
    L.gpos = o; o = align_up(o + sizeof(float) * 3 * (size_t)std::max<int64_t>(nq, 1), 256);
    if (lorder) {
        L.lcounts = o; o = align_up(o + sizeof(int32_t) * 2 * SG_LBUCKETS, 256);
        L.lkeys = o; o = align_up(o + (size_t)std::max<int64_t>(nq, 1), 256);
        L.perm = o; o = align_up(o + sizeof(int32_t) * (size_t)std::max<int64_t>(nq, 1), 256);
    }
    if (grad_V) {
        L.gacc = o; o = align_up(o + sizeof(float4) * (size_t)nV, 256);
        L.wacc = o; o = align_up(o + sizeof(float4) * 3 * (size_t)std::max<int64_t>(nF, 1), 256);
    }
    if (estimator == SG_EST_GFD) {
        L.cols = o; o = align_up(o + sizeof(float) * 4 * (size_t)std::max<int64_t>(nq, 1), 256);
        L.tasks = o; o = align_up(o + sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(nq, 1), 256);
        L.tasks40 = o; o = align_up(o + sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(nq, 1), 256);
        L.rst = o; o = align_up(o + sizeof(int4) * 2 * (size_t)std::max<int64_t>(nq, 1), 256);
    }
    L.total = o;
    return L;
}
}  // namespace

extern "C" sg_status sg_exp_map_backward_workspace_size(const sg_mesh *m, int32_t estimator, int64_t nq,
                                                        int32_t want_grad_V, size_t *bytes) {
    if (!m || !bytes || nq < 0) return SG_ERR_INVALID_ARG;
    if (estimator != SG_EST_EP && estimator != SG_EST_GFD) return SG_ERR_INVALID_ARG;
    // room for the length order whatever the options (the layout without it is smaller)
    *bytes = bwd_layout(m->nV, m->nF, nq, estimator, want_grad_V != 0, true).total;
    return SG_OK;
}

extern "C" sg_status sg_exp_map_backward(const sg_mesh *m, int32_t estimator, float eps_v, float eps_p, int64_t nq,
                                         const int32_t *mesh_id, const int32_t *face, const float *bary,
                                         const float *v, const int32_t *end_face, const float *end_bary,
                                         const float *end_dir, const uint32_t *end_status, const float *g_pos,
                                         const float *g_bary, const float *g_dir, int32_t n_w, const float *g_w,
                                         float *grad_v, float *grad_p, float *grad_bary, float *grad_V,
                                         float *grad_w, uint32_t *out_status, const sg_opts *o, void *stream) {
    if (!m || nq < 0) return SG_ERR_INVALID_ARG;
    if (estimator != SG_EST_EP && estimator != SG_EST_GFD) return SG_ERR_INVALID_ARG;
    if (nq == 0) return SG_OK;
    if (nq > (int64_t)(INT32_MAX / 4) - 1024) return SG_ERR_INVALID_ARG;
    if (!face || !bary || !v || !end_face || !end_bary || !end_dir || !g_pos) return SG_ERR_INVALID_ARG;
    if (grad_V && !end_status) return SG_ERR_INVALID_ARG;
    if (n_w < 0 || n_w > SG_BWD_MAX_W || (n_w > 0 && (!g_w) != (!grad_w))) return SG_ERR_INVALID_ARG;
    if (estimator == SG_EST_GFD && !(eps_v > 0.f && eps_p > 0.f)) return SG_ERR_INVALID_ARG;
    sg_opts r;
    sg_opts_default(&r);
    if (o) r = *o;
    if (r.boundary_mode != 0 && r.boundary_mode != 1) return SG_ERR_INVALID_ARG;
    if (r.precision >= 40) return SG_ERR_UNSUPPORTED;
    if (r.max_steps <= 0) r.max_steps = 1 << 20;
    if (r.tau_near <= 0.f) r.tau_near = 1e-4f;
    if (r.tau_snap <= 0.f) r.tau_snap = fminf(1e-6f, r.tau_near);
    if (r.tau_snap > r.tau_near) return SG_ERR_INVALID_ARG;  // a snapped vertex lies in the near band
    cudaStream_t s = (cudaStream_t)stream;
    BwdArgs A{};
    A.P.rec = m->d_rec; A.P.fv = m->d_fv; A.P.frm = m->d_frm; A.P.half = m->d_half; A.P.V = m->d_V; A.P.face_off = m->d_face_off;
    A.P.lref = m->d_lref;
    A.P.max_steps = r.max_steps; A.P.tau_near = r.tau_near; A.P.tau_snap = r.tau_snap; A.P.want_hash = 0;
    A.in.n_mesh = m->n_mesh; A.in.mesh_id = mesh_id; A.in.face = face; A.in.bary = bary; A.in.v = v;
    A.in.length = nullptr; A.in.w = nullptr;
    A.nq = nq;
    A.end_face = end_face; A.end_bary = end_bary; A.end_dir = end_dir; A.end_status = end_status; A.g_pos = g_pos;
    A.g_bary = g_bary; A.g_dir = g_dir; A.n_w = grad_w ? n_w : 0; A.g_w = g_w;
    A.grad_v = grad_v; A.grad_p = grad_p; A.grad_bary = grad_bary; A.grad_V = grad_V; A.grad_w = grad_w;
    A.out_status = out_status;
    A.eps_v = eps_v; A.eps_p = eps_p;

    // only the re-walk uses an order: the caller's (sg_opts.order, filled by the forward call), else
    // the length order rebuilt here
    const bool rewalk = estimator == SG_EST_GFD || grad_V;
    const bool lorder = rewalk && !r.order && bwd_lorder(r, nq);
    BwdLayout Lw = bwd_layout(m->nV, m->nF, nq, estimator, grad_V != nullptr, lorder);
    void *ws = nullptr;
    bool own = false;
    if (r.workspace) {
        if (r.workspace_bytes < Lw.total) return SG_ERR_OOM;
        ws = r.workspace;
    } else {
        if (cudaMallocAsync(&ws, Lw.total, s) != cudaSuccess) { cudaGetLastError(); return SG_ERR_OOM; }
        own = true;
    }
    char *base = (char *)ws;
    A.ntask = (int32_t *)(base + Lw.ntask);
    if (grad_V) {
        A.gacc = (float4 *)(base + Lw.gacc);
        A.wacc = (float4 *)(base + Lw.wacc);
    }
    if (estimator == SG_EST_GFD) {
        A.cols = (float *)(base + Lw.cols);
        A.tasks = (int32_t *)(base + Lw.tasks);
        A.tasks40 = (int32_t *)(base + Lw.tasks40);
        A.rst = (int4 *)(base + Lw.rst);
        // the wide-precision geometry of the mixed literal walks (built with the mesh; re-derived
        // here after a vertex update)
        sg_status st64 = sg_geom64_prepare(const_cast<sg_mesh *>(m), s, true);
        if (st64 != SG_OK) {
            if (own) cudaFreeAsync(ws, s);
            return st64;
        }
        P64 &Q = A.P4;
        Q.rec = m->d_rec; Q.half48 = m->d_half48; Q.half = m->d_half; Q.frm = m->d_frm; Q.rec64 = m->d_rec64;
        Q.frm64 = m->d_frm64; Q.th64 = m->d_th64; Q.fv = m->d_fv; Q.V = m->d_V; Q.face_off = m->d_face_off;
        Q.lref = m->d_lref; Q.max_steps = r.max_steps; Q.want_hash = 0; Q.tau_near = r.tau_near; Q.tau_snap = r.tau_snap;
    }
    cudaMemsetAsync(A.ntask, 0, 64, s);
    if (rewalk && r.order) {
        A.perm = r.order;
    } else if (lorder) {
        int32_t *perm = (int32_t *)(base + Lw.perm);
        sg_length_order(m, A.in, nq, (uint8_t *)(base + Lw.lkeys), (int32_t *)(base + Lw.lcounts), perm, s);
        A.perm = perm;
    }
    const unsigned gq256 = (unsigned)((nq + 255) / 256);
    if (g_bary) {  // fold the end-barycentric gradient into an effective g_pos
        float *geff = (float *)(base + Lw.gpos);
        k_fold_gbary<<<gq256, 256, 0, s>>>(A, g_pos, geff);
        A.g_pos = geff;
    }
    if (grad_V) {
        cudaMemsetAsync(A.gacc, 0, sizeof(float4) * (size_t)m->nV, s);
        cudaMemsetAsync(A.wacc, 0, sizeof(float4) * 3 * (size_t)std::max<int64_t>(m->nF, 1), s);
    }
    const unsigned g128 = (unsigned)((nq + 127) / 128), g256 = (unsigned)((nq + 255) / 256);
    if (estimator == SG_EST_EP) {
        k_ep_backward<<<g256, 256, 0, s>>>(A);
        // the grad_V re-walk rewrites the status with its walk's bits and SG_ST_NO_GRADV
        if (grad_V) k_bwd_rewalk<false, true><<<persistent_grid(k_bwd_rewalk<false, true>, nq), 128, 0, s>>>(A);
    } else {
        cudaEvent_t *pev = (cudaEvent_t *)r.prof_events;
        if (pev) cudaEventRecord(pev[0], s);
        if (grad_V) k_bwd_rewalk<true, true><<<persistent_grid(k_bwd_rewalk<true, true>, nq), 128, 0, s>>>(A);
        else k_bwd_rewalk<true, false><<<persistent_grid(k_bwd_rewalk<true, false>, nq), 128, 0, s>>>(A);
        if (pev) cudaEventRecord(pev[1], s);
        // the literal walks are done with the task list: the assemble pass reuses it for the
        // queries it defers (a chord that leaves the end face), counted in ntask[3]
        const unsigned gw = persistent_grid(k_bwd_assemble_walk<false>, nq / 16 + 1);
        if (r.boundary_mode) {
            k_bwd_literal<true><<<persistent_grid(k_bwd_literal<true>, 3 * nq), 128, 0, s>>>(A);
            k_bwd_assemble<true><<<g128, 128, 0, s>>>(A);
            k_bwd_assemble_walk<true><<<gw, 128, 0, s>>>(A);
        } else {
            k_bwd_literal<false><<<persistent_grid(k_bwd_literal<false>, 3 * nq), 128, 0, s>>>(A);
            k_bwd_literal40<<<persistent_grid(k_bwd_literal40, 3 * nq), 128, 0, s>>>(A);
            k_bwd_assemble<false><<<g128, 128, 0, s>>>(A);
            k_bwd_assemble_walk<false><<<gw, 128, 0, s>>>(A);
        }
    }
    if ((g_dir && grad_v) || (A.n_w > 0)) k_bwd_transport<<<g256, 256, 0, s>>>(A);
    if (grad_V) {
        if (g_bary) k_gradv_gbary<<<g256, 256, 0, s>>>(A);
        if (m->nE > 0)
            k_gradv_edges<<<(unsigned)((m->nE + 255) / 256), 256, 0, s>>>(m->nE, A.P, m->d_edges, A.wacc, A.gacc);
        k_gradv_flush<<<(unsigned)((m->nV + 255) / 256), 256, 0, s>>>(m->nV, A.gacc, grad_V);
    }
    if (own) cudaFreeAsync(ws, s);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

// The adjoint of the parallel transport along each query's geodesic, which is its inverse
// (App. "Additional Details on Mesh-LBFGS and GCVT": the vector is moved backwards on the
// curve).  For a fixed face sequence the transport is a rotation of the tangent planes that
// keeps each vector's signed angle to the walking direction, so the inverse is the rotation's
// transpose: the transport kernel's R^T applied to u, with no walk.
extern "C" sg_status sg_transport_back(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face,
                                       const float *bary, const float *v, const int32_t *end_face,
                                       const float *end_dir, const uint32_t *end_status, int32_t n_u,
                                       const float *u, float *out_u, const sg_opts *o, void *stream) {
    if (!m || nq < 0) return SG_ERR_INVALID_ARG;
    if (n_u < 0 || n_u > SG_BWD_MAX_W) return SG_ERR_INVALID_ARG;
    if (nq == 0 || n_u == 0) return SG_OK;
    if (nq > (int64_t)(INT32_MAX / 4) - 1024) return SG_ERR_INVALID_ARG;
    if (!face || !bary || !v || !end_face || !end_dir || !u || !out_u) return SG_ERR_INVALID_ARG;
    sg_opts r;
    sg_opts_default(&r);
    if (o) r = *o;
    if (r.precision >= 40) return SG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    BwdArgs A{};
    A.P.rec = m->d_rec; A.P.fv = m->d_fv; A.P.frm = m->d_frm; A.P.half = m->d_half; A.P.V = m->d_V; A.P.face_off = m->d_face_off;
    A.P.lref = m->d_lref;
    A.P.max_steps = 1; A.P.tau_near = 1e-4f; A.P.tau_snap = 1e-6f; A.P.want_hash = 0;
    A.in.n_mesh = m->n_mesh; A.in.mesh_id = mesh_id; A.in.face = face; A.in.bary = bary; A.in.v = v;
    A.in.length = nullptr; A.in.w = nullptr;
    A.nq = nq;
    A.end_face = end_face; A.end_dir = end_dir; A.end_status = end_status;
    A.n_w = n_u; A.g_w = u; A.grad_w = out_u;
    k_bwd_transport<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(A);
    return cudaGetLastError() == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}
