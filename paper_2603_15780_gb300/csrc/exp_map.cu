// exp_map.cu -- forward exponential map kernels, start-face sort, mesh upload and C ABI.
//
// Alg. "Parallel Geodesic Tracing CUDA Kernel" gives one thread per geodesic.  Two launch
// shapes are provided:
//   k_walk_plain       exactly that shape (grid = ceil(nq / block)), FP32 only;
//   k_walk_persistent  an SM-filling grid whose lanes pull query indices from an atomic
//                      counter as soon as their current walk ends, so lanes do not idle
//                      behind the longest walk of their warp (the long tail of path
//                      lengths the paper leaves to idle threads).  Queries can be taken in
//                      start-face order (counting sort by the start face's place on the
//                      mesh's Z-order curve of face centroids) so that neighbouring lanes start
//                      in one patch of the surface and gather nearby records.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "sgeo_internal.h"
#include "walk.cuh"

#define SG_MAX_W 4
// lanes of a warp that must be idle before the forward walk refills them together (walk on 1M
// queries of the 81,920-face sphere, length order, 256-bit record loads: 8 lanes 0.412 ms, 12
// 0.403, 16 0.424, 20 0.432)
// walk steps between refill checks of the forward walk (one: 0.522 ms against 0.389 ms with two)
// and of the trace
#ifndef SG_WALK_STEPS
#define SG_WALK_STEPS 2
#endif
#ifndef SG_TRACE_STEPS
#define SG_TRACE_STEPS 2
#endif
#ifndef SG_WALK_REFILL
#define SG_WALK_REFILL 12
#endif
// lanes of a warp with a pending hole-avoidance boundary event before those events run together
#ifndef SG_HOLE_BATCH
#define SG_HOLE_BATCH 24
#endif

struct FwdArgs {
    WalkParams P;
    QueryIn in;
    int64_t nq;
    int32_t nF_total;
    int32_t *out_face;
    float *out_bary, *out_pos, *out_dir, *out_w;
    uint32_t *out_status;
    int32_t *out_ncross;
    uint64_t *out_hash;
    const int32_t *__restrict__ perm;  // queue position -> query index (NULL: identity)
    int32_t *counter;                  // persistent work counter
    // automatic precision: queries handed to the mixed walk (precision 40) are appended to
    // esc_list (count in *esc_count) and left unwritten -- those whose length exceeds
    // esc_lmax l_ref at the start, and those whose crossing count reaches esc_ncross
    int32_t *esc_list, *esc_count;
    float esc_lmax;
    int32_t esc_ncross;
    // when a query order routed the long queries to the mixed walk: the head of perm it takes
    // (*route_n queries; the persistent FP32 walk's ticket counter starts there)
    const int32_t *route_n;
    // the mixed walk under the automatic precision: its tasks are the routed head of perm, then
    // the escalation list (lengths from device memory)
    int mix_lists;
};

// Appends query q to the escalation list (warp-aggregated: one atomic per calling warp).
__device__ __forceinline__ void escalate(const FwdArgs &a, int64_t q) {
    const unsigned mask = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(a.esc_count, __popc(mask));
    base = __shfl_sync(mask, base, leader);
    a.esc_list[base + __popc(mask & ((1u << lane) - 1u))] = (int32_t)q;
}

template <int NW>
__device__ void walker_finish(const FwdArgs &a, int64_t q, const Walker &w, const Carry<NW> &cw) {
    const FaceRec &R = w.R;
    float b2 = w.py / R.x2y;
    float b1 = (w.px - b2 * R.x2x) / R.l01;
    float b0 = 1.f - b1 - b2;
    Frame3 F = face_frame(a.P, w.f);
    a.out_face[q] = w.f - w.foff;
    a.out_bary[3 * q] = b0; a.out_bary[3 * q + 1] = b1; a.out_bary[3 * q + 2] = b2;
    a.out_pos[3 * q] = b0 * F.ox + b1 * F.x1x + b2 * F.x2x;
    a.out_pos[3 * q + 1] = b0 * F.oy + b1 * F.x1y + b2 * F.x2y;
    a.out_pos[3 * q + 2] = b0 * F.oz + b1 * F.x1z + b2 * F.x2z;
    a.out_dir[3 * q] = w.dx * F.e1x + w.dy * F.e2x;
    a.out_dir[3 * q + 1] = w.dx * F.e1y + w.dy * F.e2y;
    a.out_dir[3 * q + 2] = w.dx * F.e1z + w.dy * F.e2z;
    if (NW > 0 && a.out_w) {
        const float sg = (w.st & SG_PARITY_BIT) ? -1.f : 1.f;
        const bool nod = w.dx == 0.f && w.dy == 0.f;   // zero vector v: components against e1
        const float rx = nod ? 1.f : w.dx, ry = nod ? 0.f : w.dy;
        for (int k = 0; k < NW; ++k) {
            float c = cw.c[k], s = sg * cw.s[k];
            float u1 = c * rx - s * ry, u2 = c * ry + s * rx;
            float *o = a.out_w + (3 * NW) * q + 3 * k;
            o[0] = u1 * F.e1x + u2 * F.e2x;
            o[1] = u1 * F.e1y + u2 * F.e2y;
            o[2] = u1 * F.e1z + u2 * F.e2z;
        }
    }
    a.out_status[q] = (w.st & ~SG_PARITY_BIT) | ((w.st & SG_PARITY_BIT) ? SG_ST_FLIPPED : 0u);
    if (a.out_ncross) a.out_ncross[q] = w.ncross;
    if (a.out_hash) a.out_hash[q] = w.hash;
}

// One thread per query (Alg. "Parallel Geodesic Tracing CUDA Kernel"), or several queries in turn
// (grid-stride) when the grid is smaller than the batch (sg_opts.queries_per_thread).
template <int NW, bool ESC = false, bool AUTO = false>
__global__ void __launch_bounds__(256) k_walk_plain(FwdArgs a) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < a.nq; q += (int64_t)gridDim.x * blockDim.x) {
        Walker w;
        Carry<NW> cw;
        if (walker_init<NW>(a.P, a.in, q, w, cw)) {
            if (AUTO && w.Lh > a.esc_lmax * w.lref) {
                escalate(a, q);
                continue;
            }
            while (!walker_step<ESC>(w, a.P)) {
            }
            // the step cap of an AUTO walk is its crossing budget (see FwdJob)
            if (AUTO && a.esc_ncross && (w.st & SG_ST_MAX_STEPS)) {
                escalate(a, q);
                continue;
            }
        }
        walker_finish<NW>(a, q, w, cw);
    }
}

// AUTO: the automatic precision -- the query order gave the long queries to the mixed walk, and
// a query leaves this FP32 walk for the mixed walk when its walk reaches the crossing budget.  The
// budget is the walk's step cap (P.max_steps, set to it by the host; a crossing is a step, so no
// walk kept here crosses more edges than that), which costs no test of its own per step; a walk
// stopped by it is handed on (esc_ncross != 0) unless the caller's own cap is that low.
template <int NW, bool ESC, bool HOLE = false, bool AUTO = false>
struct FwdJob {
    const FwdArgs *a;
    Walker w;
    Carry<NW> cw;
    int64_t q;
    __device__ __forceinline__ bool init(int64_t t) {
        q = a->perm ? (int64_t)__ldg(a->perm + t) : t;
        return walker_init<NW>(a->P, a->in, q, w, cw);
    }
    __device__ __forceinline__ bool step() {
        if (HOLE) {
            // boundary events of hole avoidance wait until several lanes have one (or every
            // stepping lane does), then run together
            const bool pend = w.mode >= SG_MODE_HOLE_EDGE;
            const unsigned act = __activemask();
            const unsigned pm = __ballot_sync(act, pend);
            if (pend && __popc(pm) < SG_HOLE_BATCH && pm != act) return false;
        }
        return walker_step<ESC, HOLE>(w, a->P);
    }
    __device__ __forceinline__ void finish() {
        if (AUTO && a->esc_ncross && (w.st & SG_ST_MAX_STEPS)) {
            // (one atomic per such query: these are the walks that outran their predicted
            // length, and an aggregated append here costs the walk registers)
            a->esc_list[atomicAdd(a->esc_count, 1)] = (int32_t)q;
            return;
        }
        walker_finish<NW>(*a, q, w, cw);
    }
};

template <int NW, bool ESC, bool AUTO = false>
__global__ void __launch_bounds__(256, 4) k_walk_persistent(FwdArgs a) {
    FwdJob<NW, ESC, false, AUTO> job;
    job.a = &a;
    run_persistent<FwdJob<NW, ESC, false, AUTO>, SG_WALK_REFILL, SG_WALK_STEPS>(a.counter, a.nq, job);
}

// The mixed walk (precision 40; walk.cuh, MIX): the FP32 walker with the direction in
// double-float, a double-float start and the double-float half-edge records.  With mix_lists its
// tasks are the automatic precision's: perm[0, *route_n), then esc_list[0, *esc_count).
template <int NW, bool ESC>
struct MixJob {
    const FwdArgs *a;
    Walker w;
    Carry<NW> cw;
    int64_t q, n1;
    __device__ __forceinline__ bool init(int64_t t) {
        if (a->mix_lists) q = t < n1 ? (int64_t)__ldg(a->perm + t) : (int64_t)__ldg(a->esc_list + (t - n1));
        else q = a->perm ? (int64_t)__ldg(a->perm + t) : t;
        w.dxl = 0.f; w.dyl = 0.f;
        const bool live = walker_init<NW>(a->P, a->in, q, w, cw);
        if (live) walker_start_mix(a->P, a->in, q, w);
        return live;
    }
    __device__ __forceinline__ bool step() { return walker_step<ESC, false, true>(w, a->P); }
    __device__ __forceinline__ void finish() {
        w.st |= SG_ST_MIXED;
        walker_finish<NW>(*a, q, w, cw);
    }
};

#ifndef SG_MIX_MINB
#define SG_MIX_MINB 4
#endif
// walk steps between the mixed walk's refill checks (64-mesh batch: 2 steps 17.2 ms, 1 step 17.8 ms)
#ifndef SG_MIX_STEPS
#define SG_MIX_STEPS 2
#endif
template <int NW, bool ESC>
__global__ void __launch_bounds__(256, SG_MIX_MINB) k_walk_mixed(FwdArgs a) {
    MixJob<NW, ESC> job;
    job.a = &a;
    int64_t n = a.nq;
    job.n1 = 0;
    if (a.mix_lists) {
        job.n1 = a.route_n ? __ldg(a.route_n) : 0;
        n = job.n1 + __ldg(a.esc_count);
    }
    run_persistent<MixJob<NW, ESC>, SG_WALK_REFILL, SG_MIX_STEPS>(a.counter, n, job);
}

// hole avoidance (boundary_mode 1): the boundary handling needs more registers than the
// default walk, so it gets its own kernel and residency bound
#ifndef SG_HOLE_MINB
#define SG_HOLE_MINB 4
#endif
// walk steps between the hole-avoidance walk's refill checks: one (the boundary handling makes
// the loop body large; the sphere with 8% of its faces removed, 1M queries: 2.41 ms, against
// 4.63 ms with two steps per check)
#ifndef SG_HOLE_STEPS
#define SG_HOLE_STEPS 1
#endif
template <int NW>
__global__ void __launch_bounds__(256, SG_HOLE_MINB) k_walk_hole(FwdArgs a) {
    FwdJob<NW, true, true> job;
    job.a = &a;
    run_persistent<FwdJob<NW, true, true>, SG_WALK_REFILL, SG_HOLE_STEPS>(a.counter, a.nq, job);
}

// ------------------------------------------------------------------ geodesic tracing
// The same walk, with the traced geodesic as an extra output (the by-product named in Sec. 1
// and Sec. 4): every face the walk enters, in order, and the 3-D point where it enters it (the
// start point, then each edge crossing point or, after a vertex hit, the vertex).  Inside a
// face the straightest geodesic is a straight segment, so these points followed by the end
// point are the polyline of the geodesic.
//
// The walk records each entry point in the entered face's own terms -- the fraction along its
// entry edge, or the start barycentrics -- and a second, fully parallel pass turns these into
// 3-D points: computing them during the walk would add two dependent gathers (vertex ids, then
// positions) to every crossing.
struct TraceOut {
    int32_t cap;
    int32_t *face;  // [nq][cap] local face ids
    float *pt;      // [nq][cap][3] entry points, or NULL
    int32_t *len;   // [nq] faces entered (may exceed cap; entries past cap are dropped)
    int staged;     // 1: entries are written 8 at a time with 16-byte stores (cap % 4 == 0,
                    // 16-byte aligned buffers); 0: one entry at a time
};

// Entries of one lane are collected in shared memory and written 8 at a time: a lane's entries
// are contiguous in its query's row, so 8 of them fill whole sectors, where single entries
// written at different times by the lanes of a warp touch a separate sector each.
#define SG_TRACE_STAGE 8
struct TraceStage {
    int face[SG_TRACE_STAGE][256];
    float a[SG_TRACE_STAGE][256];
    int code[SG_TRACE_STAGE][256];
};

template <bool ESC>
struct TraceJob {
    const FwdArgs *a;
    const TraceOut *t;
    Walker w;
    Carry<0> cw;
    int64_t q;
    int n;
    TraceStage *sg;
    // code 0..2: on local edge `code` at fraction a from its first corner; 3: the start point
    // (the second pass reads its barycentrics from the query)
    __device__ __forceinline__ void put(int64_t i, int face, float a, int code) {
        t->face[i] = face;
        if (t->pt) { t->pt[3 * i] = a; t->pt[3 * i + 1] = __int_as_float(code); }
    }
    __device__ __forceinline__ void flush8(int base) {
        const int tid = threadIdx.x;
        const int64_t i = q * t->cap + base;
        int4 *fo = reinterpret_cast<int4 *>(t->face + i);
        fo[0] = make_int4(sg->face[0][tid], sg->face[1][tid], sg->face[2][tid], sg->face[3][tid]);
        fo[1] = make_int4(sg->face[4][tid], sg->face[5][tid], sg->face[6][tid], sg->face[7][tid]);
        if (t->pt) {
            float4 *po = reinterpret_cast<float4 *>(t->pt + 3 * i);
            float a[8], c[8];
            for (int j = 0; j < 8; ++j) { a[j] = sg->a[j][tid]; c[j] = __int_as_float(sg->code[j][tid]); }
            po[0] = make_float4(a[0], c[0], 0.f, a[1]);
            po[1] = make_float4(c[1], 0.f, a[2], c[2]);
            po[2] = make_float4(0.f, a[3], c[3], 0.f);
            po[3] = make_float4(a[4], c[4], 0.f, a[5]);
            po[4] = make_float4(c[5], 0.f, a[6], c[6]);
            po[5] = make_float4(0.f, a[7], c[7], 0.f);
        }
    }
    __device__ __forceinline__ void rec(float a, int code) {
        if (n < t->cap) {
            const int face = w.f - w.foff;
            if (t->staged) {
                const int j = n & (SG_TRACE_STAGE - 1), tid = threadIdx.x;
                sg->face[j][tid] = face; sg->a[j][tid] = a; sg->code[j][tid] = code;
                if (j == SG_TRACE_STAGE - 1) flush8(n - (SG_TRACE_STAGE - 1));
            } else {
                put(q * t->cap + n, face, a, code);
            }
        }
        n++;
    }
    __device__ __forceinline__ bool init(int64_t tk) {
        q = a->perm ? (int64_t)__ldg(a->perm + tk) : tk;
        n = 0;
        const bool live = walker_init<0>(a->P, a->in, q, w, cw);
        if (live && w.Lh > 0.f) rec(0.f, 3);  // Exp_p(0) = p enters no face
        return live;
    }
    __device__ __forceinline__ bool step() {
        const int nc = w.ncross;
        const bool done = walker_step<ESC>(w, a->P);
        if (w.ncross != nc) {
            // entered face h / 3 through its local edge k at fraction px from corner k (in the
            // half-edge mode the walker does not keep w.f up to date)
            if (w.mode == SG_MODE_HALF) w.f = w.h / 3;
            rec(w.px, w.h - 3 * w.f);
        } else if (!done && w.mode >= 3 && w.mode < 6) {
            // a vertex transport left the walker on corner mode-3 of face w.f
            rec(0.f, w.mode - 3);
        }
        return done;
    }
    __device__ __forceinline__ void finish() {
        walker_finish<0>(*a, q, w, cw);
        t->len[q] = n;
        if (t->staged) {  // entries still in the stage
            const int m = min(n, t->cap), rem = m & (SG_TRACE_STAGE - 1), tid = threadIdx.x;
            for (int j = 0; j < rem; ++j) put(q * t->cap + (m - rem) + j, sg->face[j][tid], sg->a[j][tid], sg->code[j][tid]);
        }
    }
};

// Entries of the trace: from the face's own terms to 3-D points, in place.  One warp per query
// (its entries are contiguous, so the lanes read and write them together).
__global__ void __launch_bounds__(256) k_trace_points(int64_t nq, int32_t cap, const int32_t *__restrict__ len,
                                                      const int32_t *__restrict__ path_face, float *pt,
                                                      const int32_t *__restrict__ mesh_id,
                                                      const float *__restrict__ bary,
                                                      const int32_t *__restrict__ face_off, const int4 *__restrict__ fv,
                                                      const float4 *__restrict__ V) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nq; q += nwarps) {
        const int n = min(__ldg(len + q), cap);
        if (n <= 0) continue;
        const int foff = __ldg(face_off + (mesh_id ? __ldg(mesh_id + q) : 0));
        for (int i = lane; i < n; i += 32) {
            const int64_t e = q * cap + i;
            const int4 t3 = __ldg(fv + foff + __ldg(path_face + e));
            float *o = pt + 3 * e;
            const float a = o[0];
            const int code = __float_as_int(o[1]);
            float w0, w1, w2;  // weights of the three corners
            if (code == 3) {
                const float b0 = fmaxf(__ldg(bary + 3 * q), 0.f), b1 = fmaxf(__ldg(bary + 3 * q + 1), 0.f);
                const float b2 = fmaxf(__ldg(bary + 3 * q + 2), 0.f);
                const float rs = 1.f / (b0 + b1 + b2);
                w0 = b0 * rs; w1 = b1 * rs; w2 = b2 * rs;
            } else {
                w0 = code == 0 ? 1.f - a : (code == 2 ? a : 0.f);
                w1 = code == 1 ? 1.f - a : (code == 0 ? a : 0.f);
                w2 = code == 2 ? 1.f - a : (code == 1 ? a : 0.f);
            }
            const float4 x0 = __ldg(V + t3.x), x1 = __ldg(V + t3.y), x2 = __ldg(V + t3.z);
            o[0] = w0 * x0.x + w1 * x1.x + w2 * x2.x;
            o[1] = w0 * x0.y + w1 * x1.y + w2 * x2.y;
            o[2] = w0 * x0.z + w1 * x1.z + w2 * x2.z;
        }
    }
}

template <bool ESC>
__global__ void __launch_bounds__(256, 4) k_trace_persistent(FwdArgs a, TraceOut t) {
    __shared__ TraceStage stage;
    TraceJob<ESC> job;
    job.a = &a;
    job.t = &t;
    job.sg = &stage;
    run_persistent<TraceJob<ESC>, SG_WALK_REFILL, SG_TRACE_STEPS>(a.counter, a.nq, job);
}

// ------------------------------------------------------------------ start-face counting sort
// The length a query walks, as the query orders see it: the given length, else |v| (the ambient
// norm, an upper bound of the projected length).
__device__ __forceinline__ float query_length(const QueryIn &in, int64_t i) {
    if (in.length) return __ldg(in.length + i);
    const float x = __ldg(in.v + 3 * i), y = __ldg(in.v + 3 * i + 1), z = __ldg(in.v + 3 * i + 2);
    return sqrtf(fmaf(x, x, fmaf(y, y, z * z)));
}

// Key of query i: the spatial rank of its start face (its place on its mesh's Z-order curve of
// face centroids, offset by the mesh's first face); nF for an invalid query.  With the automatic
// precision (esc_lmax > 0) the queries longer than esc_lmax l_ref, which the mixed walk takes,
// keep that rank as key and form the permutation's head; the others get nF + the rank, and an
// invalid query 2 nF.
__device__ __forceinline__ int face_key(const QueryIn &in, const int32_t *__restrict__ face_off,
                                        const int32_t *__restrict__ srank, const float *__restrict__ lref,
                                        int32_t nF, float esc_lmax, int64_t i) {
    const int inval = esc_lmax > 0.f ? 2 * nF : nF;
    const int m = in.mesh_id ? __ldg(in.mesh_id + i) : 0;
    if (m < 0 || m >= in.n_mesh) return inval;
    const int lo = __ldg(face_off + m), hi = __ldg(face_off + m + 1);
    const int f = __ldg(in.face + i);
    if (f < 0 || f >= hi - lo) return inval;
    int key = __ldg(srank + lo + f);  // in [lo, hi): the face's place on the mesh's Z-order curve
    if (esc_lmax > 0.f && !(query_length(in, i) > esc_lmax * __ldg(lref + m))) key += nF;
    return key;
}

__global__ void k_sort_keys_hist(int64_t nq, QueryIn in, const int32_t *__restrict__ face_off,
                                 const int32_t *__restrict__ srank, const float *__restrict__ lref, int32_t nF,
                                 float esc_lmax, int32_t *__restrict__ counts) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + face_key(in, face_off, srank, lref, nF, esc_lmax, i), 1);
}

// after the scatter offsets[k] is the end of bucket k (with the automatic precision offsets[nF - 1]
// is the number of routed queries at the head)
__global__ void k_sort_scatter(int64_t nq, QueryIn in, const int32_t *__restrict__ face_off,
                               const int32_t *__restrict__ srank, const float *__restrict__ lref, int32_t nF,
                               float esc_lmax, int32_t *__restrict__ offsets, int32_t *__restrict__ perm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        const int pos = atomicAdd(offsets + face_key(in, face_off, srank, lref, nF, esc_lmax, i), 1);
        perm[pos] = (int32_t)i;
    }
}

// ------------------------------------------------------------------ length order
// Walks of similar length end together, so a warp whose lanes hold them waits less with idle
// lanes before it refills.  Key: an eighth of an octave of L / l_ref per bucket, longest walks
// first (the short ones then fill the tail of the queue); invalid queries last.  L is the given
// length, else |v| (its ambient norm: a key, not the walked length).  With the automatic precision
// (esc_lmax > 0) bucket 0 holds the queries longer than esc_lmax l_ref, which the mixed walk
// takes: the permutation's head; the length buckets then start at 1.
__device__ __forceinline__ int length_key(const QueryIn &in, const float *__restrict__ lref, int64_t i,
                                          float esc_lmax) {
    const int m = in.mesh_id ? __ldg(in.mesh_id + i) : 0;
    if (m < 0 || m >= in.n_mesh) return SG_LBUCKETS - 1;
    const float L = query_length(in, i);
    const float lr = __ldg(lref + m);
    if (!(L > 0.f) || !(L <= 3.0e38f) || !(lr > 0.f)) return SG_LBUCKETS - 1;
    if (esc_lmax > 0.f && L > esc_lmax * lr) return 0;
    const float t = fminf(fmaxf(fmaf(8.f, __log2f(L / lr), 128.f), 0.f), (float)(SG_LBUCKETS - 2));
    const int k = SG_LBUCKETS - 2 - (int)t;
    return esc_lmax > 0.f ? max(k, 1) : k;
}

__global__ void __launch_bounds__(256) k_lorder_hist(int64_t nq, QueryIn in, const float *__restrict__ lref,
                                                     float esc_lmax, uint8_t *__restrict__ keys,
                                                     int32_t *__restrict__ counts) {
    __shared__ int32_t h[SG_LBUCKETS];
    for (int b = threadIdx.x; b < SG_LBUCKETS; b += blockDim.x) h[b] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = length_key(in, lref, i, esc_lmax);
        keys[i] = (uint8_t)k;
        atomicAdd(&h[k], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < SG_LBUCKETS; b += blockDim.x)
        if (h[b]) atomicAdd(counts + b, h[b]);
}

// counts[0, 256) the bucket totals, counts[256, 512) zeroed cursors.  Each block takes chunks of
// 256 x SG_LCHUNK queries, ranks them within the chunk per bucket in shared memory, reserves one
// range per (chunk, bucket) with a single global atomic and writes the permutation.
#define SG_LCHUNK 8
__global__ void __launch_bounds__(256) k_lorder_scatter(int64_t nq, const uint8_t *__restrict__ keys,
                                                        int32_t *__restrict__ counts, int32_t *__restrict__ perm) {
    __shared__ int32_t start[SG_LBUCKETS], lh[SG_LBUCKETS], base[SG_LBUCKETS];
    if (threadIdx.x < 32) {  // exclusive scan of the totals: 8 buckets per lane
        const int lane = threadIdx.x;
        int32_t v[SG_LBUCKETS / 32], sum = 0;
        for (int j = 0; j < SG_LBUCKETS / 32; ++j) { v[j] = counts[lane * (SG_LBUCKETS / 32) + j]; sum += v[j]; }
        int32_t x = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        int32_t e = x - sum;
        for (int j = 0; j < SG_LBUCKETS / 32; ++j) { start[lane * (SG_LBUCKETS / 32) + j] = e; e += v[j]; }
    }
    const int64_t chunk = (int64_t)blockDim.x * SG_LCHUNK;
    for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < nq; c0 += (int64_t)gridDim.x * chunk) {
        for (int b = threadIdx.x; b < SG_LBUCKETS; b += blockDim.x) lh[b] = 0;
        __syncthreads();
        int k[SG_LCHUNK], r[SG_LCHUNK];
#pragma unroll
        for (int j = 0; j < SG_LCHUNK; ++j) {
            const int64_t i = c0 + (int64_t)j * blockDim.x + threadIdx.x;
            k[j] = i < nq ? (int)keys[i] : 0;
            r[j] = i < nq ? atomicAdd(&lh[k[j]], 1) : 0;
        }
        __syncthreads();
        for (int b = threadIdx.x; b < SG_LBUCKETS; b += blockDim.x)
            if (lh[b]) base[b] = start[b] + atomicAdd(counts + SG_LBUCKETS + b, lh[b]);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < SG_LCHUNK; ++j) {
            const int64_t i = c0 + (int64_t)j * blockDim.x + threadIdx.x;
            if (i < nq) perm[base[k[j]] + r[j]] = (int32_t)i;
        }
        __syncthreads();
    }
}

#define SCAN_BLOCK 1024
#define SCAN_ITEMS 4
#define SCAN_TILE (SCAN_BLOCK * SCAN_ITEMS)

// block-wide exclusive scan of one tile in place; writes the tile total
__device__ int block_scan_tile(int32_t *data, int64_t n, int64_t base, int32_t carry_in) {
    __shared__ int32_t warp_sums[SCAN_BLOCK / 32];
    int tid = threadIdx.x;
    int32_t v[SCAN_ITEMS];
    int32_t local = 0;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)tid * SCAN_ITEMS + k;
        v[k] = i < n ? data[i] : 0;
        local += v[k];
    }
    int lane = tid & 31, wid = tid >> 5;
    int32_t x = local;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t s = lane < SCAN_BLOCK / 32 ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_BLOCK / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    int32_t excl = x - local + (wid > 0 ? warp_sums[wid - 1] : 0) + carry_in;
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int64_t i = base + (int64_t)tid * SCAN_ITEMS + k;
        if (i < n) data[i] = excl;
        excl += v[k];
    }
    int32_t total = warp_sums[SCAN_BLOCK / 32 - 1];
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_tiles(int32_t *data, int64_t n, int32_t *tile_sums) {
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int32_t tot = block_scan_tile(data, n, base, 0);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sums(int32_t *sums, int64_t n) {
    int32_t carry = 0;
    for (int64_t base = 0; base < n; base += SCAN_TILE) carry += block_scan_tile(sums, n, base, carry);
}

__global__ void k_scan_add(int32_t *data, int64_t n, const int32_t *tile_sums) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) data[i] += tile_sums[i / SCAN_TILE];
}

// ------------------------------------------------------------------ host helpers
namespace {

thread_local char g_err[256];

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct WsLayout {
    size_t counter, counts, sums, keys, perm, esc, lkeys, lcounts, total;
};

// The 64-byte counter block (zeroed by every call): [0] the walk's tickets, [1] the mixed walk's
// tickets, [2] the escalation list's length.
#define SG_CTR_MIXED 1
#define SG_CTR_ESC 2

// sort: 0 none, 1 by (mesh, start face), 2 by walk length; esc: room for the escalation list of
// the automatic precision; order: room to build the length order for a caller's order buffer
// (sg_opts.order) when the walk takes another order
WsLayout ws_layout(int64_t nF, int64_t nq, int sort, bool esc = false, bool order = false) {
    WsLayout L{};
    size_t o = 0;
    L.counter = o; o = align_up(o + 64, 256);
    if (esc) { L.esc = o; o = align_up(o + sizeof(int32_t) * std::max<int64_t>(nq, 1), 256); }
    if (sort == 1) {
        int64_t nk = esc ? 2 * nF + 1 : nF + 1;
        int64_t ntiles = (nk + SCAN_TILE - 1) / SCAN_TILE;
        L.counts = o; o = align_up(o + sizeof(int32_t) * nk, 256);
        L.sums = o; o = align_up(o + sizeof(int32_t) * ntiles, 256);
        L.perm = o; o = align_up(o + sizeof(int32_t) * std::max<int64_t>(nq, 1), 256);
    } else if (sort == 2) {
        L.counts = o; o = align_up(o + sizeof(int32_t) * 2 * SG_LBUCKETS, 256);
        L.keys = o; o = align_up(o + (size_t)std::max<int64_t>(nq, 1), 256);
        L.perm = o; o = align_up(o + sizeof(int32_t) * std::max<int64_t>(nq, 1), 256);
    }
    if (order && sort != 2) {  // the length order written into a caller's order buffer
        L.lcounts = o; o = align_up(o + sizeof(int32_t) * 2 * SG_LBUCKETS, 256);
        L.lkeys = o; o = align_up(o + (size_t)std::max<int64_t>(nq, 1), 256);
    }
    L.total = o;
    return L;
}

// The automatic choice (sort < 0), for batches of at least SG_SORT_MIN_BATCH queries: by start
// face on meshes whose walk records (128 B per face: face and half-edge records) exceed half of
// L2 (a 4.2M-face heightfield walks 12% faster so ordered), else by walk length.  Records that
// stay in L2 are gathered as fast in any order (icosphere s6 and torus walks are as fast or
// faster without the start-face order), but lanes holding walks of similar length idle less.
#define SG_SORT_MIN_BATCH 65536
// below this many queries the automatic kernel choice walks one thread per query
#define SG_SMALL_BATCH 65536
// The automatic precision (sg_opts.precision = 0) keeps a query in the FP32 walk while its walk
// stays within the range where the FP32 walk's face sequences were measured equal to the
// double-precision ones: below 256 crossings, no difference in 3.9M walks over icospheres, a
// torus and heightfields with and without slivers (differences appear from 256 crossings, about
// 3e-5 of the walks there, and grow with the crossing count).  A query whose length exceeds 96
// l_ref (about 210-255 crossings on these meshes) goes to the mixed walk at the start; one whose
// walk reaches 256 crossings is restarted there.
#define SG_AUTO_FP32_LREF 96.0f
#define SG_AUTO_FP32_CROSSINGS 256

int l2_bytes() {
    static int cached = -1;
    if (cached < 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev) != cudaSuccess) { cudaGetLastError(); v = 0; }
        cached = v > 0 ? v : (64 << 20);
    }
    return cached;
}

sg_opts resolve(const sg_opts *o, int64_t nq, int64_t nF) {
    sg_opts r;
    sg_opts_default(&r);
    if (o) r = *o;
    if (r.max_steps <= 0) r.max_steps = 1 << 20;
    if (r.block <= 0) r.block = 256;
    if (r.precision < 0) r.precision = 0;  // 0: automatic (FP32, long walks in the mixed walk)
    if (r.tau_near <= 0.f) r.tau_near = 1e-4f;
    if (r.tau_snap <= 0.f) r.tau_snap = fminf(r.precision >= 48 ? 1e-12f : 1e-6f, r.tau_near);
    if (r.kernel == SG_KERNEL_AUTO) r.kernel = SG_KERNEL_PERSISTENT;
    if (r.sort < 0)
        r.sort = nq < SG_SORT_MIN_BATCH ? 0 : (128 * nF > (int64_t)l2_bytes() / 2 ? 1 : 2);
    if (r.kernel == SG_KERNEL_PLAIN) { r.sort = 0; r.fp64_escalate = 0; }
    return r;
}

template <int NW, bool AUTO = false>
cudaError_t launch_walk(const FwdArgs &a, const sg_opts &o, cudaStream_t s) {
    if (o.kernel == SG_KERNEL_PLAIN) {
        const int64_t per_thread = std::max(o.queries_per_thread, 1);
        int64_t grid = std::max<int64_t>((a.nq + o.block * per_thread - 1) / (o.block * per_thread), 1);
        if (o.fp64_escalate) k_walk_plain<NW, true, AUTO><<<(unsigned)grid, o.block, 0, s>>>(a);
        else k_walk_plain<NW, false, AUTO><<<(unsigned)grid, o.block, 0, s>>>(a);
        return cudaGetLastError();
    }
    int dev = 0, sms = 0, per = o.blocks_per_sm;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per <= 0) {
        if (o.fp64_escalate)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_walk_persistent<NW, true>, o.block, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_walk_persistent<NW, false>, o.block, 0);
        per = std::max(per, 1);
    }
    int64_t need = (a.nq + o.block - 1) / o.block;
    if (o.boundary_mode) {  // hole avoidance: its own instantiation, FP64 classification
        if (o.blocks_per_sm <= 0) {
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_walk_hole<NW>, o.block, 0);
            per = std::max(per, 1);
        }
        int64_t grid = std::min<int64_t>((int64_t)sms * per, std::max<int64_t>(need, 1));
        k_walk_hole<NW><<<(unsigned)grid, o.block, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (o.queries_per_thread > 0)  // about that many queries per thread: fewer resident blocks
        per = (int)std::min<int64_t>(per, std::max<int64_t>(
                  (a.nq + (int64_t)o.queries_per_thread * sms * o.block - 1) / ((int64_t)o.queries_per_thread * sms * o.block), 1));
    int64_t grid = std::min<int64_t>((int64_t)sms * per, std::max<int64_t>(need, 1));
    if (o.fp64_escalate)
        k_walk_persistent<NW, true, AUTO><<<(unsigned)grid, o.block, 0, s>>>(a);
    else
        k_walk_persistent<NW, false, AUTO><<<(unsigned)grid, o.block, 0, s>>>(a);
    return cudaGetLastError();
}

template <int NW>
cudaError_t launch_mixed(const FwdArgs &a, const sg_opts &o, cudaStream_t s) {
    int dev = 0, sms = 0, per = o.blocks_per_sm;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per <= 0) {
        if (o.fp64_escalate) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_walk_mixed<NW, true>, 256, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_walk_mixed<NW, false>, 256, 0);
        per = std::max(per, 1);
    }
    const int64_t grid = std::min<int64_t>((int64_t)sms * per, std::max<int64_t>((a.nq + 255) / 256, 1));
    if (o.fp64_escalate) k_walk_mixed<NW, true><<<(unsigned)grid, 256, 0, s>>>(a);
    else k_walk_mixed<NW, false><<<(unsigned)grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_mixed_nw(const FwdArgs &a, int n_w, const sg_opts &o, cudaStream_t s) {
    switch (n_w) {
        case 0: return launch_mixed<0>(a, o, s);
        case 1: return launch_mixed<1>(a, o, s);
        case 2: return launch_mixed<2>(a, o, s);
        case 3: return launch_mixed<3>(a, o, s);
        default: return launch_mixed<4>(a, o, s);
    }
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

void sg_opts_default(sg_opts *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->max_steps = 1 << 20;
    o->kernel = SG_KERNEL_AUTO;
    o->sort = -1;
    o->block = 256;
    o->blocks_per_sm = 0;
    o->fp64_escalate = 1;
    o->tau_near = 1e-4f;
    o->tau_snap = 0.f;
    o->workspace = nullptr;
    o->workspace_bytes = 0;
    o->prof_events = nullptr;
    o->boundary_mode = 0;
    o->precision = 0;
    o->order = nullptr;
}

const char *sg_status_string(sg_status s) {
    switch (s) {
        case SG_OK: return "ok";
        case SG_ERR_INVALID_ARG: return "invalid argument";
        case SG_ERR_NONMANIFOLD: return "non-manifold mesh";
        case SG_ERR_DEGENERATE: return "degenerate face";
        case SG_ERR_CUDA: return "CUDA error";
        case SG_ERR_OOM: return "out of device memory";
        case SG_ERR_UNSUPPORTED: return "unsupported option";
    }
    return "unknown";
}

const char *sg_version(void) { return "sgeo 0.1 (sm_103a)"; }

}  // extern "C"

namespace {

// true when p is CUDA device (or managed) memory; host pointers, registered or not, are false
bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// host copy of `n` elements of p when p is device memory (the builder runs on the host)
template <class T>
const T *host_view(const T *p, size_t n, std::vector<T> &buf, bool *err) {
    if (!p || !on_device(p)) return p;
    buf.resize(std::max<size_t>(n, 1));
    if (cudaMemcpy(buf.data(), p, sizeof(T) * n, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        *err = true;
    }
    return buf.data();
}

}  // namespace

extern "C" {

sg_status sg_mesh_create_batched(const float *V, const int64_t *v_off, const int32_t *F, const int64_t *f_off,
                                 int32_t n_mesh, sg_mesh **out) {
    if (!out) return SG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!V || !v_off || !F || !f_off || n_mesh <= 0) return SG_ERR_INVALID_ARG;
    // any of the four arrays may live in device memory: copy those to the host first
    bool err = false;
    std::vector<int64_t> vo_buf, fo_buf;
    std::vector<float> v_buf;
    std::vector<int32_t> f_buf;
    v_off = host_view(v_off, (size_t)n_mesh + 1, vo_buf, &err);
    f_off = host_view(f_off, (size_t)n_mesh + 1, fo_buf, &err);
    if (err) return SG_ERR_CUDA;
    if (v_off[n_mesh] <= 0 || f_off[n_mesh] <= 0) return SG_ERR_INVALID_ARG;
    V = host_view(V, 3 * (size_t)v_off[n_mesh], v_buf, &err);
    F = host_view(F, 3 * (size_t)f_off[n_mesh], f_buf, &err);
    if (err) return SG_ERR_CUDA;
    sg_host_mesh H;
    sg_status st = sg_build_host_mesh(V, v_off, F, f_off, n_mesh, &H);
    if (st != SG_OK) return st;
    sg_mesh *m = new (std::nothrow) sg_mesh();
    if (!m) return SG_ERR_OOM;
    m->nV = v_off[n_mesh];
    m->nF = f_off[n_mesh];
    m->n_mesh = n_mesh;
    cudaGetDevice(&m->device);
    m->face_off = H.face_off64;
    m->nE = (int64_t)H.edges.size();
    if (H.edges.empty()) H.edges.push_back(int2{0, 0});
    m->vert_off = H.vert_off64;
    m->lref = H.lref64;
    auto up = [&](void **dst, const void *src, size_t bytes) -> bool {
        if (cudaMalloc(dst, bytes) != cudaSuccess) return false;
        m->device_bytes += (int64_t)bytes;
        return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    };
    bool ok = up((void **)&m->d_rec, H.rec.data(), sizeof(int4) * H.rec.size()) &&
              up((void **)&m->d_fv, H.fv.data(), sizeof(int4) * H.fv.size()) &&
              up((void **)&m->d_frm, H.frm.data(), sizeof(float4) * H.frm.size()) &&
              up((void **)&m->d_half, H.half.data(), sizeof(int4) * H.half.size()) &&
              up((void **)&m->d_edges, H.edges.data(), sizeof(int2) * std::max<size_t>(H.edges.size(), 1)) &&
              up((void **)&m->d_srank, H.srank.data(), sizeof(int32_t) * H.srank.size()) &&
              up((void **)&m->d_V, H.V.data(), sizeof(float4) * H.V.size()) &&
              up((void **)&m->d_face_off, H.face_off.data(), sizeof(int32_t) * H.face_off.size()) &&
              up((void **)&m->d_lref, H.lref.data(), sizeof(float) * H.lref.size());
    if (!ok) {
        cudaGetLastError();
        sg_mesh_destroy(m);
        return SG_ERR_OOM;
    }
    // The FP64 geometry and double-float half-edge records of the mixed, double-float and FP64
    // walks (192 B per face, 8 B per vertex), built now so that no walk call has to allocate.
    sg_status st64 = sg_geom64_prepare(m, 0, true);
    if (st64 == SG_OK && cudaStreamSynchronize(0) != cudaSuccess) st64 = SG_ERR_CUDA;
    if (st64 != SG_OK) {
        cudaGetLastError();
        sg_mesh_destroy(m);
        return st64;
    }
    *out = m;
    return SG_OK;
}

sg_status sg_mesh_create(const float *V, int64_t nV, const int32_t *F, int64_t nF, sg_mesh **out) {
    if (nV <= 0 || nF <= 0) return SG_ERR_INVALID_ARG;
    int64_t vo[2] = {0, nV}, fo[2] = {0, nF};
    return sg_mesh_create_batched(V, vo, F, fo, 1, out);
}

sg_status sg_mesh_destroy(sg_mesh *m) {
    if (!m) return SG_OK;
    cudaFree(m->d_rec);
    cudaFree(m->d_fv);
    cudaFree(m->d_frm);
    cudaFree(m->d_half);
    cudaFree(m->d_edges);
    cudaFree(m->d_srank);
    cudaFree(m->d_V);
    cudaFree(m->d_face_off);
    cudaFree(m->d_lref);
    cudaFree(m->d_theta);
    cudaFree(m->d_lsum);
    cudaFree(m->d_ecount);
    cudaFree(m->d_ndegen);
    cudaFree(m->d_rec64);
    cudaFree(m->d_frm64);
    cudaFree(m->d_th64);
    cudaFree(m->d_half48);
    delete m;
    return SG_OK;
}

sg_status sg_mesh_get_info(const sg_mesh *m, sg_mesh_info *info) {
    if (!m || !info) return SG_ERR_INVALID_ARG;
    info->n_vertices = m->nV;
    info->n_faces = m->nF;
    info->n_mesh = m->n_mesh;
    info->record_bytes = 32 + 3 * 32;
    info->device_bytes = m->device_bytes;
    info->l_ref_mean = m->lref.empty() ? 0.0 : m->lref[0];
    info->n_degenerate = 0;
    if (m->updated) {  // geometry re-derived on the device: read back the current values
        std::vector<int> nd(m->n_mesh);
        double ls = 0.0;
        unsigned long long ne = 0;
        if (cudaMemcpy(nd.data(), m->d_ndegen, sizeof(int) * nd.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&ls, m->d_lsum, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&ne, m->d_ecount, sizeof(ne), cudaMemcpyDeviceToHost) != cudaSuccess)
            return SG_ERR_CUDA;
        for (int x : nd) info->n_degenerate += x;
        info->l_ref_mean = ne ? ls / (double)ne : 0.0;
    }
    return SG_OK;
}

sg_status sg_exp_map_workspace_size(const sg_mesh *m, int64_t nq, const sg_opts *o, size_t *bytes) {
    if (!m || !bytes || nq < 0) return SG_ERR_INVALID_ARG;
    sg_opts r = resolve(o, nq, m->nF);
    if (r.sort < 0 || r.sort > 2) return SG_ERR_INVALID_ARG;
    *bytes = ws_layout(m->nF, nq, r.kernel == SG_KERNEL_PERSISTENT ? r.sort : 0,
                       r.precision == 0 && r.boundary_mode == 0, r.order != nullptr).total;
    return SG_OK;
}

}  // extern "C"

namespace {

// Fills the walk parameters and query inputs shared by the forward entry points.
FwdArgs fwd_args(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face, const float *bary,
                 const float *v, const float *length, const float *w, const sg_opts &r) {
    FwdArgs a{};
    a.P.rec = m->d_rec; a.P.fv = m->d_fv; a.P.frm = m->d_frm; a.P.half = m->d_half; a.P.V = m->d_V; a.P.face_off = m->d_face_off; a.P.lref = m->d_lref;
    a.P.max_steps = r.max_steps; a.P.tau_near = r.tau_near; a.P.tau_snap = r.tau_snap;
    a.P.half48 = m->d_half48; a.P.frm64 = m->d_frm64;
    a.nq = nq; a.in.n_mesh = m->n_mesh; a.nF_total = (int32_t)m->nF;
    a.in.mesh_id = mesh_id; a.in.face = face; a.in.bary = bary; a.in.v = v; a.in.length = length; a.in.w = w;
    return a;
}

// Work queue of the persistent kernels: the ticket counter and, when sorting, the permutation
// of queries by (mesh, start face).  Uses the caller's workspace or stream-ordered scratch
// (*own_ws = the pointer to free after the walk).
sg_status prepare_queue(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face, const sg_opts &r,
                        int sort, cudaStream_t s, FwdArgs &a, void **own_ws, bool esc = false) {
    *own_ws = nullptr;
    WsLayout L = ws_layout(m->nF, nq, sort, esc, r.order != nullptr);
    void *ws = nullptr;
    if (r.workspace) {
        if (r.workspace_bytes < L.total) return SG_ERR_OOM;
        ws = r.workspace;
    } else {
        if (cudaMallocAsync(&ws, L.total, s) != cudaSuccess) { cudaGetLastError(); return SG_ERR_OOM; }
        *own_ws = ws;
    }
    char *base = (char *)ws;
    a.counter = (int32_t *)(base + L.counter);
    if (cudaMemsetAsync(a.counter, 0, 64, s) != cudaSuccess) return SG_ERR_CUDA;
    if (esc) {
        a.esc_list = (int32_t *)(base + L.esc);
        a.esc_count = a.counter + SG_CTR_ESC;
    }
    // with the automatic precision the orders route the long queries to the mixed walk (the
    // length order's head, the start-face order's tail)
    const float lmax = esc ? SG_AUTO_FP32_LREF : 0.f;
    // A caller's order buffer (sg_opts.order) receives the length order: the queue's own when it
    // takes the queries in that order, else one built for the buffer after the queue's
    int32_t *perm = (r.order && sort == 2) ? r.order : (int32_t *)(base + L.perm);
    if (sort == 2) {
        int32_t *counts = (int32_t *)(base + L.counts);
        sg_length_order(m, a.in, nq, (uint8_t *)(base + L.keys), counts, perm, s, lmax);
        a.perm = perm;
        if (esc) a.route_n = counts;  // bucket 0: counts[0] queries
    } else if (sort == 1) {
        int32_t *counts = (int32_t *)(base + L.counts);
        int32_t *sums = (int32_t *)(base + L.sums);
        int64_t nk = esc ? 2 * m->nF + 1 : m->nF + 1;
        int64_t ntiles = (nk + SCAN_TILE - 1) / SCAN_TILE;
        cudaMemsetAsync(counts, 0, sizeof(int32_t) * nk, s);
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        int g = (int)std::min<int64_t>((nq + 255) / 256, (int64_t)sms * 8);
        k_sort_keys_hist<<<g, 256, 0, s>>>(nq, a.in, m->d_face_off, m->d_srank, m->d_lref, (int32_t)m->nF, lmax, counts);
        k_scan_tiles<<<(unsigned)ntiles, SCAN_BLOCK, 0, s>>>(counts, nk, sums);
        k_scan_sums<<<1, SCAN_BLOCK, 0, s>>>(sums, ntiles);
        k_scan_add<<<(unsigned)((nk + 255) / 256), 256, 0, s>>>(counts, nk, sums);
        k_sort_scatter<<<g, 256, 0, s>>>(nq, a.in, m->d_face_off, m->d_srank, m->d_lref, (int32_t)m->nF, lmax, counts,
                                         perm);
        a.perm = perm;
        if (esc) a.route_n = counts + m->nF - 1;  // the head: up to the end of bucket nF - 1
    }
    // the FP32 walk starts its tickets after the routed head
    if (a.route_n && cudaMemcpyAsync(a.counter, a.route_n, sizeof(int32_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return SG_ERR_CUDA;
    if (r.order && sort != 2)
        sg_length_order(m, a.in, nq, (uint8_t *)(base + L.lkeys), (int32_t *)(base + L.lcounts), r.order, s, 0.f);
    return SG_OK;
}

}  // namespace

void sg_length_order(const sg_mesh *m, const QueryIn &in, int64_t nq, uint8_t *keys, int32_t *counts, int32_t *perm,
                     cudaStream_t s, float esc_lmax) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaMemsetAsync(counts, 0, sizeof(int32_t) * 2 * SG_LBUCKETS, s);
    const int64_t g1 = std::min<int64_t>((nq + 255) / 256, (int64_t)sms * 4);
    k_lorder_hist<<<(unsigned)std::max<int64_t>(g1, 1), 256, 0, s>>>(nq, in, m->d_lref, esc_lmax, keys, counts);
    const int64_t g2 = std::min<int64_t>((nq + 256 * SG_LCHUNK - 1) / (256 * SG_LCHUNK), (int64_t)sms * 4);
    k_lorder_scatter<<<(unsigned)std::max<int64_t>(g2, 1), 256, 0, s>>>(nq, keys, counts, perm);
}

extern "C" {

sg_status sg_exp_map(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face, const float *bary,
                     const float *v, const float *length, int32_t n_w, const float *w, int32_t *out_face,
                     float *out_bary, float *out_pos, float *out_dir, float *out_w, uint32_t *out_status,
                     int32_t *out_ncross, uint64_t *out_hash, const sg_opts *o, void *stream) {
    if (!m || nq < 0 || n_w < 0 || n_w > SG_MAX_W) return SG_ERR_INVALID_ARG;
    if (nq == 0) return SG_OK;
    if (nq > (int64_t)INT32_MAX - 1024) return SG_ERR_INVALID_ARG;
    if (!face || !bary || !v || !out_face || !out_bary || !out_pos || !out_dir || !out_status) return SG_ERR_INVALID_ARG;
    if (n_w > 0 && !w) return SG_ERR_INVALID_ARG;
    const bool auto_kernel = !o || o->kernel == SG_KERNEL_AUTO;
    sg_opts r = resolve(o, nq, m->nF);
    if (r.tau_snap > r.tau_near) return SG_ERR_INVALID_ARG;  // a snapped vertex lies in the near band
    if (r.kernel != SG_KERNEL_PLAIN && r.kernel != SG_KERNEL_PERSISTENT) return SG_ERR_INVALID_ARG;
    if (r.sort > 2) return SG_ERR_INVALID_ARG;
    if (r.block % 32 != 0 || r.block > 256) return SG_ERR_INVALID_ARG;
    if (r.boundary_mode != 0 && r.boundary_mode != 1) return SG_ERR_INVALID_ARG;
    if (r.precision != 0 && r.precision != 32 && r.precision != 40 && r.precision != 48 && r.precision != 64)
        return SG_ERR_INVALID_ARG;
    // The automatic precision walks in FP32 and hands long walks to the mixed walk; hole avoidance
    // has no mixed walk, so there it is the FP32 walk.
    const bool autoprec = r.precision == 0 && r.boundary_mode == 0;
    if (r.precision == 0) r.precision = 32;
    // A small batch fills the persistent grid once, so no lane would take a second query: the
    // automatic choice walks it one thread per query with the persistent kernel's arithmetic
    // (FP64 classification kept), without the queue and its counter reset.
    if (auto_kernel && nq < SG_SMALL_BATCH && r.precision == 32 && r.boundary_mode == 0 && r.sort == 0)
        r.kernel = SG_KERNEL_PLAIN;
    if (r.boundary_mode && r.kernel == SG_KERNEL_PLAIN) return SG_ERR_UNSUPPORTED;
    if (r.precision >= 40 && (r.boundary_mode || r.kernel == SG_KERNEL_PLAIN)) return SG_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    FwdArgs a = fwd_args(m, nq, mesh_id, face, bary, v, length, w, r);
    a.P.want_hash = out_hash != nullptr;
    a.out_face = out_face; a.out_bary = out_bary; a.out_pos = out_pos; a.out_dir = out_dir;
    a.out_w = out_w; a.out_status = out_status; a.out_ncross = out_ncross; a.out_hash = out_hash;

    const bool persistent = r.kernel == SG_KERNEL_PERSISTENT;
    void *own_ws = nullptr;
    if (persistent || autoprec || r.order) {
        sg_status st = prepare_queue(m, nq, mesh_id, face, r, persistent ? r.sort : 0, s, a, &own_ws, autoprec);
        if (st != SG_OK) {
            if (own_ws) cudaFreeAsync(own_ws, s);
            return st;
        }
    }
    if (r.precision >= 40 || autoprec) {
        // the FP64 geometry and the double-float records (built with the mesh; re-derived here
        // after a vertex update)
        sg_status st = sg_geom64_prepare(const_cast<sg_mesh *>(m), s, r.precision <= 48);
        if (st != SG_OK) {
            if (own_ws) cudaFreeAsync(own_ws, s);
            return st;
        }
    }
    cudaEvent_t *pev = (cudaEvent_t *)r.prof_events;
    if (r.precision == 40) {  // the mixed walk over every query, in the chosen order
        if (pev) cudaEventRecord(pev[0], s);
        cudaError_t e = launch_mixed_nw(a, n_w, r, s);
        if (pev) cudaEventRecord(pev[1], s);
        if (own_ws) cudaFreeAsync(own_ws, s);
        return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
    }
    if (r.precision >= 40) {
        SgFwdIO io{a.in, nq, out_face, out_bary, out_pos, out_dir, out_w, out_status, out_ncross, out_hash, a.perm,
                   a.counter};
        if (pev) cudaEventRecord(pev[0], s);
        cudaError_t e = sg_launch_walk64(m, io, n_w, r, s);
        if (pev) cudaEventRecord(pev[1], s);
        if (own_ws) cudaFreeAsync(own_ws, s);
        return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
    }
    if (autoprec) {
        a.esc_lmax = SG_AUTO_FP32_LREF;
        // the FP32 walk's step cap becomes the crossing budget; the caller's cap, if lower, stays
        // final (esc_ncross = 0: nothing to hand on)
        a.esc_ncross = r.max_steps > SG_AUTO_FP32_CROSSINGS ? SG_AUTO_FP32_CROSSINGS : 0;
        a.P.max_steps = std::min(r.max_steps, SG_AUTO_FP32_CROSSINGS);
    }
    if (pev) cudaEventRecord(pev[0], s);
    cudaError_t e;
    switch (n_w) {
        case 0: e = autoprec ? launch_walk<0, true>(a, r, s) : launch_walk<0>(a, r, s); break;
        case 1: e = autoprec ? launch_walk<1, true>(a, r, s) : launch_walk<1>(a, r, s); break;
        case 2: e = autoprec ? launch_walk<2, true>(a, r, s) : launch_walk<2>(a, r, s); break;
        case 3: e = autoprec ? launch_walk<3, true>(a, r, s) : launch_walk<3>(a, r, s); break;
        default: e = autoprec ? launch_walk<4, true>(a, r, s) : launch_walk<4>(a, r, s); break;
    }
    if (e == cudaSuccess && autoprec) {
        // the mixed walk takes the queries the order routed to it (in that order), then those the
        // FP32 walk handed on at its crossing budget; its grid reads the lists' lengths from
        // device memory (no host synchronisation)
        FwdArgs am = a;
        am.counter = a.counter + SG_CTR_MIXED;
        am.mix_lists = 1;
        am.P.max_steps = r.max_steps;  // the caller's cap (the FP32 walk's was its crossing budget)
        e = launch_mixed_nw(am, n_w, r, s);
    }
    if (pev) cudaEventRecord(pev[1], s);
    if (own_ws) cudaFreeAsync(own_ws, s);
    if (e != cudaSuccess) {
        std::snprintf(g_err, sizeof g_err, "%s", cudaGetErrorString(e));
        return SG_ERR_CUDA;
    }
    return SG_OK;
}

sg_status sg_exp_map_trace(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face,
                           const float *bary, const float *v, const float *length, int32_t path_cap,
                           int32_t *out_path_face, float *out_path_pt, int32_t *out_path_len, int32_t *out_face,
                           float *out_bary, float *out_pos, float *out_dir, uint32_t *out_status,
                           int32_t *out_ncross, uint64_t *out_hash, const sg_opts *o, void *stream) {
    if (!m || nq < 0 || path_cap < 0) return SG_ERR_INVALID_ARG;
    if (nq == 0) return SG_OK;
    if (nq > (int64_t)INT32_MAX - 1024) return SG_ERR_INVALID_ARG;
    if (!face || !bary || !v || !out_face || !out_bary || !out_pos || !out_dir || !out_status || !out_path_len)
        return SG_ERR_INVALID_ARG;
    if (path_cap > 0 && !out_path_face) return SG_ERR_INVALID_ARG;
    sg_opts r = resolve(o, nq, m->nF);
    if (r.tau_snap > r.tau_near) return SG_ERR_INVALID_ARG;
    if (r.boundary_mode || r.precision >= 40) return SG_ERR_UNSUPPORTED;
    if (r.sort > 2) return SG_ERR_INVALID_ARG;
    if (r.block % 32 != 0 || r.block > 256) return SG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    FwdArgs a = fwd_args(m, nq, mesh_id, face, bary, v, length, nullptr, r);
    a.P.want_hash = out_hash != nullptr;
    a.out_face = out_face; a.out_bary = out_bary; a.out_pos = out_pos; a.out_dir = out_dir;
    a.out_w = nullptr; a.out_status = out_status; a.out_ncross = out_ncross; a.out_hash = out_hash;
    TraceOut t{path_cap, out_path_face, path_cap > 0 ? out_path_pt : nullptr, out_path_len, 0};
    t.staged = path_cap % 4 == 0 && ((uintptr_t)out_path_face % 16) == 0 &&
               (!t.pt || ((uintptr_t)t.pt % 16) == 0);
    void *own_ws = nullptr;
    sg_status st = prepare_queue(m, nq, mesh_id, face, r, r.kernel != SG_KERNEL_PLAIN ? r.sort : 0, s, a, &own_ws);
    if (st != SG_OK) {
        if (own_ws) cudaFreeAsync(own_ws, s);
        return st;
    }
    int dev = 0, sms = 0, per = r.blocks_per_sm;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool esc = r.fp64_escalate && r.kernel != SG_KERNEL_PLAIN;
    if (per <= 0) {
        if (esc) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace_persistent<true>, r.block, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace_persistent<false>, r.block, 0);
        per = std::max(per, 1);
    }
    int64_t grid = std::min<int64_t>((int64_t)sms * per, std::max<int64_t>((nq + r.block - 1) / r.block, 1));
    if (esc) k_trace_persistent<true><<<(unsigned)grid, r.block, 0, s>>>(a, t);
    else k_trace_persistent<false><<<(unsigned)grid, r.block, 0, s>>>(a, t);
    if (t.pt) {
        const int64_t blocks = std::min<int64_t>((nq + 7) / 8, (int64_t)sms * 16);  // 8 warps (queries) per block
        k_trace_points<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(nq, path_cap, out_path_len, out_path_face,
                                                                              t.pt, mesh_id, bary, m->d_face_off,
                                                                              m->d_fv, m->d_V);
    }
    cudaError_t e = cudaGetLastError();
    if (own_ws) cudaFreeAsync(own_ws, s);
    if (e != cudaSuccess) {
        std::snprintf(g_err, sizeof g_err, "%s", cudaGetErrorString(e));
        return SG_ERR_CUDA;
    }
    return SG_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free variant
// Scratch for sg_exp_map_noalloc: a fixed, file-scope device array (every GPU that loads the
// library holds it until the process exits).  Host code must not use the array's name as a
// device address; the address is looked up once per device with cudaGetSymbolAddress.
#include <mutex>

#define SG_NOALLOC_SCRATCH_BYTES (32u << 20)
#define SG_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_sg_noalloc_scratch[SG_NOALLOC_SCRATCH_BYTES];

namespace {
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[SG_NOALLOC_MAX_DEVICES] = {};
}  // namespace

extern "C" sg_status sg_exp_map_noalloc(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face,
                                        const float *bary, const float *v, const float *length, int32_t n_w,
                                        const float *w, int32_t *out_face, float *out_bary, float *out_pos,
                                        float *out_dir, float *out_w, uint32_t *out_status, int32_t *out_ncross,
                                        uint64_t *out_hash, const sg_opts *o, void *stream) {
    if (!m) return SG_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return SG_ERR_CUDA; }
    if (dev < 0 || dev >= SG_NOALLOC_MAX_DEVICES) return SG_ERR_UNSUPPORTED;
    // the scratch address is per device: it must be the device that holds the mesh records
    if (dev != m->device) return SG_ERR_INVALID_ARG;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_sg_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return SG_ERR_CUDA;
            }
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
    }
    sg_opts r;
    sg_opts_default(&r);
    if (o) r = *o;
    size_t need = 0;
    sg_status st = sg_exp_map_workspace_size(m, nq, &r, &need);
    if (st != SG_OK) return st;
    if (need > SG_NOALLOC_SCRATCH_BYTES) return SG_ERR_OOM;
    // The FP64 geometry and the double-float records are allocated with the mesh (a vertex update
    // only marks them for re-derivation, which launches kernels and allocates nothing).
    if ((r.precision == 0 || r.precision >= 40) && (!m->d_rec64 || (r.precision <= 48 && !m->d_half48)))
        return SG_ERR_UNSUPPORTED;
    r.workspace = scratch;
    r.workspace_bytes = SG_NOALLOC_SCRATCH_BYTES;
    return sg_exp_map(m, nq, mesh_id, face, bary, v, length, n_w, w, out_face, out_bary, out_pos, out_dir, out_w,
                      out_status, out_ncross, out_hash, &r, stream);
}
