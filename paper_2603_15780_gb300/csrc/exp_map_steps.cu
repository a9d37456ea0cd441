// exp_map_steps.cu -- the K-step exponential map of a vector field sampled at the vertices, in one
// persistent launch, and its backward.
//
// The flow-matching application (Sec. 5, Eq. "fmobj") integrates a vector field over the surface by
// K exponential-map steps, x_{k+1} = Exp_{x_k}(h u(x_k)), the field re-evaluated at every
// intermediate point.  Here the field is given by its values U at the mesh vertices and evaluated
// at a point by its barycentric interpolation, u(x) = sum_j b_j U[F[f, j]], the usual piecewise
// linear field of a triangle mesh.  Each step projects h u(x_k) onto the face it starts in, like
// sg_exp_map does with v.
//
// Forward (k_walk_steps): one walker per query runs the K walks back to back.  When a walk ends,
// the walker is already in its end face with the end point in that face's frame; the next step
// interpolates U there, projects it and walks on, without a round trip through memory or a second
// launch.  The per-step start states, end directions and statuses are written for the backward.
//
// Backward (sg_exp_map_steps_backward): the steps' VJPs in reverse order, each the estimator's
// (EP or GFD, sg_exp_map_backward) with the upstream gradient of its end point and end barycentrics,
// then the field's own term (k_steps_field_bwd): with v_k = h sum_j b_kj U_j,
//   grad U_j  += h b_kj grad_v_k,     grad b_kj += h <U_j, grad_v_k>,
// whose sum with the estimator's start-point gradient is the upstream gradient of the previous
// step's end barycentrics.  The walks are recomputed by the estimators (no face sequence is kept).
#include <cuda_runtime.h>

#include <algorithm>

#include "sgeo_internal.h"
#include "walk.cuh"

#define SG_STEPS_MAX 64

namespace {

struct StepsArgs {
    WalkParams P;
    int64_t nq;
    int32_t K;
    float h;
    int32_t n_mesh;
    const int32_t *__restrict__ mesh_id;
    const int32_t *__restrict__ face;
    const float *__restrict__ bary;
    const float *__restrict__ U;  // [nV][3], global vertex ids
    int32_t *out_face;
    float *out_bary, *out_pos, *out_dir;
    uint32_t *out_status;
    // per-step records (all NULL, or all set except step_hash): [K + 1][nq] faces and [K + 1][nq][3]
    // barycentrics of the step starts and the end; [K][nq][3] walked vectors and end directions;
    // [K][nq] statuses and face-sequence hashes
    int32_t *step_face;
    float *step_bary, *step_v, *step_dir;
    uint32_t *step_status;
    uint64_t *step_hash;
    const int32_t *__restrict__ perm;
    int32_t *counter;
};

// barycentrics of the walker's point in its face (face mode: R the face record, p in its frame)
__device__ __forceinline__ void walker_bary(const Walker &w, float &b0, float &b1, float &b2) {
    b2 = w.py / w.R.x2y;
    b1 = (w.px - b2 * w.R.x2x) / w.R.l01;
    b0 = 1.f - b1 - b2;
}

struct StepsJob {
    const StepsArgs *a;
    Walker w;
    int64_t q;
    int k;
    uint32_t st_all;

    // Start step k at the walker's point (face w.f, position in its frame): interpolate the field,
    // scale it by h, project it onto the face plane; returns false for a zero vector (nothing to
    // walk: Exp_p(0) = p).
    __device__ __forceinline__ bool begin_step() {
        const WalkParams &P = a->P;
        float b0, b1, b2;
        walker_bary(w, b0, b1, b2);
        const int4 t = __ldg(P.fv + w.f);
        const float c0 = fmaxf(b0, 0.f), c1 = fmaxf(b1, 0.f), c2 = fmaxf(b2, 0.f);
        const float *U = a->U;
        const float ux = a->h * (c0 * __ldg(U + 3 * t.x) + c1 * __ldg(U + 3 * t.y) + c2 * __ldg(U + 3 * t.z));
        const float uy = a->h * (c0 * __ldg(U + 3 * t.x + 1) + c1 * __ldg(U + 3 * t.y + 1) + c2 * __ldg(U + 3 * t.z + 1));
        const float uz = a->h * (c0 * __ldg(U + 3 * t.x + 2) + c1 * __ldg(U + 3 * t.y + 2) + c2 * __ldg(U + 3 * t.z + 2));
        if (a->step_face) {
            const int64_t i = (int64_t)k * a->nq + q;
            a->step_face[i] = w.f - w.foff;
            a->step_bary[3 * i] = b0; a->step_bary[3 * i + 1] = b1; a->step_bary[3 * i + 2] = b2;
            a->step_v[3 * i] = ux; a->step_v[3 * i + 1] = uy; a->step_v[3 * i + 2] = uz;
        }
        float e1x, e1y, e1z, e2x, e2y, e2z;
        frm_axes(P, w.f, e1x, e1y, e1z, e2x, e2y, e2z);
        const float v1 = ux * e1x + uy * e1y + uz * e1z, v2 = ux * e2x + uy * e2y + uz * e2z;
        const float L = sqrtf(v1 * v1 + v2 * v2);
        w.st = 0; w.steps = 0; w.ncross = 0; w.hash = SG_FNV_OFFSET; w.Ll = 0.f; w.mode = 6;
        if (!(L > 0.f) || !(L <= 3.0e38f)) {
            w.dx = w.dy = 0.f; w.Lh = 0.f;
            if (!(L <= 3.0e38f)) w.st |= SG_ST_INVALID;
            return false;
        }
        w.dx = v1 / L; w.dy = v2 / L;
        w.Lh = L;
        walker_hash(w, w.f, P.want_hash);
        return true;
    }

    // Step k has ended (the walker in its end face): its records, then the next step's start.
    // Returns true when the last step has ended.
    __device__ __forceinline__ bool end_step() {
        st_all |= w.st & ~SG_PARITY_BIT;
        if (a->step_face) {
            const int64_t i = (int64_t)k * a->nq + q;
            float e1x, e1y, e1z, e2x, e2y, e2z;
            frm_axes(a->P, w.f, e1x, e1y, e1z, e2x, e2y, e2z);
            a->step_dir[3 * i] = w.dx * e1x + w.dy * e2x;
            a->step_dir[3 * i + 1] = w.dx * e1y + w.dy * e2y;
            a->step_dir[3 * i + 2] = w.dx * e1z + w.dy * e2z;
            a->step_status[i] = (w.st & ~SG_PARITY_BIT) | ((w.st & SG_PARITY_BIT) ? SG_ST_FLIPPED : 0u);
            if (a->step_hash) a->step_hash[i] = w.hash;
        }
        if (w.st & SG_ST_INVALID) k = a->K - 1;  // nothing further to walk
        while (++k < a->K) {
            if (begin_step()) return false;
            // a zero vector: the step is the identity, recorded as such
            if (a->step_face) {
                const int64_t i = (int64_t)k * a->nq + q;
                a->step_dir[3 * i] = 0.f; a->step_dir[3 * i + 1] = 0.f; a->step_dir[3 * i + 2] = 0.f;
                a->step_status[i] = w.st;
                if (a->step_hash) a->step_hash[i] = w.hash;
            }
            st_all |= w.st;
        }
        return true;
    }

    __device__ __forceinline__ bool init(int64_t t) {
        q = a->perm ? (int64_t)__ldg(a->perm + t) : t;
        k = 0;
        st_all = 0;
        const WalkParams &P = a->P;
        const int m = a->mesh_id ? __ldg(a->mesh_id + q) : 0;
        const int lf = __ldg(a->face + q);
        bool bad = m < 0 || m >= a->n_mesh;
        const int foff = bad ? 0 : __ldg(P.face_off + m);
        const int nfm = bad ? 1 : __ldg(P.face_off + m + 1) - foff;
        bad = bad || lf < 0 || lf >= nfm;
        const float lr = bad ? 1.f : __ldg(P.lref + m);
        bad = bad || !(lr > 0.f);
        w.foff = foff;
        w.f = bad ? foff : foff + lf;
        w.lref = bad ? 1.f : lr;
        w.h = -1;
        w.R = load_rec(P.rec, w.f);
        float b0 = __ldg(a->bary + 3 * q), b1 = __ldg(a->bary + 3 * q + 1), b2 = __ldg(a->bary + 3 * q + 2);
        const float sb = b0 + b1 + b2;
        if (!(fabsf(sb - 1.f) <= 1e-6f) || b0 < -1e-7f || b1 < -1e-7f || b2 < -1e-7f) bad = true;
        if (bad) {
            w.px = w.py = 0.f;
            w.st = SG_ST_INVALID; w.steps = 0; w.ncross = 0; w.hash = SG_FNV_OFFSET;
            w.dx = w.dy = 0.f; w.Lh = 0.f; w.Ll = 0.f; w.mode = 6;
            if (a->step_face) {  // the step's record: the inputs as given, no vector
                a->step_face[q] = lf;
                a->step_bary[3 * q] = b0; a->step_bary[3 * q + 1] = b1; a->step_bary[3 * q + 2] = b2;
                a->step_v[3 * q] = 0.f; a->step_v[3 * q + 1] = 0.f; a->step_v[3 * q + 2] = 0.f;
            }
            end_step();
            return false;
        }
        const float rs = 1.f / sb;
        b1 = fmaxf(b1, 0.f) * rs; b2 = fmaxf(b2, 0.f) * rs;
        w.px = fmaf(b1, w.R.l01, b2 * w.R.x2x);
        w.py = b2 * w.R.x2y;
        if (begin_step()) return true;
        return !end_step();
    }
    // one step of the current walk; true when it has ended (the driver then calls next())
    __device__ __forceinline__ bool step() { return walker_step<true>(w, a->P); }
    // after a walk ended: its records and the next step's start; true when a walk is live again,
    // false when the query's last step has ended
    __device__ __forceinline__ bool next() { return !end_step(); }
    __device__ __forceinline__ void finish() {
        const WalkParams &P = a->P;
        float b0, b1, b2;
        walker_bary(w, b0, b1, b2);
        const Frame3 F = face_frame(P, w.f);
        a->out_face[q] = w.f - w.foff;
        a->out_bary[3 * q] = b0; a->out_bary[3 * q + 1] = b1; a->out_bary[3 * q + 2] = b2;
        a->out_pos[3 * q] = b0 * F.ox + b1 * F.x1x + b2 * F.x2x;
        a->out_pos[3 * q + 1] = b0 * F.oy + b1 * F.x1y + b2 * F.x2y;
        a->out_pos[3 * q + 2] = b0 * F.oz + b1 * F.x1z + b2 * F.x2z;
        a->out_dir[3 * q] = w.dx * F.e1x + w.dy * F.e2x;
        a->out_dir[3 * q + 1] = w.dx * F.e1y + w.dy * F.e2y;
        a->out_dir[3 * q + 2] = w.dx * F.e1z + w.dy * F.e2z;
        a->out_status[q] = st_all;
        if (a->step_face) {
            const int64_t i = (int64_t)a->K * a->nq + q;
            a->step_face[i] = w.f - w.foff;
            a->step_bary[3 * i] = b0; a->step_bary[3 * i + 1] = b1; a->step_bary[3 * i + 2] = b2;
        }
    }
};

// The persistent driver of walk.cuh (run_persistent), extended by the step transitions: a lane
// whose walk ended waits, like a lane waiting for a new query, until enough lanes of its warp are
// idle, and then the waiting lanes start their next steps together (the start interpolates the
// field and reads the face's axes: a chain of dependent loads that lanes taking it one by one
// would serialise over the warp).  Once the queue is empty the waiting lanes go on at once.
#define SG_STEPS_REFILL 12
// walk steps between refill checks (K = 5, 1M queries: one 1.47 ms, two 1.51 ms)
#ifndef SG_KSTEP_STEPS
#define SG_KSTEP_STEPS 1
#endif
__global__ void __launch_bounds__(256, 4) k_walk_steps(StepsArgs a) {
    StepsJob job;
    job.a = &a;
    const unsigned FULL = 0xffffffffu;
    bool live = false, cont = false, pending = false, exhausted = false;
    while (true) {
        const unsigned idle = __ballot_sync(FULL, !live);
        const unsigned waiting = __ballot_sync(FULL, cont);
        if (exhausted && idle == FULL && !waiting) break;
        if (__popc(idle) >= SG_STEPS_REFILL || (exhausted && waiting)) {
            bool dry = false;
            if (!live) {
                if (cont) {
                    cont = false;
                    live = job.next();
                    pending = !live;
                } else if (!exhausted) {
                    if (pending) {
                        job.finish();
                        pending = false;
                    }
                    const int64_t t = fetch_ticket(a.counter);
                    if (t >= a.nq) {
                        dry = true;
                    } else {
                        live = job.init(t);
                        if (!live) job.finish();
                    }
                }
            }
            exhausted = exhausted || __any_sync(FULL, dry);
        }
#pragma unroll
        for (int s = 0; s < SG_KSTEP_STEPS; ++s) {
            if (live && job.step()) {
                live = false;
                cont = true;
            }
        }
        if (exhausted && pending) {
            job.finish();
            pending = false;
        }
    }
}

// The field's term of step k's VJP (see the file comment), one thread per query: gb_next[q] =
// grad_bary[q] + h <U_j, grad_v[q]> (the upstream gradient of step k-1's end barycentrics, or the
// start barycentrics' gradient for k = 0) and grad U_j += h b_kj grad_v[q].
__global__ void __launch_bounds__(256) k_steps_field_bwd(int64_t nq, float h, const int32_t *__restrict__ mesh_id,
                                                         const int32_t *__restrict__ face_off, const int4 *__restrict__ fv,
                                                         const float *__restrict__ U, const int32_t *__restrict__ face_k,
                                                         const float *__restrict__ bary_k, const uint32_t *__restrict__ st_k,
                                                         const float *__restrict__ grad_v, const float *__restrict__ grad_bary,
                                                         float *gb_next, float *grad_U) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    float gb[3] = {grad_bary ? grad_bary[3 * q] : 0.f, grad_bary ? grad_bary[3 * q + 1] : 0.f,
                   grad_bary ? grad_bary[3 * q + 2] : 0.f};
    if (!(__ldg(st_k + q) & SG_ST_INVALID)) {
        const int m = mesh_id ? __ldg(mesh_id + q) : 0;
        const int4 t = __ldg(fv + __ldg(face_off + m) + __ldg(face_k + q));
        const int vj[3] = {t.x, t.y, t.z};
        const float gx = grad_v[3 * q], gy = grad_v[3 * q + 1], gz = grad_v[3 * q + 2];
        for (int j = 0; j < 3; ++j) {
            const float *u = U + 3 * vj[j];
            gb[j] += h * (__ldg(u) * gx + __ldg(u + 1) * gy + __ldg(u + 2) * gz);
            if (grad_U) {
                const float b = fmaxf(__ldg(bary_k + 3 * q + j), 0.f) * h;
                atomicAdd(grad_U + 3 * vj[j], b * gx);
                atomicAdd(grad_U + 3 * vj[j] + 1, b * gy);
                atomicAdd(grad_U + 3 * vj[j] + 2, b * gz);
            }
        }
    }
    gb_next[3 * q] = gb[0]; gb_next[3 * q + 1] = gb[1]; gb_next[3 * q + 2] = gb[2];
}

inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

extern "C" {

sg_status sg_exp_map_steps(const sg_mesh *m, int32_t K, float h, const float *U, int64_t nq, const int32_t *mesh_id,
                           const int32_t *face, const float *bary, int32_t *out_face, float *out_bary, float *out_pos,
                           float *out_dir, uint32_t *out_status, int32_t *step_face, float *step_bary, float *step_v,
                           float *step_dir, uint32_t *step_status, uint64_t *step_hash, const sg_opts *o,
                           void *stream) {
    if (!m || nq < 0 || K < 1 || K > SG_STEPS_MAX || !(h == h)) return SG_ERR_INVALID_ARG;
    if (nq == 0) return SG_OK;
    if (nq > (int64_t)INT32_MAX - 1024 || (int64_t)(K + 1) * nq > (int64_t)INT32_MAX) return SG_ERR_INVALID_ARG;
    if (!U || !face || !bary || !out_face || !out_bary || !out_pos || !out_dir || !out_status) return SG_ERR_INVALID_ARG;
    const bool rec = step_face != nullptr;
    if (rec != (step_bary != nullptr) || rec != (step_v != nullptr) || rec != (step_dir != nullptr) ||
        rec != (step_status != nullptr) || (step_hash && !rec))
        return SG_ERR_INVALID_ARG;
    sg_opts r;
    sg_opts_default(&r);
    if (o) r = *o;
    if (r.precision != 0 && r.precision != 32) return SG_ERR_UNSUPPORTED;  // the FP32 walk
    if (r.boundary_mode) return SG_ERR_UNSUPPORTED;
    const float tau_near = r.tau_near > 0.f ? r.tau_near : 1e-4f, tau_snap = r.tau_snap > 0.f ? r.tau_snap : fminf(1e-6f, tau_near);
    if (tau_snap > tau_near) return SG_ERR_INVALID_ARG;  // a snapped vertex lies in the near band
    cudaStream_t s = (cudaStream_t)stream;
    StepsArgs a{};
    a.P.rec = m->d_rec; a.P.fv = m->d_fv; a.P.frm = m->d_frm; a.P.half = m->d_half; a.P.V = m->d_V;
    a.P.face_off = m->d_face_off; a.P.lref = m->d_lref;
    a.P.max_steps = r.max_steps > 0 ? r.max_steps : (1 << 20);
    a.P.tau_near = tau_near; a.P.tau_snap = tau_snap; a.P.want_hash = step_hash != nullptr;
    a.nq = nq; a.K = K; a.h = h; a.n_mesh = m->n_mesh; a.mesh_id = mesh_id; a.face = face; a.bary = bary; a.U = U;
    a.out_face = out_face; a.out_bary = out_bary; a.out_pos = out_pos; a.out_dir = out_dir; a.out_status = out_status;
    a.step_face = step_face; a.step_bary = step_bary; a.step_v = step_v; a.step_dir = step_dir;
    a.step_status = step_status; a.step_hash = step_hash;
    // scratch: the work-queue counter (the caller's workspace or stream-ordered memory)
    void *ws = r.workspace;
    void *own = nullptr;
    if (!ws || r.workspace_bytes < 64) {
        if (cudaMallocAsync(&own, 64, s) != cudaSuccess) { cudaGetLastError(); return SG_ERR_OOM; }
        ws = own;
    }
    a.counter = (int32_t *)ws;
    cudaMemsetAsync(a.counter, 0, 64, s);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_walk_steps, 256, 0);
    per = std::max(per, 1);
    const int64_t grid = std::min<int64_t>((int64_t)sms * per, (nq + 255) / 256);
    cudaEvent_t *pev = (cudaEvent_t *)r.prof_events;
    if (pev) cudaEventRecord(pev[0], s);
    k_walk_steps<<<(unsigned)grid, 256, 0, s>>>(a);
    if (pev) cudaEventRecord(pev[1], s);
    cudaError_t e = cudaGetLastError();
    if (own) cudaFreeAsync(own, s);
    return e == cudaSuccess ? SG_OK : SG_ERR_CUDA;
}

sg_status sg_exp_map_steps_backward_workspace_size(const sg_mesh *m, int32_t estimator, int32_t K, int64_t nq,
                                                   int32_t want_grad_V, size_t *bytes) {
    if (!m || !bytes || nq < 0 || K < 1 || K > SG_STEPS_MAX) return SG_ERR_INVALID_ARG;
    size_t inner = 0;
    sg_status st = sg_exp_map_backward_workspace_size(m, estimator, nq, want_grad_V, &inner);
    if (st != SG_OK) return st;
    const size_t v3 = al256(sizeof(float) * 3 * (size_t)std::max<int64_t>(nq, 1));
    // zeros (an absent end-point gradient), grad_v, grad_bary, two upstream-barycentric buffers
    *bytes = al256(inner) + 5 * v3;
    return SG_OK;
}

sg_status sg_exp_map_steps_backward(const sg_mesh *m, int32_t estimator, float eps_v, float eps_p, int32_t K,
                                    float h, const float *U, int64_t nq, const int32_t *mesh_id,
                                    const int32_t *step_face, const float *step_bary, const float *step_v,
                                    const float *step_dir, const uint32_t *step_status, const float *g_pos,
                                    const float *g_bary, float *grad_U, float *grad_bary, float *grad_V,
                                    const sg_opts *o, void *stream) {
    if (!m || nq < 0 || K < 1 || K > SG_STEPS_MAX) return SG_ERR_INVALID_ARG;
    if (nq == 0) return SG_OK;
    if (!U || !step_face || !step_bary || !step_v || !step_dir || !step_status || !g_pos || !grad_bary)
        return SG_ERR_INVALID_ARG;
    sg_opts r;
    sg_opts_default(&r);
    if (o) r = *o;
    size_t need = 0;
    sg_status st = sg_exp_map_steps_backward_workspace_size(m, estimator, K, nq, grad_V != nullptr, &need);
    if (st != SG_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    void *ws = r.workspace;
    void *own = nullptr;
    if (!ws) {
        if (cudaMallocAsync(&own, need, s) != cudaSuccess) { cudaGetLastError(); return SG_ERR_OOM; }
        ws = own;
    } else if (r.workspace_bytes < need) {
        return SG_ERR_OOM;
    }
    size_t inner = 0;
    sg_exp_map_backward_workspace_size(m, estimator, nq, grad_V != nullptr, &inner);
    const size_t v3 = al256(sizeof(float) * 3 * (size_t)nq);
    char *base = (char *)ws;
    void *inner_ws = base;
    float *zeros = (float *)(base + al256(inner));
    float *gv = (float *)(base + al256(inner) + v3);
    float *gbs = (float *)(base + al256(inner) + 2 * v3);
    float *gb[2] = {(float *)(base + al256(inner) + 3 * v3), (float *)(base + al256(inner) + 4 * v3)};
    cudaMemsetAsync(zeros, 0, sizeof(float) * 3 * (size_t)nq, s);
    sg_opts ri = r;
    ri.workspace = inner_ws;
    ri.workspace_bytes = inner;
    ri.prof_events = nullptr;
    const float *g_b = g_bary;  // upstream gradient of the current step's end barycentrics
    for (int k = K - 1; k >= 0 && st == SG_OK; --k) {
        const int64_t i0 = (int64_t)k * nq, i1 = (int64_t)(k + 1) * nq;
        st = sg_exp_map_backward(m, estimator, eps_v, eps_p, nq, mesh_id, step_face + i0, step_bary + 3 * i0,
                                 step_v + 3 * i0, step_face + i1, step_bary + 3 * i1, step_dir + 3 * i0,
                                 step_status + i0, k == K - 1 ? g_pos : zeros, g_b, nullptr, 0, nullptr, gv,
                                 nullptr, gbs, grad_V, nullptr, nullptr, &ri, stream);
        if (st != SG_OK) break;
        float *dst = k == 0 ? grad_bary : gb[k & 1];
        k_steps_field_bwd<<<(unsigned)((nq + 255) / 256), 256, 0, s>>>(nq, h, mesh_id, m->d_face_off, m->d_fv, U,
                                                                       step_face + i0, step_bary + 3 * i0,
                                                                       step_status + i0, gv, gbs, dst, grad_U);
        if (cudaGetLastError() != cudaSuccess) st = SG_ERR_CUDA;
        g_b = dst;
    }
    if (own) cudaFreeAsync(own, s);
    return st;
}

}  // extern "C"
