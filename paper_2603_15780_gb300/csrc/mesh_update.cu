// mesh_update.cu -- re-derive the geometry of an existing mesh from new vertex positions on
// the device (same faces, same adjacency).
//
// Sec. 4: the walk records hold only intrinsic quantities of the faces (edge lengths, the apex
// of each face in an edge frame, the face frame in 3-D) and the total angle theta(x) of each
// vertex, the sum of its incident corner angles.  All of these are functions of the vertex
// positions alone; the adjacency (neighbour links, flip bits, edge ids, boundary flags) depends
// on F only.  Moving the vertices -- e.g. a descent step on the vertex-position gradient --
// therefore rewrites the geometric words of the records in place and leaves the topological
// words untouched.
//
// The arithmetic is the FP64 arithmetic of the host builder, operation for operation (this file
// is compiled without FMA contraction, the host builder likewise), so an updated mesh holds the
// same records as a mesh created from the new positions.  Sums (theta per vertex, edge length per
// mesh) are accumulated with FP64 atomics, whose order differs from the host's; the rounding to
// FP32 absorbs that except in rare last-bit cases.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "sgeo_internal.h"

namespace {

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double norm(D3 a) { return sqrt(dot(a, a)); }
__device__ __forceinline__ D3 scale(D3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ int bits(float f) { return __float_as_int(f); }
__device__ __forceinline__ D3 load3(const float *X, int v) {
    return D3{(double)X[3 * v], (double)X[3 * v + 1], (double)X[3 * v + 2]};
}

struct UpdArgs {
    const float *X;  // new positions [nV][3]
    int64_t nF, nV;
    int32_t n_mesh;
    const int4 *fv;
    int4 *rec, *half;
    float4 *frm, *V;
    double *theta;              // [nV] corner-angle sums
    double *lsum;               // [n_mesh] sum of edge lengths (each edge once)
    unsigned long long *ecount; // [n_mesh] number of edges
    int *ndegen;                // [n_mesh] degenerate faces
    float *lref;                // [n_mesh]
};

// One thread per face: face record shape words, face frame, the three half-edge records'
// geometric words, the corner angles into theta, and this face's share of the edge lengths
// (each interior edge counted by its canonical half-edge, each boundary edge by its only one).
__global__ void k_update_faces(UpdArgs A) {
    int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= A.nF) return;
    const int4 t = A.fv[f];
    const int tv[3] = {t.x, t.y, t.z};
    const int m = t.w;
    D3 x0 = load3(A.X, t.x), x1 = load3(A.X, t.y), x2 = load3(A.X, t.z);
    D3 e1 = sub(x1, x0), e2 = sub(x2, x0);
    D3 n = cross(e1, e2);
    double l01 = norm(e1), nn = norm(n);
    // the host builder's zero-area test; also false for any non-finite coordinate
    if (!(nn > 1e-14 * fmax(dot(e1, e1), dot(e2, e2)))) atomicAdd(A.ndegen + m, 1);
    D3 u = scale(e1, 1.0 / l01);
    D3 nh = scale(n, 1.0 / nn);
    D3 w = cross(nh, u);
    double x2x = dot(e2, u), x2y = dot(e2, w);
    double l12 = norm(sub(x2, x1)), l20 = norm(e2);

    int4 r0 = A.rec[2 * f];
    r0.w = bits((float)l01);
    A.rec[2 * f] = r0;
    A.rec[2 * f + 1] = int4{bits((float)x2x), bits((float)x2y), bits((float)(1.0 / l12)), bits((float)(1.0 / l20))};
    A.frm[2 * f] = float4{(float)u.x, (float)u.y, (float)u.z, (float)w.x};
    A.frm[2 * f + 1] = float4{(float)w.y, (float)w.z, 0.f, 0.f};

    const D3 X3[3] = {x0, x1, x2};
    for (int k = 0; k < 3; ++k) {
        D3 a = sub(X3[(k + 1) % 3], X3[k]), b = sub(X3[(k + 2) % 3], X3[k]);
        atomicAdd(A.theta + tv[k], atan2(norm(cross(a, b)), dot(a, b)));
    }

    const double Px[3] = {0.0, l01, x2x}, Py[3] = {0.0, 0.0, x2y};
    double ls = 0.0;
    unsigned ne = 0;
    for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        double ex = Px[k1] - Px[k], ey = Py[k1] - Py[k];
        double l = sqrt(ex * ex + ey * ey);
        double ca = ex / l, sa = ey / l;
        double rx = Px[k2] - Px[k], ry = Py[k2] - Py[k];
        double cx = rx * ca + ry * sa, cy = -rx * sa + ry * ca;
        const int64_t h = 3 * f + k;
        int4 h0 = A.half[2 * h], h1 = A.half[2 * h + 1];
        h0.x = bits((float)l); h0.y = bits((float)cx); h0.z = bits((float)cy);
        h1.y = bits((float)ca); h1.z = bits((float)sa);
        A.half[2 * h] = h0;
        A.half[2 * h + 1] = h1;
        if (h1.w < 0 || (h1.w & 1) == 0) {  // boundary, or the canonical half-edge of an interior edge
            ls += norm(sub(X3[k1], X3[k]));
            ++ne;
        }
    }
    if (ne) {
        atomicAdd(A.lsum + m, ls);
        atomicAdd(A.ecount + m, (unsigned long long)ne);
    }
}

// One thread per vertex: new position, new theta, boundary sign kept from the old word.
__global__ void k_update_vertices(UpdArgs A) {
    int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= A.nV) return;
    float old = A.V[v].w;
    float th = (float)A.theta[v];
    A.V[v] = float4{A.X[3 * v], A.X[3 * v + 1], A.X[3 * v + 2], copysignf(th, old)};
}

// One thread per mesh: l_ref = mean edge length; a mesh with a degenerate face gets l_ref = -1,
// which the walk's query initialisation rejects (SG_ST_INVALID).
__global__ void k_update_meshes(UpdArgs A) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= A.n_mesh) return;
    double lr = A.lsum[m] / (double)A.ecount[m];
    A.lref[m] = A.ndegen[m] ? -1.f : (float)lr;
}

}  // namespace

extern "C" sg_status sg_mesh_update_vertices(sg_mesh *m, const float *V, void *stream) {
    if (!m || !V) return SG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!m->d_theta) {
        size_t b0 = sizeof(double) * (size_t)m->nV, b1 = sizeof(double) * (size_t)m->n_mesh,
               b2 = sizeof(unsigned long long) * (size_t)m->n_mesh, b3 = sizeof(int) * (size_t)m->n_mesh;
        if (cudaMalloc((void **)&m->d_theta, b0) != cudaSuccess ||
            cudaMalloc((void **)&m->d_lsum, b1) != cudaSuccess ||
            cudaMalloc((void **)&m->d_ecount, b2) != cudaSuccess ||
            cudaMalloc((void **)&m->d_ndegen, b3) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(m->d_theta); cudaFree(m->d_lsum); cudaFree(m->d_ecount); cudaFree(m->d_ndegen);
            m->d_theta = nullptr; m->d_lsum = nullptr; m->d_ecount = nullptr; m->d_ndegen = nullptr;
            return SG_ERR_OOM;
        }
        m->device_bytes += (int64_t)(b0 + b1 + b2 + b3);
    }
    UpdArgs A;
    A.X = V; A.nF = m->nF; A.nV = m->nV; A.n_mesh = m->n_mesh;
    A.fv = m->d_fv; A.rec = m->d_rec; A.half = m->d_half; A.frm = m->d_frm; A.V = m->d_V;
    A.theta = m->d_theta; A.lsum = m->d_lsum; A.ecount = m->d_ecount; A.ndegen = m->d_ndegen;
    A.lref = m->d_lref;
    if (cudaMemsetAsync(A.theta, 0, sizeof(double) * (size_t)m->nV, s) != cudaSuccess ||
        cudaMemsetAsync(A.lsum, 0, sizeof(double) * (size_t)m->n_mesh, s) != cudaSuccess ||
        cudaMemsetAsync(A.ecount, 0, sizeof(unsigned long long) * (size_t)m->n_mesh, s) != cudaSuccess ||
        cudaMemsetAsync(A.ndegen, 0, sizeof(int) * (size_t)m->n_mesh, s) != cudaSuccess)
        return SG_ERR_CUDA;
    k_update_faces<<<(unsigned)((m->nF + 255) / 256), 256, 0, s>>>(A);
    k_update_vertices<<<(unsigned)((m->nV + 255) / 256), 256, 0, s>>>(A);
    k_update_meshes<<<(unsigned)((m->n_mesh + 127) / 128), 128, 0, s>>>(A);
    if (cudaGetLastError() != cudaSuccess) return SG_ERR_CUDA;
    m->updated = true;
    m->geom64_stale = true;
    m->half48_stale = true;
    return SG_OK;
}
