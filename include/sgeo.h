/*
 * sgeo.h -- C ABI of the GB300 straightest-geodesic exponential-map library (libsgeo.so).
 *
 * The library computes, for a batch of queries on triangle meshes, the discrete
 * exponential map by straightest geodesics (Sec. 3 "exponential map"; Sec. 4
 * "Straightest geodesics"; Alg. "Parallel Geodesic Tracing CUDA Kernel"), the parallel
 * transport of carried tangent vectors (Sec. 4 "Parallel Transport"), and the two
 * backward estimators of Sec. 4: the extrinsic proxy (EP, Eq. "proxy_func") and geodesic
 * finite differences (GFD, Eqs. "jv", "jp", batched as in App. "Speed-up GFD and EP
 * through batching"), plus the gradient with respect to vertex positions.
 *
 * Conventions for every entry point
 *   - Plain C types only.  "device" pointers are CUDA global-memory pointers of the
 *     current device; "host" pointers are ordinary CPU memory.
 *   - The caller owns every query, output and gradient buffer.  The library owns the
 *     mesh object (created by sg_mesh_create*, released by sg_mesh_destroy).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  All
 *     device work of sg_exp_map / sg_exp_map_backward is enqueued on it; those calls do
 *     not synchronise the host.  sg_mesh_create* is synchronous.
 *   - API-level errors come back as sg_status.  A failed launch returns SG_ERR_CUDA and
 *     leaves the outputs unspecified.  Per-query outcomes are written to a status word
 *     (SG_ST_* bits) and never abort the batch.
 *   - Points are (face, barycentric) pairs (Sec. 4): p = b0 x0 + b1 x1 + b2 x2 with
 *     (x0, x1, x2) the face's vertices in the order given in F.
 *   - Arrays are dense, row-major: bary/v/pos/dir are [nq][3] float32, carried vectors
 *     are [nq][n_w][3] float32, faces are int32.
 */
#ifndef SGEO_H
#define SGEO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sg_mesh sg_mesh; /* opaque, library-owned */

typedef enum sg_status {
    SG_OK = 0,
    SG_ERR_INVALID_ARG = 1,  /* null pointer, negative size, index out of range, bad option */
    SG_ERR_NONMANIFOLD = 2,  /* an edge with >2 faces or a vertex with more than one fan (Sec. 4) */
    SG_ERR_DEGENERATE = 3,   /* a face with repeated vertices or zero area */
    SG_ERR_CUDA = 4,         /* a CUDA runtime call or kernel launch failed */
    SG_ERR_OOM = 5,          /* device allocation failed or workspace too small */
    SG_ERR_UNSUPPORTED = 6   /* option combination not implemented */
} sg_status;

/* per-query status bits (out_status) */
#define SG_ST_BOUNDARY 1u        /* walk stopped on a boundary edge/vertex (Sec. 4, original rule) */
#define SG_ST_MAX_STEPS 2u       /* MAX_STEPS reached (Alg. gpu_parallel) */
#define SG_ST_NEAR_VERTEX 4u     /* ray passed within tau_near*l_ref of a vertex without snapping */
#define SG_ST_NEAR_EDGE 8u       /* end point within tau_near*l_ref of an edge of its face */
#define SG_ST_VERTEX_HIT 16u     /* at least one vertex transport (straightest rule) was applied */
#define SG_ST_FP64 32u           /* edge-exit / vertex-hit classification was re-evaluated in FP64 */
#define SG_ST_START_ON_EDGE 64u  /* the start point has a zero barycentric coordinate */
#define SG_ST_INVALID 128u       /* query rejected (bad face, barycentrics, or vector); outputs = start */
#define SG_ST_GFD_SPLIT 256u     /* (backward) a GFD perturbed ray left the base ray's face strip */
#define SG_ST_FLIPPED 512u       /* the end face's orientation is reversed relative to the start
                                    (odd number of inconsistently oriented edges crossed) */
#define SG_ST_NO_GRADV 1024u     /* (backward) no vertex-position gradient for this query (vertex
                                    hit or boundary stop: the map is not differentiable there) */

/* kernels */
#define SG_KERNEL_AUTO 0
#define SG_KERNEL_PLAIN 1        /* one thread per query, grid = ceil(nq / block), no sort, FP32 only */
#define SG_KERNEL_PERSISTENT 2   /* SM-filling grid pulling queries from an atomic counter */

typedef struct sg_opts {
    int32_t max_steps;      /* loop cap per query (Alg. gpu_parallel MAX_STEPS); <= 0: 1<<20 */
    int32_t kernel;         /* SG_KERNEL_*; AUTO = persistent */
    int32_t sort;           /* 1: order queries by (mesh, start face) before walking; 0: no; <0: auto (on) */
    int32_t block;          /* threads per block; <= 0: 256 */
    int32_t blocks_per_sm;  /* persistent kernel residency; <= 0: as many as fit */
    int32_t fp64_escalate;  /* 1: re-evaluate near-vertex classification in FP64 (persistent only) */
    float tau_near;         /* flag radius / l_ref for NEAR_VERTEX, NEAR_EDGE and the FP64 band; <= 0: 1e-4 */
    float tau_snap;         /* vertex-snap radius / l_ref; <= 0: 1e-6 */
    void *workspace;        /* optional device scratch (see sg_exp_map_workspace_size); NULL: the
                               library allocates stream-ordered scratch itself */
    size_t workspace_bytes;
    void *prof_events;      /* optional: pointer to two cudaEvent_t recorded on `stream` right
                               before and after the call's walk kernel (forward walk, or the
                               backward re-walk), for per-kernel timing; NULL: none */
} sg_opts;

/* Fills `o` with the defaults described above. */
void sg_opts_default(sg_opts *o);

/* Human-readable name of a status code (static string). */
const char *sg_status_string(sg_status s);

/*
 * sg_mesh_create -- build the walk records of one triangle mesh M = {X, F} (Sec. 4).
 *   V   host float32 [nV][3] vertex positions
 *   F   host int32 [nF][3] vertex indices, 0 <= F < nV
 * Builds, in FP64 on the host, the triangle adjacency (only adjacencies are stored, so
 * non-orientable meshes work, App. "Main differences with SotA implementation"), the
 * per-face intrinsic 2-D shape, the vertex total angle theta(x) (Sec. 4), boundary
 * flags and the mean edge length l_ref, then uploads them to the current device.
 * Validates the manifold definition of Sec. 4.  Synchronous.  On success *out owns
 * device memory until sg_mesh_destroy.
 * Errors: SG_ERR_INVALID_ARG, SG_ERR_NONMANIFOLD, SG_ERR_DEGENERATE, SG_ERR_OOM, SG_ERR_CUDA.
 */
sg_status sg_mesh_create(const float *V, int64_t nV, const int32_t *F, int64_t nF, sg_mesh **out);

/*
 * sg_mesh_create_batched -- several meshes in one object for heterogeneous batching
 * (Sec. 4 "Parallelisation on the GPU": face indices and (f, b) offset per mesh).
 *   V      host float32 [v_off[n_mesh]][3], meshes concatenated
 *   v_off  host int64 [n_mesh + 1] vertex offsets (v_off[0] = 0)
 *   F      host int32 [f_off[n_mesh]][3], indices LOCAL to each mesh's vertices
 *   f_off  host int64 [n_mesh + 1] face offsets (f_off[0] = 0)
 * Queries then name a mesh (mesh_id) and a face local to it.  Same errors as above.
 */
sg_status sg_mesh_create_batched(const float *V, const int64_t *v_off, const int32_t *F,
                                 const int64_t *f_off, int32_t n_mesh, sg_mesh **out);

/* Releases a mesh (device memory included).  NULL is accepted. */
sg_status sg_mesh_destroy(sg_mesh *m);

typedef struct sg_mesh_info {
    int64_t n_vertices, n_faces;
    int32_t n_mesh;
    int32_t record_bytes;      /* bytes per face walk record */
    int64_t device_bytes;      /* total device memory held by the mesh */
    double l_ref_mean;         /* mean edge length of mesh 0 */
} sg_mesh_info;

sg_status sg_mesh_get_info(const sg_mesh *m, sg_mesh_info *info);

/*
 * sg_exp_map_workspace_size -- bytes of device scratch sg_exp_map needs for nq queries
 * with options `o` (the start-face sort and the work-queue counter).
 */
sg_status sg_exp_map_workspace_size(const sg_mesh *m, int64_t nq, const sg_opts *o, size_t *bytes);

/*
 * sg_exp_map -- batched forward exponential map with parallel transport.
 * Alg. "Parallel Geodesic Tracing CUDA Kernel" with Alg. geodesic_step,
 * transport_over_edge and transport_over_vertex; initialise_trace projects v (and w)
 * onto the start face plane and sets L = |v| unless `length` is given.
 *   mesh_id  device int32 [nq] or NULL (all queries on mesh 0)
 *   face     device int32 [nq] start face, local to its mesh
 *   bary     device float32 [nq][3] start barycentrics (sum within 1e-6 of 1, >= 0)
 *   v        device float32 [nq][3] ambient tangent vector (projected onto the face plane)
 *   length   device float32 [nq] geodesic length, or NULL for |v|
 *   n_w, w   number of carried vectors (0..4) and device float32 [nq][n_w][3] (NULL if 0)
 * Outputs (device, caller-allocated; out_w/out_ncross/out_hash may be NULL):
 *   out_face int32 [nq] end face (local), out_bary float32 [nq][3], out_pos float32 [nq][3],
 *   out_dir float32 [nq][3] transported unit direction, out_w float32 [nq][n_w][3],
 *   out_status uint32 [nq] (SG_ST_*), out_ncross int32 [nq] edge crossings,
 *   out_hash uint64 [nq] word-wise FNV-1a 64 hash of the visited face sequence (local ids).
 * Invalid queries get SG_ST_INVALID and their start as output.  Asynchronous on `stream`.
 */
sg_status sg_exp_map(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face,
                     const float *bary, const float *v, const float *length, int32_t n_w,
                     const float *w, int32_t *out_face, float *out_bary, float *out_pos,
                     float *out_dir, float *out_w, uint32_t *out_status, int32_t *out_ncross,
                     uint64_t *out_hash, const sg_opts *o, void *stream);

/*
 * sg_exp_map_noalloc -- sg_exp_map for callers that cannot allocate device memory when they
 * call in: for example code running inside a framework that owns all device memory through
 * its own pool, or a latency-critical loop where a cudaMalloc/cudaFree (which can
 * synchronise the device) is not allowed.  The paper has no counterpart; it is an interface
 * convenience of this library.
 * Same arguments, outputs and errors as sg_exp_map; o->workspace is ignored.  The scratch
 * (work-queue counter and start-face sort) lives in one fixed 32 MiB device array inside the
 * library, which every GPU that loads the library holds until the process exits.  Batches
 * whose scratch (sg_exp_map_workspace_size with the same options) exceeds 32 MiB are rejected
 * with SG_ERR_OOM and nothing is launched; with o->sort = 0 the scratch is 64 bytes and any
 * batch size fits.  No cudaMalloc, cudaFree or allocating library routine is called.
 * The first call on a device looks the array's address up (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.  All calls share the one
 * array: the library clears what must start at zero on every call, but calls whose GPU work
 * overlaps in time (concurrent streams, several host threads) race on it and must be
 * serialised by the caller.
 */
sg_status sg_exp_map_noalloc(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face,
                             const float *bary, const float *v, const float *length, int32_t n_w,
                             const float *w, int32_t *out_face, float *out_bary, float *out_pos,
                             float *out_dir, float *out_w, uint32_t *out_status, int32_t *out_ncross,
                             uint64_t *out_hash, const sg_opts *o, void *stream);

/* backward estimators */
#define SG_EST_EP 0   /* Eq. proxy_func: J^v = R, J^p zeroed */
#define SG_EST_GFD 1  /* Eqs. jv, jp: geodesic finite differences */

/*
 * sg_exp_map_backward -- vector-Jacobian products of the end point p' = Exp_p(v).
 *   estimator  SG_EST_EP or SG_EST_GFD; eps_v, eps_p the GFD steps (world units, > 0)
 *   mesh_id, face, bary, v   the forward inputs (device, as in sg_exp_map; L = |v|)
 *   end_face, end_bary, end_dir  the forward outputs for these queries (device)
 *   end_status the forward status words (device) or NULL (then SG_ST_FLIPPED is taken as 0,
 *              exact for orientable meshes)
 *   g_pos      device float32 [nq][3] upstream gradient dL/dp'
 * Outputs (device, caller-allocated, any may be NULL):
 *   grad_v     float32 [nq][3]  dL/dv (tangent to the start face)
 *   grad_p     float32 [nq][3]  dL/dp in the start face plane (zero for EP, Sec. 4)
 *   grad_bary  float32 [nq][3]  dL/db_k = <grad_p, x_k> (meaningful up to the simplex gauge)
 *   grad_V     float32 [nV][3]  dL/dX, ACCUMULATED (+=) over queries; the derivative of the
 *                               end point with the face sequence held fixed (see DESIGN)
 *   out_status uint32 [nq]      SG_ST_* of the extra walks (GFD) or of the re-walk
 * Asynchronous on `stream`.
 */
sg_status sg_exp_map_backward(const sg_mesh *m, int32_t estimator, float eps_v, float eps_p,
                              int64_t nq, const int32_t *mesh_id, const int32_t *face,
                              const float *bary, const float *v, const int32_t *end_face,
                              const float *end_bary, const float *end_dir,
                              const uint32_t *end_status, const float *g_pos,
                              float *grad_v, float *grad_p, float *grad_bary, float *grad_V,
                              uint32_t *out_status, const sg_opts *o, void *stream);

/*
 * sg_exp_map_backward_workspace_size -- bytes of device scratch sg_exp_map_backward needs for
 * nq queries with `estimator` (SG_EST_*) and, if want_grad_V != 0, the vertex gradient: the
 * GFD column table (16 B per query) and swept-perturbation task list (12 B per query), and
 * a float4 accumulator per vertex for grad_V.  Pass it as o->workspace; without it the
 * library allocates stream-ordered scratch itself.
 */
sg_status sg_exp_map_backward_workspace_size(const sg_mesh *m, int32_t estimator, int64_t nq,
                                             int32_t want_grad_V, size_t *bytes);

/* Library version string. */
const char *sg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SGEO_H */
