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
#define SG_ST_HOLE 2048u         /* hole avoidance (boundary_mode 1) traced along the boundary */
#define SG_ST_MIXED 4096u        /* walked by the mixed-precision walk (precision 40, or chosen by the
                                    automatic precision for a walk beyond the FP32 walk's range) */
#define SG_ST_REWALK_DIVERGED 8192u /* (backward) the FP32 re-walk ended in another face than the
                                    forward walk (possible only where the forward walk was the
                                    mixed walk): the gradients follow the re-walk's path */

/* kernels */
#define SG_KERNEL_AUTO 0
#define SG_KERNEL_PLAIN 1        /* one thread per query, grid = ceil(nq / block), no sort, FP32 only */
#define SG_KERNEL_PERSISTENT 2   /* SM-filling grid pulling queries from an atomic counter */

typedef struct sg_opts {
    int32_t max_steps;      /* loop cap per query (Alg. gpu_parallel MAX_STEPS); <= 0: 1<<20 */
    int32_t kernel;         /* SG_KERNEL_*; AUTO: the persistent kernel, except that sg_exp_map
                               walks a batch of fewer than 65,536 queries taken in input order
                               (FP32 precision, boundary_mode 0) one thread per query with the
                               persistent kernel's arithmetic (FP64 classification kept): such a
                               batch fills the persistent grid once, so the queue gains nothing */
    int32_t sort;           /* order in which the persistent kernels take the queries:
                               0: input order; 1: by (mesh, start face), the faces taken along
                               the mesh's Z-order curve of face centroids so that neighbouring
                               queries start in one patch of the surface; 2: by walk length,
                               longest first (L or |v| over l_ref, an eighth of an octave per
                               bucket: lanes of a warp then finish together and idle less);
                               <0: auto -- for batches of >= 65536 queries, 1 on meshes whose
                               walk records (128 B per face) exceed half of L2 (locality of the
                               gathers), else 2; input order for smaller batches.  Outputs are
                               always in input order.  sg_exp_map_backward's re-walk uses the
                               length order when sort is 2, or auto with >= 65536 queries. */
    int32_t block;          /* threads per block; <= 0: 256 */
    int32_t blocks_per_sm;  /* persistent kernel residency; <= 0: as many as fit */
    int32_t fp64_escalate;  /* 1: re-evaluate near-vertex classification in FP64 (persistent only) */
    float tau_near;         /* flag radius / l_ref for NEAR_VERTEX, NEAR_EDGE and the FP64 band; <= 0: 1e-4 */
    float tau_snap;         /* vertex-snap radius / l_ref; <= 0: 1e-6 (precision 0, 32, 40), 1e-12
                               (48, 64), or tau_near if that is smaller; a value above tau_near is
                               rejected (SG_ERR_INVALID_ARG): a snapped vertex lies inside the
                               near band */
    void *workspace;        /* optional device scratch (see sg_exp_map_workspace_size); NULL: the
                               library allocates stream-ordered scratch itself */
    size_t workspace_bytes;
    void *prof_events;      /* optional: pointer to two cudaEvent_t recorded on `stream` right
                               before and after the call's walk kernel (forward walk, or the
                               backward re-walk), for per-kernel timing; NULL: none */
    int32_t boundary_mode;  /* 0: a walk stops on the boundary (Sec. 4, the original rule);
                               1: hole avoidance (Sec. 4): trace along the boundary and resume
                               with the last straightest direction as soon as a face receives
                               it (SG_ST_HOLE).  Mode 1 runs on the persistent kernel with FP64
                               classification; the plain kernel and sg_exp_map_trace reject it
                               (SG_ERR_UNSUPPORTED). */
    int32_t precision;      /* 0 (default): automatic -- each query walks in FP32 (with FP64
                               classification near vertices) while its walk stays within the range
                               where the FP32 walk's face sequences were measured equal to the
                               double-precision ones (at most 256 crossings), else in the mixed walk
                               (40): queries longer than 96 l_ref are routed to it by the query order,
                               and a walk that reaches 256 crossings is restarted there (SG_ST_MIXED
                               marks both).  sg_exp_map_trace, the backward and hole avoidance
                               (boundary_mode 1) walk in FP32 under this setting;
                               32: the FP32 walk for every query;
                               40: the mixed walk: the FP32 walk's orientation tests, exit points and
                               length, with the walking direction and the records' edge vectors in
                               double-float (pairs of FP32 numbers), so that the direction's error no
                               longer grows with the path;
                               48: the double-float walk: every crossing in double-float arithmetic
                               (about 48 significant bits), the rare events (vertex hits, boundary
                               stops, starts on an edge or vertex) in FP64;
                               64: every quantity of the walk in FP64 (state, face shapes, frames,
                               vertex angles).
                               40, 48 and 64 run on the persistent kernel, forward only (the trace,
                               the backward, boundary_mode 1 and the plain kernel reject them with
                               SG_ERR_UNSUPPORTED).  Their FP64 geometry and double-float records
                               (192 B per face, 8 B per vertex) are built with the mesh. */
    int32_t queries_per_thread; /* <= 0: the default launch.  Plain kernel: each thread walks this
                               many queries in turn (grid-stride; grid = ceil(nq / (block * qpt))).
                               Persistent kernel: the grid is sized so that each thread takes about
                               this many queries from the queue on average (blocks per SM =
                               ceil(nq / (qpt * SMs * block)), at most the occupancy limit and the
                               blocks_per_sm given); the autotuner sweeps it. */
    int32_t *order;         /* optional device int32[nq] buffer holding a query order.  sg_exp_map
                               and sg_exp_map_trace write into it the walk-length order of the
                               queries (longest first, the order sg_exp_map_backward's re-walk
                               takes): their own queue's order when they took the queries in that
                               order (no cost), else one built for the buffer (two launches, after
                               a start-face or input-order walk).  sg_exp_map_backward reads it,
                               when given, as the order of its re-walk instead of rebuilding the
                               length order (two launches fewer): pass the buffer the forward call
                               filled for the same queries.  It must be a permutation of
                               0..nq-1; an entry out of that range is skipped (no query is walked
                               for it).  NULL: none. */
} sg_opts;

/* Fills `o` with the defaults described above. */
void sg_opts_default(sg_opts *o);

/* Human-readable name of a status code (static string). */
const char *sg_status_string(sg_status s);

/*
 * sg_mesh_create -- build the walk records of one triangle mesh M = {X, F} (Sec. 4).
 *   V   float32 [nV][3] vertex positions, host or device memory (detected)
 *   F   int32 [nF][3] vertex indices, 0 <= F < nV, host or device memory (detected)
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
 *   V      float32 [v_off[n_mesh]][3], meshes concatenated
 *   v_off  int64 [n_mesh + 1] vertex offsets (v_off[0] = 0)
 *   F      int32 [f_off[n_mesh]][3], indices LOCAL to each mesh's vertices
 *   f_off  int64 [n_mesh + 1] face offsets (f_off[0] = 0)
 * Each array may be host or device memory (detected with cudaPointerGetAttributes; device
 * arrays are copied to the host, where the adjacency is built).
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
    int64_t n_degenerate;      /* faces left degenerate by the last sg_mesh_update_vertices */
} sg_mesh_info;

/* Fills `info`.  After sg_mesh_update_vertices it reads the current l_ref and degenerate
 * count back from the device (a synchronous copy that waits for the update). */
sg_status sg_mesh_get_info(const sg_mesh *m, sg_mesh_info *info);

/*
 * sg_mesh_update_vertices -- move the vertices of a mesh to new positions, keeping its faces
 * and adjacency, and re-derive on the device every geometric word of its walk records: the
 * per-face intrinsic shape and 3-D frame, the half-edge records, the total angle theta(x) of
 * each vertex and l_ref (Sec. 4 "Straightest geodesics": all of them are functions of the
 * vertex positions; the adjacency and boundary flags depend on F only).  This serves
 * optimisation of vertex positions with the grad_V output of sg_exp_map_backward, without a
 * host round trip or a rebuild of the adjacency.
 *   m       a mesh from sg_mesh_create*
 *   V       device float32 [n_vertices][3] new positions, in the mesh's vertex order
 *           (meshes of a batch concatenated, as at creation); read during the call's kernels
 *   stream  cudaStream_t as void*; the work is enqueued on it and the host is not synchronised,
 *           except by the first call on a mesh, which allocates O(n_vertices) FP64 scratch
 *           (cudaMalloc) that the mesh keeps until sg_mesh_destroy.
 * The records are rewritten in place: walks reading the mesh on other streams must be ordered
 * before the call by the caller.  The arithmetic is that of sg_mesh_create (FP64, no
 * multiply-add contraction), so an updated mesh walks like one created from the new positions;
 * the FP64 sums (theta, l_ref) are accumulated in a different order, which can move their FP32
 * values by one unit in the last place.  The faces' places on the Z-order curve that keys the
 * start-face query order keep the creation positions (an order, not a result: walks give the same
 * outputs in any order).
 * A face that the new positions make zero-area or non-finite marks its mesh (its member of a
 * batch) unusable: every query on it returns SG_ST_INVALID until a later update makes all of
 * its faces valid again; sg_mesh_get_info reports the count.
 * Errors: SG_ERR_INVALID_ARG (null mesh or V), SG_ERR_OOM (first-call scratch), SG_ERR_CUDA.
 */
sg_status sg_mesh_update_vertices(sg_mesh *m, const float *V, void *stream);

/*
 * sg_exp_map_workspace_size -- bytes of device scratch sg_exp_map needs for nq queries
 * with options `o` (the query order, the work-queue counter, the automatic precision's
 * escalation list, and, when o->order is set and the walk takes another order than the length
 * order, the length order's keys: 1 byte per query and 2 KiB).  Set o->order before asking.
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
 * Two more rules keep it allocation-free.  The current device must be the one the mesh was
 * created on (else SG_ERR_INVALID_ARG: the array's address is per device).  The FP64 geometry
 * and double-float records that the automatic, mixed, double-float and FP64 precisions walk on
 * are allocated by sg_mesh_create; after a vertex update they are re-derived in place, on
 * `stream`, by the next call.
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
 * sg_exp_map_trace -- the forward walk with the traced geodesic as an extra output.
 * Straightest geodesics trace geodesics as a by-product of the exponential map (Sec. 1,
 * Sec. 4 "Straightest geodesics"): inside a face the geodesic is a straight segment, so the
 * ordered faces it enters and the points where it enters them, followed by the end point, are
 * its polyline.  Same walk, inputs and end outputs as sg_exp_map without carried vectors, on
 * the persistent kernel (opts.kernel only chooses whether queries are sorted: PLAIN disables
 * the sort and the FP64 classification).
 *   path_cap       entries stored per query (>= 0)
 *   out_path_face  device int32 [nq][path_cap]: local ids of the faces entered, in order (the
 *                  start face first; a vertex hit that leaves through the same face repeats
 *                  it).  Entries past min(path_len, path_cap) are not written.
 *   out_path_pt    device float32 [nq][path_cap][3] or NULL: the point where the walk enters
 *                  each face (the start point, an edge crossing point, or the hit vertex)
 *   out_path_len   device int32 [nq]: faces entered; above path_cap the path was truncated
 *                  (0 for invalid and zero-length queries, which enter no face)
 * The face sequence is the one that out_hash hashes.  Asynchronous on `stream`.
 * Errors: as sg_exp_map.
 */
sg_status sg_exp_map_trace(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face,
                           const float *bary, const float *v, const float *length, int32_t path_cap,
                           int32_t *out_path_face, float *out_path_pt, int32_t *out_path_len, int32_t *out_face,
                           float *out_bary, float *out_pos, float *out_dir, uint32_t *out_status,
                           int32_t *out_ncross, uint64_t *out_hash, const sg_opts *opts, void *stream);

/*
 * sg_exp_map_backward -- vector-Jacobian products of the forward outputs (Sec. 4 "Gradient
 * computation": the chain rule through Exp, with J^v, J^p from EP, Eq. proxy_func, or GFD,
 * Eqs. jv, jp).
 *   estimator  SG_EST_EP or SG_EST_GFD; eps_v, eps_p the GFD steps (world units, > 0)
 *   mesh_id, face, bary, v   the forward inputs (device, as in sg_exp_map; L = |v|)
 *   end_face, end_bary, end_dir  the forward outputs for these queries (device)
 *   end_status the forward status words (device) or NULL (then SG_ST_FLIPPED is taken as 0,
 *              exact for orientable meshes)
 * Upstream gradients (device float32; all but g_pos may be NULL):
 *   g_pos      [nq][3]  dL/dp' of the end point
 *   g_bary     [nq][3]  dL/db' of the end barycentrics (e.g. when b' starts a next step): it
 *                       enters as the tangent vector g_t with g_t . dp = sum_k g_bary_k db'_k
 *   g_dir      [nq][3]  dL/dd' of the transported unit direction: differentiated with the
 *                       rotation R = M_p' M_p^T of Eq. proxy_func held fixed (both estimators):
 *                       grad_v += (I - d0 d0^T) R^T g_dir / |v|
 *   n_w, g_w   [nq][n_w][3] dL/dw' of the carried vectors (0 <= n_w <= 4; g_w and grad_w
 *                       both given or both NULL)
 * Outputs (device, caller-allocated, any may be NULL):
 *   grad_v     float32 [nq][3]  dL/dv (tangent to the start face)
 *   grad_p     float32 [nq][3]  dL/dp in the start face plane (zero for EP, Sec. 4)
 *   grad_bary  float32 [nq][3]  dL/db_k = <grad_p, x_k> (meaningful up to the simplex gauge)
 *   grad_V     float32 [nV][3]  dL/dX, ACCUMULATED (+=) over queries: the derivative of the end
 *                               point (and barycentrics) in the vertex positions with the face
 *                               sequence held fixed; queries with a vertex hit or a boundary stop
 *                               add nothing and get SG_ST_NO_GRADV
 *   grad_w     float32 [nq][n_w][3]  dL/dw = R^T g_w (parallel transport is a rotation of the
 *                               tangent planes for a fixed face sequence; exact)
 *   out_status uint32 [nq]      SG_ST_* of the extra walks (GFD) or of the re-walk
 * The re-walk (GFD, or grad_V) takes the queries in the order o->order holds when it is given
 * (the forward call's, see sg_opts.order), else in its own length order.
 * Asynchronous on `stream`.  Errors: SG_ERR_INVALID_ARG (bad estimator, eps <= 0 for GFD, a
 * required array NULL, nq above 536,869,887), SG_ERR_UNSUPPORTED (precision 40, 48 or 64), SG_ERR_OOM
 * (no workspace given and none could be allocated), SG_ERR_CUDA.
 */
sg_status sg_exp_map_backward(const sg_mesh *m, int32_t estimator, float eps_v, float eps_p,
                              int64_t nq, const int32_t *mesh_id, const int32_t *face,
                              const float *bary, const float *v, const int32_t *end_face,
                              const float *end_bary, const float *end_dir,
                              const uint32_t *end_status, const float *g_pos, const float *g_bary,
                              const float *g_dir, int32_t n_w, const float *g_w,
                              float *grad_v, float *grad_p, float *grad_bary, float *grad_V,
                              float *grad_w, uint32_t *out_status, const sg_opts *o, void *stream);

/*
 * sg_exp_map_steps -- the K-step exponential map of a vector field sampled at the mesh vertices,
 * x_{k+1} = Exp_{x_k}(h u(x_k)) for k = 0..K-1, in one launch (Sec. 5, Eq. "fmobj": the flow is
 * integrated by K exponential-map steps with the field re-evaluated at every intermediate point).
 * The field is given by its values at the vertices and evaluated at a point by barycentric
 * interpolation, u(x) = sum_j b_j U[F[f, j]]; each step projects h u(x_k) onto the face it starts
 * in and walks it with the FP32 walk of sg_exp_map (FP64 classification near vertices).
 *   K          number of steps, 1..64;  h  the step's scale (for example 1 / K)
 *   U          device float32 [n_vertices][3] ambient field vectors (global vertex ids of a batch)
 *   mesh_id, face, bary  the start points, as in sg_exp_map
 * Outputs (device, caller-allocated): out_face, out_bary, out_pos, out_dir of the last step;
 * out_status the OR of the steps' status bits (SG_ST_FLIPPED excluded).  Per-step records, all
 * given or all NULL (step_hash may be NULL), needed by sg_exp_map_steps_backward:
 *   step_face  int32 [K + 1][nq]: each step's start face (local), then the end face
 *   step_bary  float32 [K + 1][nq][3]: each step's start barycentrics, then the end's
 *   step_v     float32 [K][nq][3]: the ambient vector h u(x_k) each step was given
 *   step_dir   float32 [K][nq][3]: each step's end direction
 *   step_status uint32 [K][nq]: each step's status (SG_ST_FLIPPED relative to its own start)
 *   step_hash  uint64 [K][nq]: each step's face-sequence hash (as sg_exp_map's out_hash)
 * A zero vector makes its step the identity.  opts: kernel, sort and block are ignored (the
 * persistent kernel, queries in input order); precision 0 and 32 walk in FP32, others and
 * boundary_mode 1 are rejected with SG_ERR_UNSUPPORTED.  Scratch: 64 bytes (o->workspace, or
 * stream-ordered memory).  Asynchronous on `stream`.
 * Errors: SG_ERR_INVALID_ARG (K out of range, a required array NULL, records given in part),
 * SG_ERR_UNSUPPORTED, SG_ERR_OOM, SG_ERR_CUDA.
 */
sg_status sg_exp_map_steps(const sg_mesh *m, int32_t K, float h, const float *U, int64_t nq, const int32_t *mesh_id,
                           const int32_t *face, const float *bary, int32_t *out_face, float *out_bary, float *out_pos,
                           float *out_dir, uint32_t *out_status, int32_t *step_face, float *step_bary, float *step_v,
                           float *step_dir, uint32_t *step_status, uint64_t *step_hash, const sg_opts *o,
                           void *stream);

/*
 * sg_exp_map_steps_backward -- vector-Jacobian product of sg_exp_map_steps (the chain rule through
 * the K steps, Sec. 4 "Gradient computation"): from the last step back to the first, the
 * estimator's VJP of the step (sg_exp_map_backward, EP or GFD, which recomputes the step's walk)
 * with the upstream gradients of its end point (g_pos, last step only) and end barycentrics, then
 * the field's term: with v_k = h sum_j b_kj U_j, grad U_j += h b_kj grad_v_k and the gradient of
 * the step's start barycentrics gains h <U_j, grad_v_k>; their sum is the upstream gradient of the
 * previous step's end barycentrics.
 *   step_*     the forward's per-step records;  U, h, K, mesh_id as given to the forward
 *   g_pos      device float32 [nq][3] dL/dx_K;  g_bary  [nq][3] dL/db_K or NULL
 * Outputs (device): grad_U float32 [n_vertices][3] ACCUMULATED (+=) or NULL; grad_bary float32
 * [nq][3] dL/db_0 (meaningful up to the simplex gauge); grad_V [n_vertices][3] accumulated or NULL.
 * Scratch: sg_exp_map_steps_backward_workspace_size (o->workspace, or stream-ordered memory).
 * Asynchronous on `stream`.  Errors: as sg_exp_map_backward.
 */
sg_status sg_exp_map_steps_backward(const sg_mesh *m, int32_t estimator, float eps_v, float eps_p, int32_t K,
                                    float h, const float *U, int64_t nq, const int32_t *mesh_id,
                                    const int32_t *step_face, const float *step_bary, const float *step_v,
                                    const float *step_dir, const uint32_t *step_status, const float *g_pos,
                                    const float *g_bary, float *grad_U, float *grad_bary, float *grad_V,
                                    const sg_opts *o, void *stream);
sg_status sg_exp_map_steps_backward_workspace_size(const sg_mesh *m, int32_t estimator, int32_t K, int64_t nq,
                                                   int32_t want_grad_V, size_t *bytes);

/*
 * sg_transport_back -- the adjoint of the parallel transport along each query's geodesic,
 * which is its inverse: tangent vectors at the end point p' are moved backwards along the
 * curve to the start point p (App. "Additional Details on Mesh-LBFGS and GCVT": the vector
 * transport of the Riemannian L-BFGS and its adjoint; Sec. 4 "Parallel Transport").  The
 * forward transport keeps each vector's signed angle to the walking direction, so for the
 * forward's face sequence it is a rotation R of the tangent planes and this call applies R^T:
 * no walk is repeated.  For every tangent a at p and u at p', <R a, u> = <a, R^T u>.
 *   mesh_id, face, bary, v   the forward inputs (device, as in sg_exp_map; L = |v|)
 *   end_face, end_dir        the forward outputs for these queries (device)
 *   end_status               the forward status words (device) or NULL (SG_ST_FLIPPED taken
 *                            as 0, exact for orientable meshes)
 *   n_u, u    device float32 [nq][n_u][3] vectors at the end points (0 <= n_u <= 4); their
 *             components normal to the end face are dropped
 *   out_u     device float32 [nq][n_u][3], caller-allocated: the vectors at the start points,
 *             tangent to the start face.  Zero for invalid queries; for a zero vector v the
 *             path is empty and out_u is u projected onto the start face.
 * Asynchronous on `stream`; no scratch.  Errors: SG_ERR_INVALID_ARG (NULL array, n_u out of
 * range), SG_ERR_UNSUPPORTED (opts->precision 40, 48 or 64), SG_ERR_CUDA.
 */
sg_status sg_transport_back(const sg_mesh *m, int64_t nq, const int32_t *mesh_id, const int32_t *face,
                            const float *bary, const float *v, const int32_t *end_face,
                            const float *end_dir, const uint32_t *end_status, int32_t n_u,
                            const float *u, float *out_u, const sg_opts *o, void *stream);

/*
 * sg_exp_map_backward_workspace_size -- bytes of device scratch sg_exp_map_backward needs for
 * nq queries with `estimator` (SG_EST_*) and, if want_grad_V != 0, the vertex gradient: for
 * GFD the column table (16 B per query), the literal-walk task list (12 B per query, reused for
 * the queries whose chords are walked) and the literal walks' restart records (32 B per query);
 * for grad_V a float4 accumulator per vertex and three float4 windows per face (the crossing
 * coefficients of each pair of the face's edges); 12 B per query for an end-barycentric upstream
 * gradient; and the re-walk's length order (5 B per query; not used when o->order carries the
 * forward's order).  Pass it as o->workspace; without it the library allocates stream-ordered
 * scratch itself.
 */
sg_status sg_exp_map_backward_workspace_size(const sg_mesh *m, int32_t estimator, int64_t nq,
                                             int32_t want_grad_V, size_t *bytes);

/* Library version string. */
const char *sg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SGEO_H */
