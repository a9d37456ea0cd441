/*
 * sgeo_oracle.c -- plain FP64 CPU oracle for the straightest-geodesic exponential map.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct restatement of
 * the method against which the CUDA library is checked.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load it; the library never does.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Formulation: the paper's extrinsic 3-D one (Sec. 4 and App. "Implementation of the
 * Geodesic Step"): points are (face, barycentric) pairs, directions are 3-D unit
 * vectors in the face plane, an edge crossing unfolds the direction about the shared
 * edge, a vertex hit applies the straightest rule (equal left/right angle theta/2).
 *
 *   Alg. "geodesic_step"          -> om_walk(), in-face march
 *   Alg. "transport_over_edge"    -> om_walk(), edge-crossing branch (unfold_apply)
 *   Alg. "transport_over_vertex"  -> om_walk(), vertex-hit branch (fan walk)
 *   Alg. "Parallel Geodesic Tracing CUDA Kernel" -> om_exp_map() (one query per loop
 *                                    iteration, OpenMP over queries)
 *   Eq. "proxy_func" (EP)         -> om_ep_backward()
 *   Eqs. "jv", "jp" (GFD) + App. "Speed-up GFD and EP through batching"
 *                                 -> om_gfd_backward()
 *
 * Readings where the paper is silent or ambiguous (each listed in the design notes):
 *   - the final in-face segment is truncated at the remaining length (Alg. gpu_parallel
 *     loops on L_traced < L_target but Alg. geodesic_step always marches to an edge);
 *   - exact "b_k = 0 / b_k = 1" tests become a vertex snap when the ray passes within
 *     tau_snap * l_ref of a vertex (l_ref = mean edge length); a pass within
 *     tau_near * l_ref is reported as NEAR_VERTEX;
 *   - transport over an edge/vertex happens only when the ray leaves the face there;
 *   - the vertex rule walks the fan from the reversed incoming direction until the
 *     accumulated angle reaches theta/2 and leaves at the excess angle from the entry
 *     edge (both fan directions give the same ray);
 *   - carried vectors keep their signed angle to the direction at a vertex (Sec. 4
 *     "Parallel Transport": the normalised angle is held constant);
 *   - a boundary vertex or boundary edge stops the walk (Sec. 4, original behaviour);
 *   - a start exactly on a vertex must point into the start face's corner; otherwise
 *     the query is INVALID;
 *   - EP uses R = M_p' M_p^T (rotation that takes v/|v| to its transported version).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* status bits (same meaning as the library's per-query status word) */
#define OST_BOUNDARY 1u
#define OST_MAX_STEPS 2u
#define OST_NEAR_VERTEX 4u
#define OST_NEAR_EDGE 8u
#define OST_VERTEX_HIT 16u
#define OST_START_ON_EDGE 64u
#define OST_INVALID 128u
#define OST_HOLE 2048u     /* hole avoidance traced along the boundary */

typedef struct om_mesh {
    int64_t nV, nF;
    double *X;       /* nV*3 */
    int32_t *F;      /* nF*3 */
    int64_t *adj;    /* nF*3: face across the edge OPPOSITE corner k, -1 on the boundary */
    double *theta;   /* nV: sum of corner angles */
    uint8_t *bnd;    /* nV: 1 if the vertex lies on a boundary edge */
    double lref;     /* mean edge length */
} om_mesh;

typedef struct om_opts {
    int32_t max_steps;
    int32_t path_cap;   /* entries per query in out_path (0: none) */
    double tau_snap;    /* vertex snap radius / l_ref */
    double tau_near;    /* near-vertex / near-edge flag radius / l_ref */
    int32_t boundary_mode; /* 0: stop at the boundary (Sec. 4, original rule); 1: hole avoidance */
} om_opts;

/* ------------------------------------------------------------------ small vector ops */
static inline void vsub(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double vdot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void vcross(const double *a, const double *b, double *o) {
    double t0 = a[1] * b[2] - a[2] * b[1], t1 = a[2] * b[0] - a[0] * b[2], t2 = a[0] * b[1] - a[1] * b[0];
    o[0] = t0; o[1] = t1; o[2] = t2;
}
static inline double vnorm(const double *a) { return sqrt(vdot(a, a)); }
static inline void vscale(double *a, double s) { a[0] *= s; a[1] *= s; a[2] *= s; }
static inline void vaxpy(double *y, double s, const double *x) { y[0] += s * x[0]; y[1] += s * x[1]; y[2] += s * x[2]; }
static inline void vcopy(double *o, const double *a) { o[0] = a[0]; o[1] = a[1]; o[2] = a[2]; }
static inline void vnormalize(double *a) { double n = vnorm(a); if (n > 0) vscale(a, 1.0 / n); }

/* unsigned angle between two vectors, atan2(|a x b|, a.b) */
static double vangle(const double *a, const double *b) {
    double c[3];
    vcross(a, b, c);
    return atan2(vnorm(c), vdot(a, b));
}

static inline const double *VX(const om_mesh *m, int64_t v) { return m->X + 3 * v; }

static void face_normal(const om_mesh *m, int64_t f, double *n) {
    const int32_t *t = m->F + 3 * f;
    double e1[3], e2[3];
    vsub(VX(m, t[1]), VX(m, t[0]), e1);
    vsub(VX(m, t[2]), VX(m, t[0]), e2);
    vcross(e1, e2, n);
    vnormalize(n);
}

/* ------------------------------------------------------------------ mesh build */
typedef struct { int32_t a, b; int64_t f; int32_t k; } om_edge;

static int edge_cmp(const void *pa, const void *pb) {
    const om_edge *x = (const om_edge *)pa, *y = (const om_edge *)pb;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    if (x->f != y->f) return x->f < y->f ? -1 : 1;
    return x->k - y->k;
}

void om_mesh_free(om_mesh *m) {
    if (!m) return;
    free(m->X); free(m->F); free(m->adj); free(m->theta); free(m->bnd);
    free(m);
}

/* corner index of vertex v in face f, or -1 */
static int corner_of(const om_mesh *m, int64_t f, int32_t v) {
    const int32_t *t = m->F + 3 * f;
    return t[0] == v ? 0 : t[1] == v ? 1 : t[2] == v ? 2 : -1;
}

/*
 * Builds adjacency (Sec. 4: only triangle adjacencies are stored, no half-edges, so
 * non-orientable meshes work), validates the manifold definition of Sec. 4 (each edge
 * has one or two faces, the faces around a vertex form one fan), and precomputes the
 * vertex total angle theta(x) = sum of incident corner angles (Sec. 4).
 * Returns 0 ok, 1 invalid input, 2 non-manifold, 3 degenerate face.
 */
int om_mesh_build(const double *X, int64_t nV, const int32_t *F, int64_t nF, om_mesh **out) {
    *out = NULL;
    if (nV <= 0 || nF <= 0 || !X || !F) return 1;
    for (int64_t i = 0; i < 3 * nF; ++i)
        if (F[i] < 0 || F[i] >= nV) return 1;
    om_mesh *m = (om_mesh *)calloc(1, sizeof(om_mesh));
    m->nV = nV; m->nF = nF;
    m->X = (double *)malloc(sizeof(double) * 3 * nV);
    m->F = (int32_t *)malloc(sizeof(int32_t) * 3 * nF);
    m->adj = (int64_t *)malloc(sizeof(int64_t) * 3 * nF);
    m->theta = (double *)calloc(nV, sizeof(double));
    m->bnd = (uint8_t *)calloc(nV, 1);
    memcpy(m->X, X, sizeof(double) * 3 * nV);
    memcpy(m->F, F, sizeof(int32_t) * 3 * nF);
    for (int64_t f = 0; f < nF; ++f) {
        const int32_t *t = F + 3 * f;
        if (t[0] == t[1] || t[1] == t[2] || t[0] == t[2]) { om_mesh_free(m); return 3; }
        double e1[3], e2[3], c[3];
        vsub(VX(m, t[1]), VX(m, t[0]), e1);
        vsub(VX(m, t[2]), VX(m, t[0]), e2);
        vcross(e1, e2, c);
        double l = fmax(vdot(e1, e1), vdot(e2, e2));
        if (!(vnorm(c) > 1e-14 * l)) { om_mesh_free(m); return 3; }
    }
    om_edge *E = (om_edge *)malloc(sizeof(om_edge) * 3 * nF);
    for (int64_t f = 0; f < nF; ++f)
        for (int k = 0; k < 3; ++k) {
            int32_t a = F[3 * f + (k + 1) % 3], b = F[3 * f + (k + 2) % 3];
            om_edge *e = &E[3 * f + k];
            e->a = a < b ? a : b; e->b = a < b ? b : a; e->f = f; e->k = k;
        }
    qsort(E, (size_t)(3 * nF), sizeof(om_edge), edge_cmp);
    for (int64_t i = 0; i < 3 * nF; ++i) m->adj[i] = -1;
    double lsum = 0.0;
    int64_t nedge = 0;
    for (int64_t i = 0; i < 3 * nF;) {
        int64_t j = i + 1;
        while (j < 3 * nF && E[j].a == E[i].a && E[j].b == E[i].b) ++j;
        if (j - i > 2) { free(E); om_mesh_free(m); return 2; }
        double d[3];
        vsub(VX(m, E[i].a), VX(m, E[i].b), d);
        lsum += vnorm(d);
        ++nedge;
        if (j - i == 2) {
            if (E[i].f == E[i + 1].f) { free(E); om_mesh_free(m); return 2; }
            m->adj[3 * E[i].f + E[i].k] = E[i + 1].f;
            m->adj[3 * E[i + 1].f + E[i + 1].k] = E[i].f;
        } else {
            m->bnd[E[i].a] = 1; m->bnd[E[i].b] = 1;
        }
        i = j;
    }
    free(E);
    m->lref = lsum / (double)nedge;
    /* corner angles -> theta; incident face counts for the single-fan check */
    int32_t *deg = (int32_t *)calloc(nV, sizeof(int32_t));
    int64_t *anyf = (int64_t *)malloc(sizeof(int64_t) * nV);
    for (int64_t v = 0; v < nV; ++v) anyf[v] = -1;
    for (int64_t f = 0; f < nF; ++f)
        for (int k = 0; k < 3; ++k) {
            int32_t v = F[3 * f + k];
            double a[3], b[3];
            vsub(VX(m, F[3 * f + (k + 1) % 3]), VX(m, v), a);
            vsub(VX(m, F[3 * f + (k + 2) % 3]), VX(m, v), b);
            m->theta[v] += vangle(a, b);
            deg[v]++;
            anyf[v] = f;
        }
    /* single fan: walking around the vertex through adjacency must reach every incident face */
    for (int64_t v = 0; v < nV; ++v) {
        if (deg[v] == 0) continue;
        int64_t seen = 1;
        for (int dir = 0; dir < 2; ++dir) {
            int64_t f = anyf[v];
            int c = corner_of(m, f, (int32_t)v);
            /* edge opposite corner (c+1) contains v and corner c+2; opposite (c+2) contains v and c+1 */
            int opp = dir == 0 ? (c + 1) % 3 : (c + 2) % 3;
            int32_t other = F[3 * f + (dir == 0 ? (c + 2) % 3 : (c + 1) % 3)];
            for (int guard = 0; guard < deg[v] + 1; ++guard) {
                int64_t g = m->adj[3 * f + opp];
                if (g < 0 || g == anyf[v]) break;
                ++seen;
                int cg = corner_of(m, g, (int32_t)v);
                int co = corner_of(m, g, other);
                int third = 3 - cg - co;
                opp = co;  /* edge opposite the shared vertex contains v and the third vertex */
                other = F[3 * g + third];
                f = g;
            }
            if (!m->bnd[v]) break; /* closed fan: one direction covers it */
        }
        if (seen != deg[v]) { free(deg); free(anyf); om_mesh_free(m); return 2; }
    }
    free(deg); free(anyf);
    *out = m;
    return 0;
}

double om_mesh_lref(const om_mesh *m) { return m->lref; }
void om_mesh_theta(const om_mesh *m, double *theta, uint8_t *bnd) {
    memcpy(theta, m->theta, sizeof(double) * m->nV);
    memcpy(bnd, m->bnd, m->nV);
}
void om_mesh_adjacency(const om_mesh *m, int64_t *adj) { memcpy(adj, m->adj, sizeof(int64_t) * 3 * m->nF); }

/* ------------------------------------------------------------------ walk */
typedef struct {
    int64_t f;
    double b[3];       /* barycentric coordinates in f */
    double d[3];       /* unit direction in f's plane */
    double L;          /* remaining length */
    int at_corner;     /* -1, or the corner of f the walker sits on after a vertex hit */
    int entry_opp;     /* -1, or the corner opposite the edge the walker entered through */
} om_state;

typedef struct {
    uint32_t status;
    int32_t ncross, nvert, nsteps;
    uint64_t hash;
    double margin;     /* min line-to-vertex distance / l_ref over visited faces */
    int32_t *path; int32_t path_cap, path_len;
    double *path_pt;   /* optional: the 3-D point at which the walk entered each recorded face */
} om_rec;

static void bary_point(const om_mesh *m, int64_t f, const double *b, double *p) {
    const int32_t *t = m->F + 3 * f;
    p[0] = p[1] = p[2] = 0.0;
    for (int k = 0; k < 3; ++k) vaxpy(p, b[k], VX(m, t[k]));
}

/* the walk enters face s->f at barycentric point s->b: hash it and, when tracing, record the
 * face and the point (the polyline of the traced geodesic is these points, then the end point) */
static inline void rec_face(om_rec *r, const om_mesh *m, const om_state *s) {
    r->hash ^= (uint64_t)(uint32_t)s->f;
    r->hash *= 0x100000001b3ULL;
    if (r->path && r->path_len < r->path_cap) {
        r->path[r->path_len] = (int32_t)s->f;
        if (r->path_pt) bary_point(m, s->f, s->b, r->path_pt + 3 * r->path_len);
    }
    r->path_len++;
}

/* unit vector in the plane spanned by u and h, at angle a from u toward h's side */
static void rotate_toward(const double *u, const double *h, double a, double *o) {
    double uu[3], hh[3];
    vcopy(uu, u); vnormalize(uu);
    vcopy(hh, h); vaxpy(hh, -vdot(h, uu), uu); vnormalize(hh);
    for (int i = 0; i < 3; ++i) o[i] = cos(a) * uu[i] + sin(a) * hh[i];
}

/* map a tangent vector of f across edge {x_a, x_b} into f2 by unfolding about the edge:
 *   x' = <x,e> e - <x,u_f> u_f2,   u_g = unit in-plane normal of the edge pointing into g.
 * This is the rotation of Alg. transport_over_edge by the signed dihedral angle for
 * consistently oriented faces, written without reference to orientation. */
typedef struct { double e[3], uf[3], uf2[3]; } om_unfold;

static void unfold_setup(const om_mesh *m, int32_t va, int32_t vb, int32_t vf, int32_t vf2, om_unfold *U) {
    vsub(VX(m, vb), VX(m, va), U->e); vnormalize(U->e);
    double t[3];
    vsub(VX(m, vf), VX(m, va), t);
    vaxpy(t, -vdot(t, U->e), U->e); vnormalize(t); vcopy(U->uf, t);
    vsub(VX(m, vf2), VX(m, va), t);
    vaxpy(t, -vdot(t, U->e), U->e); vnormalize(t); vcopy(U->uf2, t);
}
static void unfold_apply(const om_unfold *U, double *x) {
    double a = vdot(x, U->e), c = vdot(x, U->uf);
    for (int i = 0; i < 3; ++i) x[i] = a * U->e[i] - c * U->uf2[i];
}

/*
 * Hole avoidance (Sec. 4 "Straightest geodesics": rather than stopping at the boundary, trace
 * along it and resume the straightest walk as soon as possible with the last straightest
 * direction; App. transport_over_vertex / transport_over_edge, hole-avoidance branches).
 * The walker sits on boundary vertex v0 = corner c of face s->f.  D is the direction it had
 * when it reached the boundary (3-D, unit) and n0 the normal of the face it was in; carried
 * vector q has signed angle phi[q] to D about n0 and length wl[q].
 * Readings (the paper describes transport_error but does not define it):
 *   - a face f around v0 receives D when D, projected onto f's plane, points strictly into
 *     f's corner at v0; its error is |<D, n_f>|, the sine of D's angle to the plane; the
 *     receiving face of least error is taken and the walk resumes from v0 inside it;
 *   - when no face receives D, the walk follows the boundary to the next boundary vertex,
 *     spending the edge's length, and tries again there: it keeps its sense along the
 *     boundary (the edge it did not arrive by); at a vertex hit directly by the ray it takes
 *     the boundary edge whose unit direction has the larger dot product with D.  If the
 *     length runs out on an edge the walk ends there, with D projected onto that face as its
 *     direction;
 *   - carried vectors keep their signed angle to the direction;
 *   - a decision closer than tau_near (a wedge sine, the difference of the two least errors,
 *     or of the two edge cosines) is flagged NEAR_VERTEX.
 * Returns 1 when the walk resumes (s on the corner of the receiving face), 0 when it ended.
 */
static int om_hole(const om_mesh *m, om_state *s, int c, int32_t came_from, int nw, double *w,
                   const double *phi, const double *wl, const double *D, const om_opts *o, om_rec *r) {
    const double tau = o->tau_near;
    int flip_ref = 0;   /* orientation of s->f relative to the face the boundary was reached in */
    r->status |= OST_HOLE;
    while (1) {
        const int64_t f0 = s->f;
        const int32_t v0 = m->F[3 * f0 + c];
        const double *x0 = VX(m, v0);
        int64_t fan[512];
        int fflip[512], nf = 0;
        int64_t bface[2];
        int32_t bvert[2];
        int bflip[2], nb = 0;
        fan[nf] = f0; fflip[nf] = 0; nf++;
        for (int dir = 0; dir < 2; ++dir) {
            int64_t cur = f0;
            int cc = c, fl = 0;
            int opp = dir == 0 ? (cc + 2) % 3 : (cc + 1) % 3;  /* the edge (v0, corner 3-cc-opp) */
            for (int guard = 0; guard < 512; ++guard) {
                const int32_t vs = m->F[3 * cur + (3 - cc - opp)];
                const int64_t g = m->adj[3 * cur + opp];
                if (g < 0) {
                    if (nb < 2) { bface[nb] = cur; bvert[nb] = vs; bflip[nb] = fl; nb++; }
                    break;
                }
                if (g == f0 || nf >= 512) break;
                const int cg = corner_of(m, g, v0), sg = corner_of(m, g, vs), cs = corner_of(m, cur, vs);
                /* a consistent orientation lists the shared edge in opposite directions */
                if ((((cc + 1) % 3) == cs) == (((cg + 1) % 3) == sg)) fl ^= 1;
                fan[nf] = g; fflip[nf] = fl; nf++;
                cur = g; cc = cg; opp = sg;
            }
        }
        /* the receiving face of least error */
        int best = -1;
        double best_err = INFINITY, second = INFINITY, bu[3] = {0, 0, 0};
        for (int i = 0; i < nf; ++i) {
            const int64_t g = fan[i];
            const int cg = corner_of(m, g, v0);
            double ng[3], u[3], ea[3], eb[3], t[3];
            face_normal(m, g, ng);
            vcopy(u, D);
            vaxpy(u, -vdot(D, ng), ng);
            const double lu = vnorm(u);
            if (!(lu > 1e-12)) continue;
            vscale(u, 1.0 / lu);
            vsub(VX(m, m->F[3 * g + (cg + 1) % 3]), x0, ea);
            vsub(VX(m, m->F[3 * g + (cg + 2) % 3]), x0, eb);
            vcross(ea, u, t);
            const double sa = vdot(t, ng) / vnorm(ea);
            vcross(u, eb, t);
            const double sb = vdot(t, ng) / vnorm(eb);
            const double mg = fmin(sa, sb);
            if (fabs(mg) < tau) r->status |= OST_NEAR_VERTEX;
            if (!(mg > 0.0)) continue;
            const double err = fabs(vdot(D, ng));
            if (err < best_err) { second = best_err; best_err = err; best = i; vcopy(bu, u); }
            else if (err < second) second = err;
        }
        if (best >= 0) {
            if (second - best_err < tau) r->status |= OST_NEAR_VERTEX;
            const int64_t g = fan[best];
            const int cg = corner_of(m, g, v0);
            double ng[3], cu[3];
            face_normal(m, g, ng);
            if (flip_ref ^ fflip[best]) vscale(ng, -1.0);
            vcross(ng, bu, cu);
            for (int q = 0; q < nw; ++q)
                for (int i = 0; i < 3; ++i) w[3 * q + i] = wl[q] * (cos(phi[q]) * bu[i] + sin(phi[q]) * cu[i]);
            s->f = g;
            for (int i = 0; i < 3; ++i) s->b[i] = i == cg ? 1.0 : 0.0;
            vcopy(s->d, bu);
            s->at_corner = cg;
            s->entry_opp = -1;
            rec_face(r, m, s);
            return 1;
        }
        /* no face receives D: follow the boundary edge that agrees best with D */
        if (nb == 0) { r->status |= OST_BOUNDARY; return 0; }
        int k = 0;
        double dk[2] = {-INFINITY, -INFINITY};
        for (int i = 0; i < nb; ++i) {
            double e[3];
            vsub(VX(m, bvert[i]), x0, e);
            dk[i] = vdot(D, e) / vnorm(e);
        }
        if (nb == 2) {
            if (came_from >= 0) {
                k = bvert[0] == came_from ? 1 : 0;
            } else {
                k = dk[1] > dk[0] ? 1 : 0;
                if (fabs(dk[1] - dk[0]) < tau) r->status |= OST_NEAR_VERTEX;
            }
        }
        const int64_t fb = bface[k];
        const int cb = corner_of(m, fb, v0), co = corner_of(m, fb, bvert[k]);
        flip_ref ^= bflip[k];
        if (fb != s->f) {
            s->f = fb;
            for (int i = 0; i < 3; ++i) s->b[i] = i == cb ? 1.0 : 0.0;
            rec_face(r, m, s);
        }
        if (r->nsteps >= o->max_steps) {
            r->status |= OST_MAX_STEPS;
            for (int i = 0; i < 3; ++i) s->b[i] = i == cb ? 1.0 : 0.0;
            return 0;
        }
        r->nsteps++;
        double e[3];
        vsub(VX(m, bvert[k]), x0, e);
        const double le = vnorm(e);
        if (s->L <= le) {
            const double t = s->L / le;
            for (int i = 0; i < 3; ++i) s->b[i] = i == cb ? 1.0 - t : i == co ? t : 0.0;
            s->L = 0.0;
            double nbv[3], u[3], cu[3];
            face_normal(m, fb, nbv);
            vcopy(u, D);
            vaxpy(u, -vdot(D, nbv), nbv);
            if (vnorm(u) > 1e-12) vnormalize(u); else { vcopy(u, e); vscale(u, 1.0 / le); }
            vcopy(s->d, u);
            if (flip_ref) vscale(nbv, -1.0);
            vcross(nbv, u, cu);
            for (int q = 0; q < nw; ++q)
                for (int i = 0; i < 3; ++i) w[3 * q + i] = wl[q] * (cos(phi[q]) * u[i] + sin(phi[q]) * cu[i]);
            s->at_corner = -1;
            s->entry_opp = -1;
            return 0;
        }
        s->L -= le;
        for (int i = 0; i < 3; ++i) s->b[i] = i == co ? 1.0 : 0.0;
        c = co;
        came_from = v0;
    }
}

/* signed angles (about the normal n of the current face) and lengths of the carried vectors
 * relative to the direction, kept through a hole-avoidance detour */
static void carried_angles(const om_state *s, const double *n, int nw, const double *w, double *phi, double *wl) {
    for (int q = 0; q < nw; ++q) {
        double c[3];
        vcross(s->d, w + 3 * q, c);
        phi[q] = atan2(vdot(c, n), vdot(s->d, w + 3 * q));
        wl[q] = vnorm(w + 3 * q);
    }
}

/*
 * One query: Alg. "Parallel Geodesic Tracing CUDA Kernel" body with Alg. geodesic_step,
 * transport_over_edge and transport_over_vertex (black lines), FP64.
 * w (nw carried vectors, 3-D) is transported alongside.
 */
static void om_walk(const om_mesh *m, om_state *s, int nw, double *w, const om_opts *o, om_rec *r) {
    const double snap = o->tau_snap * m->lref, near = o->tau_near * m->lref;
    r->margin = INFINITY;
    rec_face(r, m, s);
    while (1) {
        if (r->nsteps >= o->max_steps) { r->status |= OST_MAX_STEPS; return; }
        r->nsteps++;
        const int32_t *t = m->F + 3 * s->f;
        const double *x[3] = {VX(m, t[0]), VX(m, t[1]), VX(m, t[2])};
        double n[3], e1[3], e2[3], p[3];
        vsub(x[1], x[0], e1); vsub(x[2], x[0], e2);
        vcross(e1, e2, n);
        double area2 = vnorm(n);
        vscale(n, 1.0 / area2);
        bary_point(m, s->f, s->b, p);
        /* line-to-vertex distances of this face's vertices (margin bookkeeping) */
        double dist[3];
        for (int k = 0; k < 3; ++k) {
            double q[3], c[3];
            vsub(x[k], p, q);
            vcross(s->d, q, c);
            dist[k] = vnorm(c);
        }
        /* barycentric form of d: bd_i = grad(b_i) . d, grad(b_i) = n x (x_{i+2} - x_{i+1}) / (2A) */
        double bd[3];
        for (int i = 0; i < 3; ++i) {
            double ed[3], g[3];
            vsub(x[(i + 2) % 3], x[(i + 1) % 3], ed);
            vcross(n, ed, g);
            bd[i] = vdot(g, s->d) / area2;
        }
        /* exit parameter lambda = min{-b_i / bd_i > 0} over admissible edges (edge i = opposite corner i) */
        int istar = -1;
        double tstar = INFINITY;
        for (int i = 0; i < 3; ++i) {
            if (s->at_corner >= 0 && i != s->at_corner) continue;  /* from a corner only the opposite edge */
            if (s->entry_opp == i) continue;                         /* never leave through the entry edge */
            if (!(bd[i] < 0.0)) continue;
            double ti = fmax(s->b[i], 0.0) / (-bd[i]);
            if (ti < tstar) { tstar = ti; istar = i; }
        }
        if (istar < 0) { r->status |= OST_INVALID; return; } /* cannot happen for a tangent direction */
        int j = (istar + 1) % 3, k2 = (istar + 2) % 3;
        /* vertex snap: the ray passes (essentially) through an endpoint of the exit edge */
        int hit = -1;
        if (dist[j] <= snap || dist[k2] <= snap) hit = dist[j] <= dist[k2] ? j : k2;
        for (int q = 0; q < 3; ++q) {
            if (q == s->at_corner || q == hit) continue;
            double mq = dist[q] / m->lref;
            if (mq < r->margin) r->margin = mq;
        }
        if (tstar >= s->L) {
            /* final, truncated segment (reading: stop inside the face once the length is used) */
            for (int i = 0; i < 3; ++i) s->b[i] += s->L * bd[i];
            s->L = 0.0;
            /* NEAR_EDGE: the end point lies within tau_near * l_ref of an edge of its face
             * (distance to the edge opposite corner i = b_i * 2A / |edge_i|) */
            for (int i = 0; i < 3; ++i) {
                double ed[3];
                vsub(x[(i + 2) % 3], x[(i + 1) % 3], ed);
                if (s->b[i] * area2 / vnorm(ed) <= near) r->status |= OST_NEAR_EDGE;
            }
            return;
        }
        s->L -= tstar;
        if (hit >= 0) {
            /* ---------------- vertex hit: Alg. transport_over_vertex */
            int32_t v0 = t[hit];
            r->status |= OST_VERTEX_HIT;
            r->nvert++;
            if (m->bnd[v0]) {
                for (int i = 0; i < 3; ++i) s->b[i] = i == hit ? 1.0 : 0.0;
                if (!o->boundary_mode) { r->status |= OST_BOUNDARY; return; }
                double phi[8], wl[8], D[3];
                carried_angles(s, n, nw, w, phi, wl);
                vcopy(D, s->d);
                if (om_hole(m, s, hit, -1, nw, w, phi, wl, D, o, r)) continue;
                return;
            }
            double half = 0.5 * m->theta[v0];
            double rdir[3] = {-s->d[0], -s->d[1], -s->d[2]};
            /* signed angles of the carried vectors to the incoming direction (normal of f) */
            double phi[8], wl[8];
            for (int q = 0; q < nw; ++q) {
                double c[3];
                vcross(s->d, w + 3 * q, c);
                phi[q] = atan2(vdot(c, n), vdot(s->d, w + 3 * q));
                wl[q] = vnorm(w + 3 * q);
            }
            /* walk the fan toward the corner (hit+1) side */
            int64_t cur = s->f;
            int32_t va = t[(hit + 1) % 3];
            double ea[3];
            vsub(VX(m, va), VX(m, v0), ea);
            double A = vangle(rdir, ea);
            double dout[3];
            int64_t fexit;
            int flips = 0;
            if (A >= half) {
                rotate_toward(rdir, ea, half, dout);
                fexit = cur;
            } else {
                int guard = 0;
                while (1) {
                    int ca = corner_of(m, cur, va), c0 = corner_of(m, cur, v0);
                    int opp = 3 - ca - c0;
                    int64_t g = m->adj[3 * cur + opp];
                    if (g < 0 || ++guard > 100000) { r->status |= OST_BOUNDARY; for (int i = 0; i < 3; ++i) s->b[i] = i == hit ? 1.0 : 0.0; return; }
                    int ga = corner_of(m, g, va), g0 = corner_of(m, g, v0);
                    int gz = 3 - ga - g0;
                    /* consistent orientation: the shared edge appears reversed in the two faces */
                    if ((c0 + 1) % 3 == ca ? (g0 + 1) % 3 == ga : (ga + 1) % 3 == g0) flips ^= 1;
                    int32_t vz = m->F[3 * g + gz];
                    double ez[3];
                    vsub(VX(m, vz), VX(m, v0), ez);
                    vsub(VX(m, va), VX(m, v0), ea);
                    double gam = vangle(ea, ez);
                    if (A + gam >= half) {
                        rotate_toward(ea, ez, half - A, dout);
                        fexit = g;
                        break;
                    }
                    A += gam;
                    cur = g;
                    va = vz;
                }
            }
            double n2[3];
            face_normal(m, fexit, n2);
            if (flips) vscale(n2, -1.0);
            for (int q = 0; q < nw; ++q) {
                double c[3];
                vcross(n2, dout, c);
                for (int i = 0; i < 3; ++i) w[3 * q + i] = wl[q] * (cos(phi[q]) * dout[i] + sin(phi[q]) * c[i]);
            }
            vcopy(s->d, dout);
            s->f = fexit;
            int cc = corner_of(m, fexit, v0);
            for (int i = 0; i < 3; ++i) s->b[i] = i == cc ? 1.0 : 0.0;
            s->at_corner = cc;
            s->entry_opp = -1;
            rec_face(r, m, s);
            continue;
        }
        /* ---------------- edge crossing: Alg. transport_over_edge */
        double bx[3];
        for (int i = 0; i < 3; ++i) bx[i] = s->b[i] + tstar * bd[i];
        bx[istar] = 0.0;
        double sj = fmax(bx[j], 0.0), sk = fmax(bx[k2], 0.0), ss = sj + sk;
        sj /= ss; sk /= ss;
        int64_t g = m->adj[3 * s->f + istar];
        if (g < 0) {
            s->b[istar] = 0.0; s->b[j] = sj; s->b[k2] = sk;
            if (!o->boundary_mode) { r->status |= OST_BOUNDARY; return; }
            /* hole avoidance, edge branch: slide along the boundary edge toward the endpoint
             * the direction points to (corner k2 when <d, x_k2 - x_j> >= 0, else corner j) */
            double e[3];
            vsub(x[k2], x[j], e);
            const double le = vnorm(e), de = vdot(s->d, e) / le;
            if (fabs(de) < o->tau_near) r->status |= OST_NEAR_VERTEX;
            const int tgt = de >= 0.0 ? k2 : j;
            const double dist = (tgt == k2 ? sj : sk) * le;   /* distance from the hit point to the target */
            r->status |= OST_HOLE;
            if (s->L <= dist) {
                const double tmv = s->L / le;
                if (tgt == k2) { s->b[k2] += tmv; s->b[j] -= tmv; } else { s->b[j] += tmv; s->b[k2] -= tmv; }
                s->L = 0.0;
                return;
            }
            s->L -= dist;
            r->nsteps++;
            for (int i = 0; i < 3; ++i) s->b[i] = i == tgt ? 1.0 : 0.0;
            double phi[8], wl[8], D[3];
            carried_angles(s, n, nw, w, phi, wl);
            vcopy(D, s->d);
            if (om_hole(m, s, tgt, t[tgt == k2 ? j : k2], nw, w, phi, wl, D, o, r)) continue;
            return;
        }
        int32_t vj = t[j], vk = t[k2];
        int gj = corner_of(m, g, vj), gk = corner_of(m, g, vk);
        int gz = 3 - gj - gk;
        om_unfold U;
        unfold_setup(m, vj, vk, t[istar], m->F[3 * g + gz], &U);
        unfold_apply(&U, s->d);
        vnormalize(s->d);
        for (int q = 0; q < nw; ++q) unfold_apply(&U, w + 3 * q);
        s->f = g;
        s->b[gj] = sj; s->b[gk] = sk; s->b[gz] = 0.0;
        s->entry_opp = gz;
        s->at_corner = -1;
        r->ncross++;
        rec_face(r, m, s);
    }
}

/* initialise_trace (Alg. gpu_parallel): normalise b, project v and w onto the face plane,
 * L = |v| (or the given length), d = v/|v|.  Returns 0 if the query is valid. */
static int om_init(const om_mesh *m, int64_t f, const double *b, const double *v, const double *len,
                   int nw, const double *w_in, double *w, om_state *s, uint32_t *status) {
    s->f = f; s->at_corner = -1; s->entry_opp = -1;
    if (f < 0 || f >= m->nF) return 1;
    double sb = b[0] + b[1] + b[2];
    if (!(fabs(sb - 1.0) <= 1e-6) || b[0] < -1e-12 || b[1] < -1e-12 || b[2] < -1e-12) return 1;
    for (int k = 0; k < 3; ++k) s->b[k] = fmax(b[k], 0.0) / sb;
    double n[3];
    face_normal(m, f, n);
    double vp[3];
    vcopy(vp, v);
    vaxpy(vp, -vdot(vp, n), n);
    double L = vnorm(vp);
    for (int q = 0; q < nw; ++q) {
        vcopy(w + 3 * q, w_in + 3 * q);
        vaxpy(w + 3 * q, -vdot(w + 3 * q, n), n);
    }
    if (!(L <= 1e300)) return 1;  /* a non-finite vector is invalid input */
    if (len) {
        if (!(*len >= 0.0 && *len <= 1e300)) return 1;
        if (L == 0.0 && *len > 0.0) return 1;
        s->L = *len;
    } else {
        s->L = L;
    }
    if (L > 0.0) { vcopy(s->d, vp); vscale(s->d, 1.0 / L); }
    else { s->d[0] = s->d[1] = s->d[2] = 0.0; }
    int zeros = (s->b[0] == 0.0) + (s->b[1] == 0.0) + (s->b[2] == 0.0);
    if (zeros) *status |= OST_START_ON_EDGE;
    if (zeros == 2 && s->L > 0.0) {
        /* on a vertex: the direction must point into this face's corner */
        int c = s->b[0] == 1.0 ? 0 : s->b[1] == 1.0 ? 1 : 2;
        const int32_t *t = m->F + 3 * f;
        double a[3], bb[3], ca[3], cb[3];
        vsub(VX(m, t[(c + 1) % 3]), VX(m, t[c]), a);
        vsub(VX(m, t[(c + 2) % 3]), VX(m, t[c]), bb);
        vcross(a, s->d, ca);
        vcross(s->d, bb, cb);
        if (!(vdot(ca, n) > 0.0 && vdot(cb, n) > 0.0)) return 1;
        s->at_corner = c;
    }
    return 0;
}

static void om_output(const om_mesh *m, const om_state *s, int nw, const double *w, const om_rec *r,
                      int64_t i, int32_t *of, double *ob, double *op, double *od, double *ow,
                      uint32_t *ost, int32_t *onc, int32_t *onv, uint64_t *oh, double *omg) {
    if (of) of[i] = (int32_t)s->f;
    if (ob) for (int k = 0; k < 3; ++k) ob[3 * i + k] = s->b[k];
    if (op) bary_point(m, s->f, s->b, op + 3 * i);
    if (od) vcopy(od + 3 * i, s->d);
    if (ow) memcpy(ow + 3 * nw * i, w, sizeof(double) * 3 * nw);
    if (ost) ost[i] = r->status;
    if (onc) onc[i] = r->ncross;
    if (onv) onv[i] = r->nvert;
    if (oh) oh[i] = r->hash;
    if (omg) omg[i] = r->margin;
}

static void default_opts(const om_opts *o, om_opts *out) {
    out->max_steps = (o && o->max_steps > 0) ? o->max_steps : (1 << 20);
    out->path_cap = o ? o->path_cap : 0;
    out->tau_snap = (o && o->tau_snap > 0) ? o->tau_snap : 1e-12;
    out->tau_near = (o && o->tau_near > 0) ? o->tau_near : 1e-4;
    out->boundary_mode = o ? o->boundary_mode : 0;
}

/* single walk from a fully specified start; used by the batch entry and by GFD */
static void om_query(const om_mesh *m, int64_t f, const double *b, const double *v, const double *len,
                     int nw, const double *w_in, double *w, om_state *s, om_rec *r, const om_opts *o) {
    memset(r, 0, sizeof(*r));
    r->hash = 0xcbf29ce484222325ULL;
    r->margin = INFINITY;
    if (om_init(m, f, b, v, len, nw, w_in, w, s, &r->status)) {
        r->status |= OST_INVALID;
        if (f < 0 || f >= m->nF) s->f = 0;
        return;
    }
    if (s->L > 0.0) om_walk(m, s, nw, w, o, r);  /* Exp_p(0) = p: nothing to walk */
    if (r->margin < o->tau_near) r->status |= OST_NEAR_VERTEX;
}

void om_exp_map(const om_mesh *m, int64_t nq, const int32_t *face, const double *bary, const double *v,
                const double *length, int32_t nw, const double *w,
                int32_t *out_face, double *out_bary, double *out_pos, double *out_dir, double *out_w,
                uint32_t *out_status, int32_t *out_ncross, int32_t *out_nvert, uint64_t *out_hash,
                double *out_margin, int32_t *out_path, double *out_path_pt, int32_t *out_path_len,
                const om_opts *opts, int nthreads) {
    om_opts o;
    default_opts(opts, &o);
    if (nw > 8) nw = 8;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t i = 0; i < nq; ++i) {
        om_state s;
        om_rec r;
        double wl[24];
        memset(&r, 0, sizeof r);
        om_query(m, face[i], bary + 3 * i, v + 3 * i, length ? length + i : NULL, nw, w ? w + 3 * nw * i : NULL, wl, &s, &r, &o);
        (void)out_path;
        om_output(m, &s, nw, wl, &r, i, out_face, out_bary, out_pos, out_dir, out_w, out_status, out_ncross,
                  out_nvert, out_hash, out_margin);
    }
    if (out_path && o.path_cap > 0) {
        /* second, serial pass that records the face sequence (debug / small cases only) */
        for (int64_t i = 0; i < nq; ++i) {
            om_state s;
            om_rec r;
            double wl[24];
            memset(&r, 0, sizeof r);
            int32_t *pp = out_path + (int64_t)o.path_cap * i;
            for (int k = 0; k < o.path_cap; ++k) pp[k] = -1;
            r.path = pp; r.path_cap = o.path_cap;
            r.path_pt = out_path_pt ? out_path_pt + 3 * (int64_t)o.path_cap * i : NULL;
            if (r.path_pt) for (int k = 0; k < 3 * o.path_cap; ++k) r.path_pt[k] = 0.0;
            r.hash = 0xcbf29ce484222325ULL;
            if (out_path_len) out_path_len[i] = 0;
            if (om_init(m, face[i], bary + 3 * i, v + 3 * i, length ? length + i : NULL, nw, w ? w + 3 * nw * i : NULL, wl, &s, &r.status)) continue;
            if (s.L > 0.0) om_walk(m, &s, nw, wl, &o, &r);  /* Exp_p(0) = p: no face sequence */
            if (out_path_len) out_path_len[i] = r.path_len;
        }
    }
}

/* ------------------------------------------------------------------ differentiation */
/* start frame pieces shared by EP and GFD: n (start normal), e_par = v/|v|, e_perp = n x e_par */
static int start_frame(const om_mesh *m, int64_t f, const double *v, double *n, double *ep, double *eq, double *L) {
    face_normal(m, f, n);
    double vp[3];
    vcopy(vp, v);
    vaxpy(vp, -vdot(vp, n), n);
    *L = vnorm(vp);
    if (!(*L > 0.0)) return 1;
    vcopy(ep, vp); vscale(ep, 1.0 / *L);
    vcross(n, ep, eq);
    return 0;
}

/*
 * EP backward, Eq. "proxy_func": phi(p, v) = R (p + v) + t with R = M_p' M_p^T,
 * M_p = [v/|v|, n x v/|v|, n] at the start and M_p' the same frame transported to the
 * end point.  J^v = R, J^p zeroed.  The frame is transported by walking the query and
 * carrying e_perp = n x v/|v| as a parallel-transported vector (so the end frame is
 * [d', Pi(e_perp), d' x Pi(e_perp)], which also holds on non-orientable meshes).  The VJP
 * restricted to the start tangent plane (the input v is projected there) is
 *   grad_v = e_par <d', g> + e_perp <Pi(e_perp), g>,   grad_p = 0, grad_bary = 0.
 */
void om_ep_backward(const om_mesh *m, int64_t nq, const int32_t *face, const double *bary, const double *v,
                    const double *g_pos, double *grad_v, uint32_t *out_flags, const om_opts *opts, int nthreads) {
    om_opts o;
    default_opts(opts, &o);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t i = 0; i < nq; ++i) {
        double n[3], ep[3], eq[3], L, wq[3];
        for (int k = 0; k < 3; ++k) grad_v[3 * i + k] = 0;
        if (start_frame(m, face[i], v + 3 * i, n, ep, eq, &L)) { if (out_flags) out_flags[i] = OST_INVALID; continue; }
        om_state s;
        om_rec r;
        om_query(m, face[i], bary + 3 * i, v + 3 * i, NULL, 1, eq, wq, &s, &r, &o);
        double a = vdot(s.d, g_pos + 3 * i), b = vdot(wq, g_pos + 3 * i);
        for (int k = 0; k < 3; ++k) grad_v[3 * i + k] = a * ep[k] + b * eq[k];
        if (out_flags) out_flags[i] = r.status;
    }
}

/* projector onto the plane of face f applied to x */
static void project_plane(const om_mesh *m, int64_t f, double *x) {
    double n[3];
    face_normal(m, f, n);
    vaxpy(x, -vdot(x, n), n);
}

/*
 * GFD backward, Eqs. "jv" and "jp" with the batching of App. "Speed-up GFD and EP through
 * batching", evaluated by independent FP64 walks:
 *   round 1: Exp(p, v), Exp(p, v + eps_v e_perp), Exp(p, eps_p e_u), Exp(p, eps_p e_v)
 *   round 2: Exp(p', Pi(eps_v e_par)), Exp(p_u, v_u), Exp(p_v, v_v)
 * Columns are (Exp(.) - p') / eps projected onto the end-face plane (M M^dagger = the
 * orthogonal projector onto span(e_u', e_v')).  VJP:
 *   grad_v = e_par <c_par, g> + e_perp <c_perp, g>
 *   grad_p = M (M^T M)^{-1} [<c_u, g>, <c_v, g>],  M = [e_u e_v] of the start face
 *   grad_bary_k = <grad_p, x_k>
 * out_flags (optional) receives, per query, the OR of the status words of all walks.
 */
void om_gfd_backward(const om_mesh *m, int64_t nq, const int32_t *face, const double *bary, const double *v,
                     double eps_v, double eps_p, const double *g_pos,
                     double *grad_v, double *grad_p, double *grad_bary, uint32_t *out_flags,
                     const om_opts *opts, int nthreads) {
    om_opts o;
    default_opts(opts, &o);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < nq; ++i) {
        const double *g = g_pos + 3 * i;
        double n[3], ep[3], eq[3], L;
        for (int k = 0; k < 3; ++k) { grad_v[3 * i + k] = 0; grad_p[3 * i + k] = 0; grad_bary[3 * i + k] = 0; }
        uint32_t fl = 0;
        if (start_frame(m, face[i], v + 3 * i, n, ep, eq, &L)) { if (out_flags) out_flags[i] = OST_INVALID; continue; }
        om_state s0, s;
        om_rec r;
        double wv[3], pend[3], pcur[3], col[3];
        /* base walk, carrying v itself so that Pi(e_par) is the end direction */
        om_query(m, face[i], bary + 3 * i, v + 3 * i, NULL, 0, NULL, wv, &s0, &r, &o);
        fl |= r.status;
        bary_point(m, s0.f, s0.b, pend);
        /* perpendicular column: Exp(p, v + eps e_perp) */
        double vq[3];
        vcopy(vq, v + 3 * i); vaxpy(vq, eps_v, eq);
        om_query(m, face[i], bary + 3 * i, vq, NULL, 0, NULL, wv, &s, &r, &o);
        fl |= r.status;
        bary_point(m, s.f, s.b, pcur);
        vsub(pcur, pend, col); vscale(col, 1.0 / eps_v); project_plane(m, s0.f, col);
        double gq = vdot(col, g);
        /* parallel column: Exp(p', Pi(eps e_par)) = short walk from the end point */
        double vp2[3];
        vcopy(vp2, s0.d); vscale(vp2, eps_v);
        om_query(m, s0.f, s0.b, vp2, NULL, 0, NULL, wv, &s, &r, &o);
        fl |= r.status;
        bary_point(m, s.f, s.b, pcur);
        vsub(pcur, pend, col); vscale(col, 1.0 / eps_v); project_plane(m, s0.f, col);
        double gp = vdot(col, g);
        for (int k = 0; k < 3; ++k) grad_v[3 * i + k] = gp * ep[k] + gq * eq[k];
        /* position columns: p_u = Exp(p, eps e_u) carrying v, then Exp(p_u, v_u) */
        const int32_t *t = m->F + 3 * face[i];
        double eu[3], ev[3], gu[2];
        vsub(VX(m, t[1]), VX(m, t[0]), eu); vnormalize(eu);
        vsub(VX(m, t[2]), VX(m, t[0]), ev); vnormalize(ev);
        for (int c = 0; c < 2; ++c) {
            double step[3], vt[3];
            vcopy(step, c == 0 ? eu : ev); vscale(step, eps_p);
            om_state s1;
            om_query(m, face[i], bary + 3 * i, step, NULL, 1, v + 3 * i, vt, &s1, &r, &o);
            fl |= r.status;
            om_query(m, s1.f, s1.b, vt, NULL, 0, NULL, wv, &s, &r, &o);
            fl |= r.status;
            bary_point(m, s.f, s.b, pcur);
            vsub(pcur, pend, col); vscale(col, 1.0 / eps_p); project_plane(m, s0.f, col);
            gu[c] = vdot(col, g);
        }
        /* grad_p = M (M^T M)^{-1} [gu0, gu1] */
        double a11 = vdot(eu, eu), a12 = vdot(eu, ev), a22 = vdot(ev, ev);
        double det = a11 * a22 - a12 * a12;
        double c0 = (a22 * gu[0] - a12 * gu[1]) / det, c1 = (-a12 * gu[0] + a11 * gu[1]) / det;
        for (int k = 0; k < 3; ++k) grad_p[3 * i + k] = c0 * eu[k] + c1 * ev[k];
        for (int k = 0; k < 3; ++k) grad_bary[3 * i + k] = vdot(grad_p + 3 * i, VX(m, t[k]));
        if (out_flags) out_flags[i] = fl;
    }
}
