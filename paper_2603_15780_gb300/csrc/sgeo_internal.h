// sgeo_internal.h -- data layout shared by the host mesh builder and the CUDA kernels.
//
// Device layout of a mesh (all arrays indexed by GLOBAL ids: meshes are concatenated):
//
//   rec   int4[2*nF]   32-byte walk record per face = exactly one L2 sector:
//                      rec[2f]   = { nbr0, nbr1, nbr2, bits(l01) }
//                      rec[2f+1] = { bits(x2x), bits(x2y), bits(il1), bits(il2) }
//                      nbr_k = (g << 3) | (flip << 2) | k'  : face g lies across local edge k
//                      (edge k runs from corner k to corner k+1); in g that edge is local
//                      edge k'; flip = 1 when g lists the edge in the same direction as f
//                      (inconsistent orientation, e.g. a Moebius strip); -1 on the boundary.
//                      Intrinsic 2-D shape in the face's own frame (corner 0 at the origin,
//                      corner 1 on +x, corner 2 in the upper half plane):
//                      P0 = (0,0), P1 = (l01,0), P2 = (x2x,x2y); il1 = 1/|P2-P1|, il2 = 1/|P2|.
//   fv    int4[nF]     global vertex ids of the face corners, .w = mesh index
//   frm   float4[2*nF] the face frame in 3-D: {e1x, e1y, e1z, e2x}, {e2y, e2z, 0, 0} with
//                      e1 = (x1-x0)/|x1-x0|, e2 = n x e1 (the axes of the 2-D record frame);
//                      read by the backward pass (lifting 2-D adjoints, chord walks)
//   half  int4[6*nF]   32-byte half-edge record per (face f, local edge k), id h = 3f + k, in the
//                      edge's own frame (origin at corner k, x along the edge, the face on +y):
//                      half[2h]   = { bits(l), bits(cx), bits(cy), linkR }
//                      half[2h+1] = { linkL, bits(ca), bits(sa), edge }
//                      l = |edge k|, (cx, cy) = corner k+2 (the apex), (ca, sa) = the edge's unit
//                      direction in the face frame (edge frame -> face frame rotation); linkR /
//                      linkL = (h' << 1) | flip for the twin half-edge across edge k+1 (apex side
//                      B -> C) / edge k+2 (C -> A), -1 on the boundary; edge = (e << 1) | o for
//                      an interior edge e (o = 1 when this half-edge is not e's canonical one,
//                      the lower half-edge id), -1 on the boundary.
//   edges int2[nE]     (canonical half-edge, twin half-edge) of each interior edge
//   V     float4[nV]   vertex position (x,y,z); .w = total angle theta(x), negated for boundary
//                      vertices (Sec. 4: theta = sum of incident corner angles)
//   srank int32[nF]    spatial rank of each face: face_off[m] + its position in the Z-order
//                      (Morton order) of the face centroids of mesh m, the key of the start-face
//                      query order (queries of a warp then start in one patch of the surface)
//   face_off int32[n_mesh+1], lref float[n_mesh] (mean edge length per mesh; -1 marks a mesh whose
//                      vertices were moved to a degenerate face, every query on it is rejected)
//
// The walk of a query touches one record per edge crossing (one dependent 32-B gather);
// fv/V are read only at the start, at vertex hits and at the end.
#pragma once
#include <cstdint>
#include <vector>

#include "../../include/sgeo.h"

#define SG_MAX_FACES (1LL << 28)

struct sg_mesh {
    int64_t nV = 0, nF = 0;
    int32_t n_mesh = 0;
    int device = 0;
    int4 *d_rec = nullptr;
    int4 *d_fv = nullptr;
    float4 *d_frm = nullptr;
    int4 *d_half = nullptr;
    int2 *d_edges = nullptr;
    int64_t nE = 0;
    int32_t *d_srank = nullptr;
    float4 *d_V = nullptr;
    int32_t *d_face_off = nullptr;
    float *d_lref = nullptr;
    std::vector<int64_t> face_off, vert_off;
    std::vector<double> lref;
    int64_t device_bytes = 0;
    // scratch of sg_mesh_update_vertices (allocated by its first call)
    double *d_theta = nullptr;
    double *d_lsum = nullptr;
    unsigned long long *d_ecount = nullptr;
    int *d_ndegen = nullptr;
    bool updated = false;
    // FP64 geometry of the full-precision walk (built by its first call, refreshed after an update)
    double *d_rec64 = nullptr;
    double *d_frm64 = nullptr;
    double *d_th64 = nullptr;
    bool geom64_stale = true;
    // double-float half-edge records of the double-float walk, int4[6*nF]: {l, cx} and {cy,
    // linkR, linkL} of each half-edge with every length split into two FP32 words hi + lo
    // (built from the FP64 geometry by the walk's first call, refreshed after an update)
    int4 *d_half48 = nullptr;
    bool half48_stale = true;
};

// host-side builder (mesh_build.cpp); fills the host arrays, returns SG_OK or an error
struct sg_host_mesh {
    std::vector<int4> rec, fv, half;
    std::vector<int2> edges;
    std::vector<int32_t> srank;
    std::vector<float4> frm;
    std::vector<float4> V;
    std::vector<int32_t> face_off;
    std::vector<float> lref;
    std::vector<double> lref64;
    std::vector<int64_t> face_off64, vert_off64;
};

sg_status sg_build_host_mesh(const float *V, const int64_t *v_off, const int32_t *F, const int64_t *f_off,
                             int32_t n_mesh, sg_host_mesh *out);
