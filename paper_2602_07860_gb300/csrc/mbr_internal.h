// mbr_internal.h -- launch wrappers shared between the kernel translation units and the C ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mbr_common.cuh"

namespace mbr {

struct RasterParams;
struct WorkQueue;

void launch_face_normals(const float* verts, const int32_t* faces, int F, int V, float* nacc, int* status,
                         cudaStream_t st);
void launch_xform(const float* verts, const float* nacc, int V, const SlotXform* xf, int n_slots, float th,
                  float4* pos, float4* nrm, cudaStream_t st);
void launch_setup(const float4* pos, const int32_t* faces, int F, int V, const int2* set_slots, int n_sets,
                  float znear, TriRec* recs, cudaStream_t st);
// both bin sets of a render: [0] core (undilated), [1] soft (dilated by r_soft)
struct BinTargets {
  int32_t* counts_or_cursor[2];  // count pass: zeroed counts; fill pass: zeroed cursors (slot = offset + cursor)
  int32_t* list[2];              // fill pass: CSR face lists
  const int32_t* off[2];         // fill pass: CSR offsets
  int cap[2];                    // fill pass: list capacities
};
void launch_bin(bool fill, const TriRec* recs, int F, const Group* groups, int G, int W, int H, int tw, int th,
                int tiles_x, int n_tiles, float r_core, float r_soft, const BinTargets& t, int* status,
                cudaStream_t st);
// exclusive scans of the core and soft bin counts in one set of launches; the counts are zeroed
// (they become the fill pass's cursors) and total[q] (if set) receives out[q][n]
struct ScanPair {
  int32_t* in[2];    // [n] counts
  int32_t* out[2];   // [n + 1] offsets
  int32_t* sums[2];  // [scan_temp_ints(n)] scratch
  int32_t* total;    // [2] or null
  int n;
};
size_t scan_temp_ints(int n);
// zero up to four buffers of 32-bit words in one launch (null entries are skipped)
struct ZeroList {
  int32_t* p[4];
  size_t n[4];
};
void launch_zero(const ZeroList& z, cudaStream_t st);
int launch_scan_pair(const ScanPair& sp, cudaStream_t st);  // returns the kernels launched
// persistent raster launches; kind 0 plain only, 1 fast only, 2 mixed, plus kKindExt for the
// kernels with the variants (texture colours, perspective-correct weights, sigmoid probability)
constexpr int kKindMask = 3, kKindExt = 4;
void launch_raster_fwd(const WorkQueue& Q, int tile, int spt, int kind, int grid, cudaStream_t st);
int persistent_grid_fwd(int num_sms, int tile, int spt, int kind);
int persistent_grid_bwd(int num_sms, int tile, int spt, int kind);
// LPT visiting order of a render's units (patch x group split) from its bin offsets (one launch);
// scratch holds unit_order_ints(n_units) ints; cost_zero, cost_zero2 (if set, [n_units]) are
// cleared
size_t unit_order_ints(int n_units);
void launch_unit_order(const int32_t* core_off, const int32_t* soft_off, int G, int n_tiles, int tile, int n_split,
                       int n_units, int32_t* order, int32_t* scratch, int32_t* cost_zero, int32_t* cost_zero2,
                       cudaStream_t st);
// the same from a measured cost per unit (a raster's own measurement); cost_zero (may be cost)
// and cost_zero2 (if set) are cleared after reading
void launch_unit_order_measured(const int32_t* cost, int n_units, int32_t* order, int32_t* scratch,
                                int32_t* cost_zero, int32_t* cost_zero2, cudaStream_t st);
// measurement build of the forward raster (16 x 16 tiles): counts soft terms / covered samples
void launch_raster_count(const WorkQueue& Q, int spt, int kind, int grid, cudaStream_t st);
void launch_count(const TriRec* recs, int F, const Group* groups, int G, int W, int H, float r,
                  unsigned long long* out, cudaStream_t st);

// FP32 peak measurement: one launch of FMA chains filling every SM; returns the flops it executes
double launch_fma_peak(int num_sms, int iters, float* sink, cudaStream_t st);

void launch_raster_bwd(const WorkQueue& Q, int tile, int spt, int kind, int grid, cudaStream_t st);
void launch_slot_chain(const float* verts, const float* nacc, int V, const SlotXform* xf, int n_slots, float th,
                       const float4* g_slot, const float4* g_alb4, float* g_verts, float* g_m, float* g_albedo,
                       cudaStream_t st);
void launch_normals_bwd(const float* verts, const int32_t* faces, int F, int V, const float* g_m, float* g_verts,
                        cudaStream_t st);

// SDF -> mesh (rotational recovery): per edge id (7 per grid point) a sign-change flag and per
// tetrahedron (6 per cube) its triangle count; then, from their exclusive scans, the vertices
// (positions, grid edges) and the oriented faces; and the adjoint dL/dverts -> dL/ds (accumulated)
void launch_sdf_count(int n, const float* s, int32_t* edge_flag, int32_t* tet_count, cudaStream_t st);
void launch_sdf_write(int n, const float* s, const float lo[3], float h, const int32_t* vert_off,
                      const int32_t* face_off, float* verts, int32_t* vert_edges, int32_t* faces, cudaStream_t st);
void launch_sdf_grad(int n, const float* s, float h, int nv, const int32_t* vert_edges, const float* dl_dverts,
                     float* dl_ds, cudaStream_t st);

}  // namespace mbr
