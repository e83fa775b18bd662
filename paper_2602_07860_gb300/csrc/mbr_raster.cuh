// mbr_raster.cuh -- per-candidate arithmetic of the tiled raster kernels (forward and adjoint).
//
// One CTA owns a TW x TH pixel tile (one pixel per thread) and a contiguous range of sample
// groups.  For each group the tile's candidate triangles (from the group's tile bin) are staged
// in shared memory in chunks; each thread evaluates them against its pixel for all of the
// group's samples, which live in registers (SPT of them).  Pass 1 finds the z-test winner per
// sample, pass 2 (only if some sample of the tile is uncovered) multiplies the soft-coverage
// factors, then the winners are shaded and everything is accumulated in registers; the pixel
// is written once.
#pragma once
#include "mbr_common.cuh"

namespace mbr {

constexpr int kStageCap = 64;  // candidate records staged per chunk

struct RasterParams {
  const TriRec* recs;
  const Group* groups;
  const int32_t* bin_off;    // [G * n_tiles + 1]
  const int32_t* bin_faces;  // CSR face lists
  const float4* slot_nrm;    // [slots][V]
  const int32_t* faces;      // [F,3]
  const float* albedo;       // [V,3]
  int32_t F, V, G;
  int32_t H, W, tiles_x, tiles_y, n_split;
  float r2, inv_delta, delta;
  float lx, ly, lz, ka, kd;
  float inv_T;
  float4* out;               // image (n_split == 1, scaled) or partial sums [n_split][H*W]
  int32_t dbg_k;             // sub-frame whose winners are written to dbg_ids (or -1)
  int32_t* dbg_ids;
  // backward only
  const float4* dl_dimage;   // [H*W]
  float* g_slot;             // [slots][V][5] gradients on (x, y, nx, ny, nz)
  float* g_albedo;           // [V,3] or null
};

// Edge-function values of one candidate at one sample (local frame; see TriRec).
struct EdgeVals {
  float N0, N1, N2, D;
};

template <bool MOVING>
struct PixelSetup {
  float q0x, q0y;    // pixel relative to the record origin
  float A3_1, A3_2;  // tau^0 terms of N1, N2
  float A2_1, A2_2;  // tau^1 terms of N1, N2 (MOVING)
};

template <bool MOVING>
__device__ __forceinline__ PixelSetup<MOVING> pixel_setup(const float4* r, float u, float v) {
  PixelSetup<MOVING> s;
  s.q0x = u - r[0].x;
  s.q0y = v - r[0].y;
  s.A3_1 = cross2(s.q0x, s.q0y, r[1].x, r[1].y);  // cross(q0, e2)
  s.A3_2 = cross2(r[0].z, r[0].w, s.q0x, s.q0y);  // cross(e1, q0)
  if (MOVING) {
    s.A2_1 = cross2(s.q0x, s.q0y, r[3].z, r[3].w) + r[4].z;  // cross(q0, d2) - cross(g, e2)
    s.A2_2 = cross2(r[3].x, r[3].y, s.q0x, s.q0y) + r[4].w;  // cross(d1, q0) - cross(e1, g)
  } else {
    s.A2_1 = s.A2_2 = 0.f;
  }
  return s;
}

template <bool MOVING>
__device__ __forceinline__ EdgeVals edge_vals(const float4* r, const PixelSetup<MOVING>& s, float tau) {
  EdgeVals e;
  if (MOVING) {
    e.N1 = fmaf(fmaf(r[5].x, tau, s.A2_1), tau, s.A3_1);
    e.N2 = fmaf(fmaf(r[5].y, tau, s.A2_2), tau, s.A3_2);
    e.D = fmaf(fmaf(r[5].w, tau, r[5].z), tau, r[1].z);
  } else {
    e.N1 = s.A3_1;
    e.N2 = s.A3_2;
    e.D = r[1].z;
  }
  e.N0 = e.D - e.N1 - e.N2;
  return e;
}

__device__ __forceinline__ bool covers(const EdgeVals& e) {
  const bool pos = e.N0 >= 0.f && e.N1 >= 0.f && e.N2 >= 0.f;
  const bool neg = e.N0 <= 0.f && e.N1 <= 0.f && e.N2 <= 0.f;
  return (pos || neg) && fabsf(e.D) > kDetMin;
}

// Perspective-correct inverse depth sum_i w_i / z_i(tau): larger is nearer.
template <bool MOVING>
__device__ __forceinline__ float inv_depth(const float4* r, const EdgeVals& e, float tau) {
  float z0 = r[2].x, z1 = r[2].y, z2 = r[2].z;
  if (MOVING) {
    z0 = fmaf(tau, r[6].x, z0);
    z1 = fmaf(tau, r[6].y, z1);
    z2 = fmaf(tau, r[6].z, z2);
  }
  return (e.N0 / z0 + e.N1 / z1 + e.N2 / z2) / e.D;
}

// Soft-coverage distance of an uncovered sample (Eqs. probability-function .. euc-dist-approx-3).
// MOVING (fast solver): closest point w* of F(X) to F(X) w(tau), distance measured at F(tau) w*.
// Static (plain solver): exact closest point of F(t) to p.
struct SoftGeom {
  float d;          // squared distance
  Closest c;        // closest point (region / weights) in the search triangle
  float w1, w2;     // w(tau) (MOVING)
  float ppx, ppy;   // F(X) w(tau) relative to v0(X) (MOVING)
  float rx, ry;     // F(tau) w* - p
};

template <bool MOVING>
__device__ __forceinline__ SoftGeom soft_geom(const float4* r, const PixelSetup<MOVING>& s,
                                              const EdgeVals& e, float tau, int X) {
  SoftGeom g;
  if (MOVING) {
    const float fx = (float)X;
    const float e1Xx = fmaf(fx, r[3].x, r[0].z), e1Xy = fmaf(fx, r[3].y, r[0].w);
    const float e2Xx = fmaf(fx, r[3].z, r[1].x), e2Xy = fmaf(fx, r[3].w, r[1].y);
    const float invD = 1.0f / e.D;
    g.w1 = e.N1 * invD;
    g.w2 = e.N2 * invD;
    g.ppx = fmaf(g.w1, e1Xx, g.w2 * e2Xx);
    g.ppy = fmaf(g.w1, e1Xy, g.w2 * e2Xy);
    g.c = closest_local(e1Xx, e1Xy, e2Xx, e2Xy, g.ppx, g.ppy);
    const float e1tx = fmaf(tau, r[3].x, r[0].z), e1ty = fmaf(tau, r[3].y, r[0].w);
    const float e2tx = fmaf(tau, r[3].z, r[1].x), e2ty = fmaf(tau, r[3].w, r[1].y);
    const float qtx = fmaf(-tau, r[4].x, s.q0x), qty = fmaf(-tau, r[4].y, s.q0y);
    g.rx = fmaf(g.c.w1, e1tx, fmaf(g.c.w2, e2tx, -qtx));
    g.ry = fmaf(g.c.w1, e1ty, fmaf(g.c.w2, e2ty, -qty));
    g.d = fmaf(g.rx, g.rx, g.ry * g.ry);
  } else {
    g.c = closest_local(r[0].z, r[0].w, r[1].x, r[1].y, s.q0x, s.q0y);
    g.w1 = g.w2 = g.ppx = g.ppy = 0.f;
    g.rx = fmaf(g.c.w1, r[0].z, fmaf(g.c.w2, r[1].x, -s.q0x));
    g.ry = fmaf(g.c.w1, r[0].w, fmaf(g.c.w2, r[1].y, -s.q0y));
    g.d = g.c.d2;
  }
  return g;
}

// Cooperative stage of records [c0, c0 + cnt) of the tile's list into shared memory.
template <int NT, bool MOVING>
__device__ __forceinline__ void stage_records(float4* s_rec, const TriRec* recs_set,
                                              const int32_t* list, int cnt) {
  constexpr int NF4 = MOVING ? kRecF4 : 3;
  for (int idx = threadIdx.x; idx < cnt * NF4; idx += NT) {
    const int j = idx / NF4, q = idx - j * NF4;
    const int f = __ldg(list + j);
    s_rec[j * kRecF4 + q] = __ldg(&recs_set[f].f4[q]);
  }
}

}  // namespace mbr
