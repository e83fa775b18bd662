// mbr_raster.cuh -- per-candidate arithmetic and the shared passes of the tiled raster kernels
// (forward and adjoint).
//
// One CTA owns a TW x TH pixel tile (one pixel per thread) and a contiguous range of sample
// groups.  For each group:
//   pass 1  the tile's "core" candidates (swept bounding box, no soft dilation) are staged in
//           shared memory in chunks; while staging, one thread per candidate marks which of the
//           group's samples can touch the tile and a pixel-reject box.  Each thread evaluates the
//           surviving (candidate, sample) pairs: edge functions of Eq. time-dependent2, coverage,
//           perspective-correct z-test (Sec. 3.1).  Samples live in registers (SPT of them).
//   pass 2  only if some pixel of the tile has an uncovered sample: the r_soft-dilated candidate
//           list, staged the same way, multiplies the soft-coverage factors 1 - exp(-d/delta)
//           (Eqs. probability-function .. back) of the uncovered samples.
// The forward then shades the winners (Eq. fore + Lambert) and accumulates; the adjoint adds a
// third pass for the soft-term gradients.
#pragma once
#include "mbr_common.cuh"

namespace mbr {

constexpr int kStageCap = 64;  // candidate records staged per chunk
// record field slots (see TriRec)
constexpr int kR_O = 0, kR_E2 = 1, kR_Z = 2, kR_BB = 3, kR_DBB = 4, kR_D = 5, kR_G = 6, kR_A = 7, kR_DZ = 8;
constexpr float kCoreMargin = 1e-5f;  // NDC slack of the undilated boxes (covers FP32 rounding)

struct BinLists {
  const int32_t* off;    // [G * n_tiles + 1]
  const int32_t* faces;  // CSR face lists
};

struct RasterParams {
  const TriRec* recs;
  const Group* groups;
  BinLists core, soft;       // undilated (coverage) and r_soft-dilated (soft coverage) bins
  const float4* slot_nrm;    // [slots][V]
  const int32_t* faces;      // [F,3]
  const float* albedo;       // [V,3]
  int32_t F, V, G;
  int32_t H, W, tiles_x, tiles_y, n_split;
  float r, r2, inv_delta, delta;
  float lx, ly, lz, ka, kd;
  float inv_T;
  float4* out;               // image (n_split == 1, scaled) or partial sums [n_split][H*W]
  int32_t dbg_k;             // sub-frame whose winners are written to dbg_ids (or -1)
  int32_t* dbg_ids;
  // adjoint only
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
  s.q0x = u - r[kR_O].x;
  s.q0y = v - r[kR_O].y;
  s.A3_1 = cross2(s.q0x, s.q0y, r[kR_E2].x, r[kR_E2].y);  // cross(q0, e2)
  s.A3_2 = cross2(r[kR_O].z, r[kR_O].w, s.q0x, s.q0y);    // cross(e1, q0)
  if (MOVING) {
    s.A2_1 = cross2(s.q0x, s.q0y, r[kR_D].z, r[kR_D].w) + r[kR_G].z;  // cross(q0, d2) - cross(g, e2)
    s.A2_2 = cross2(r[kR_D].x, r[kR_D].y, s.q0x, s.q0y) + r[kR_G].w;  // cross(d1, q0) - cross(e1, g)
  } else {
    s.A2_1 = s.A2_2 = 0.f;
  }
  return s;
}

template <bool MOVING>
__device__ __forceinline__ EdgeVals edge_vals(const float4* r, const PixelSetup<MOVING>& s, float tau) {
  EdgeVals e;
  if (MOVING) {
    e.N1 = fmaf(fmaf(r[kR_A].x, tau, s.A2_1), tau, s.A3_1);
    e.N2 = fmaf(fmaf(r[kR_A].y, tau, s.A2_2), tau, s.A3_2);
    e.D = fmaf(fmaf(r[kR_A].w, tau, r[kR_A].z), tau, r[kR_E2].z);
  } else {
    e.N1 = s.A3_1;
    e.N2 = s.A3_2;
    e.D = r[kR_E2].z;
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
  float z0 = r[kR_Z].x, z1 = r[kR_Z].y, z2 = r[kR_Z].z;
  if (MOVING) {
    z0 = fmaf(tau, r[kR_DZ].x, z0);
    z1 = fmaf(tau, r[kR_DZ].y, z1);
    z2 = fmaf(tau, r[kR_DZ].z, z2);
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
    const float e1Xx = fmaf(fx, r[kR_D].x, r[kR_O].z), e1Xy = fmaf(fx, r[kR_D].y, r[kR_O].w);
    const float e2Xx = fmaf(fx, r[kR_D].z, r[kR_E2].x), e2Xy = fmaf(fx, r[kR_D].w, r[kR_E2].y);
    const float invD = 1.0f / e.D;
    g.w1 = e.N1 * invD;
    g.w2 = e.N2 * invD;
    g.ppx = fmaf(g.w1, e1Xx, g.w2 * e2Xx);
    g.ppy = fmaf(g.w1, e1Xy, g.w2 * e2Xy);
    g.c = closest_local(e1Xx, e1Xy, e2Xx, e2Xy, g.ppx, g.ppy);
    const float e1tx = fmaf(tau, r[kR_D].x, r[kR_O].z), e1ty = fmaf(tau, r[kR_D].y, r[kR_O].w);
    const float e2tx = fmaf(tau, r[kR_D].z, r[kR_E2].x), e2ty = fmaf(tau, r[kR_D].w, r[kR_E2].y);
    const float qtx = fmaf(-tau, r[kR_G].x, s.q0x), qty = fmaf(-tau, r[kR_G].y, s.q0y);
    g.rx = fmaf(g.c.w1, e1tx, fmaf(g.c.w2, e2tx, -qtx));
    g.ry = fmaf(g.c.w1, e1ty, fmaf(g.c.w2, e2ty, -qty));
    g.d = fmaf(g.rx, g.rx, g.ry * g.ry);
  } else {
    g.c = closest_local(r[kR_O].z, r[kR_O].w, r[kR_E2].x, r[kR_E2].y, s.q0x, s.q0y);
    g.w1 = g.w2 = g.ppx = g.ppy = 0.f;
    g.rx = fmaf(g.c.w1, r[kR_O].z, fmaf(g.c.w2, r[kR_E2].x, -s.q0x));
    g.ry = fmaf(g.c.w1, r[kR_O].w, fmaf(g.c.w2, r[kR_E2].y, -s.q0y));
    g.d = g.c.d2;
  }
  return g;
}

// pixel inside the record's box at tau, dilated by m (the lerped keyframe boxes contain the
// lerped triangle)
__device__ __forceinline__ bool in_box_at(const float4* r, float tau, float m, float u, float v) {
  const float4 b = r[kR_BB], db = r[kR_DBB];
  return u >= fmaf(tau, db.x, b.x) - m && u <= fmaf(tau, db.y, b.y) + m && v >= fmaf(tau, db.z, b.z) - m &&
         v <= fmaf(tau, db.w, b.w) + m;
}

// Tile geometry in NDC (pixel centres of the tile, clipped to the image).
struct TileBox {
  float u_lo, u_hi, v_lo, v_hi;
};

template <int TW, int TH>
__device__ __forceinline__ TileBox tile_box(int tx, int ty, int W, int H) {
  const int x0 = tx * TW, x1 = min(W, x0 + TW) - 1, y0 = ty * TH, y1 = min(H, y0 + TH) - 1;
  TileBox t;
  t.u_lo = (2.f * x0 + 1.f) / W - 1.f;
  t.u_hi = (2.f * x1 + 1.f) / W - 1.f;
  t.v_hi = 1.f - (2.f * y0 + 1.f) / H;
  t.v_lo = 1.f - (2.f * y1 + 1.f) / H;
  return t;
}

// Cooperative stage of candidates [0, cnt) of a bin list into shared memory.  All threads load
// the record float4s; thread j < cnt also derives the candidate's sample mask (samples whose box,
// dilated by m, meets the tile) and a pixel-reject box (union of those samples' boxes).
template <int NT, bool MOVING>
__device__ __forceinline__ void stage_candidates(float4* s_rec, float4* s_box, uint32_t* s_mask,
                                                 const TriRec* recs_set, const int32_t* list, int cnt,
                                                 const Group& grp, const TileBox& tb, float m) {
  constexpr int NF4 = MOVING ? kRecF4 : kRecF4Static;
  for (int idx = threadIdx.x; idx < cnt * NF4; idx += NT) {
    const int j = idx / NF4, q = idx - j * NF4;
    const int f = __ldg(list + j);
    s_rec[j * kRecF4 + q] = __ldg(&recs_set[f].f4[q]);
  }
  if ((int)threadIdx.x < cnt) {
    const int f = __ldg(list + threadIdx.x);
    const float4 b = __ldg(&recs_set[f].f4[kR_BB]);
    float4 db = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MOVING) db = __ldg(&recs_set[f].f4[kR_DBB]);
    uint32_t mask = 0;
    float tlo = INFINITY, thi = -INFINITY;
    for (int i = 0; i < grp.n; ++i) {
      const float tau = MOVING ? grp.tau[i] : 0.f;
      const bool hit = fmaf(tau, db.x, b.x) - m <= tb.u_hi && fmaf(tau, db.y, b.y) + m >= tb.u_lo &&
                       fmaf(tau, db.z, b.z) - m <= tb.v_hi && fmaf(tau, db.w, b.w) + m >= tb.v_lo;
      if (hit) {
        mask |= 1u << i;
        tlo = fminf(tlo, tau);
        thi = fmaxf(thi, tau);
      }
    }
    float4 box = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
    if (mask) {
      box.x = fminf(fmaf(tlo, db.x, b.x), fmaf(thi, db.x, b.x)) - m;
      box.y = fmaxf(fmaf(tlo, db.y, b.y), fmaf(thi, db.y, b.y)) + m;
      box.z = fminf(fmaf(tlo, db.z, b.z), fmaf(thi, db.z, b.z)) - m;
      box.w = fmaxf(fmaf(tlo, db.w, b.w), fmaf(thi, db.w, b.w)) + m;
    }
    s_box[threadIdx.x] = box;
    s_mask[threadIdx.x] = mask;
  }
}

__device__ __forceinline__ bool in_box(const float4& b, float u, float v) {
  return u >= b.x && u <= b.y && v >= b.z && v <= b.w;
}

// Shared memory of a raster CTA.
struct RasterSmem {
  float4 rec[kStageCap * kRecF4];
  float4 box[kStageCap];
  uint32_t mask[kStageCap];
  Group grp;
};

template <int NT>
__device__ __forceinline__ void load_group(RasterSmem& sm, const Group* groups, int g) {
  __syncthreads();
  if (threadIdx.x < sizeof(Group) / 4)
    reinterpret_cast<int*>(&sm.grp)[threadIdx.x] = reinterpret_cast<const int*>(groups + g)[threadIdx.x];
  __syncthreads();
}

// pass 1: z-test winners of the group's samples for this pixel
template <int NT, int SPT, bool MOVING>
__device__ __forceinline__ void pass_winners(RasterSmem& sm, const TriRec* recs_set, const int32_t* list, int beg,
                                             int end, const TileBox& tb, bool in_img, float u, float v,
                                             float (&bestk)[SPT], int (&bestf)[SPT]) {
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    bestk[i] = -INFINITY;
    bestf[i] = -1;
  }
  for (int c0 = beg; c0 < end; c0 += kStageCap) {
    const int cnt = min(kStageCap, end - c0);
    __syncthreads();
    stage_candidates<NT, MOVING>(sm.rec, sm.box, sm.mask, recs_set, list + c0, cnt, sm.grp, tb, kCoreMargin);
    __syncthreads();
    if (!in_img) continue;
    for (int j = 0; j < cnt; ++j) {
      const uint32_t mask = sm.mask[j];
      if (!mask || !in_box(sm.box[j], u, v)) continue;
      const float4* r = sm.rec + j * kRecF4;
      const int face = __float_as_int(r[kR_E2].w);
      const PixelSetup<MOVING> ps = pixel_setup<MOVING>(r, u, v);
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        if (mask & (1u << i)) {
          const float tau = MOVING ? sm.grp.tau[i] : 0.f;
          const EdgeVals e = edge_vals<MOVING>(r, ps, tau);
          if (covers(e)) {
            const float key = inv_depth<MOVING>(r, e, tau);
            if (key > bestk[i] || (key == bestk[i] && face < bestf[i])) {
              bestk[i] = key;
              bestf[i] = face;
            }
          }
        }
      }
    }
  }
}

// Visit every soft-coverage term of the uncovered samples (uncov bit i) of this pixel:
// fn(j, r, ps, e, sg, i, tau, X) for each (candidate, sample) with d <= r^2.  The staging (and
// the __syncthreads inside) is executed by every thread of the CTA.
template <int NT, int SPT, bool MOVING, typename Fn>
__device__ __forceinline__ void for_soft_terms(RasterSmem& sm, const TriRec* recs_set, const int32_t* list, int beg,
                                               int end, const TileBox& tb, bool active, float u, float v,
                                               uint32_t uncov, float r_soft, float r2, Fn&& fn) {
  for (int c0 = beg; c0 < end; c0 += kStageCap) {
    const int cnt = min(kStageCap, end - c0);
    __syncthreads();
    stage_candidates<NT, MOVING>(sm.rec, sm.box, sm.mask, recs_set, list + c0, cnt, sm.grp, tb, r_soft + kCoreMargin);
    __syncthreads();
    for (int j = 0; j < cnt; ++j) {
      const uint32_t mask = sm.mask[j] & (active ? uncov : 0u);
      const bool hit = mask && in_box(sm.box[j], u, v);
      fn.begin(j);
      if (hit) {
        const float4* r = sm.rec + j * kRecF4;
        const PixelSetup<MOVING> ps = pixel_setup<MOVING>(r, u, v);
#pragma unroll
        for (int i = 0; i < SPT; ++i) {
          if (mask & (1u << i)) {
            const float tau = MOVING ? sm.grp.tau[i] : 0.f;
            if (MOVING && !in_box_at(r, tau, r_soft + kCoreMargin, u, v)) continue;
            const EdgeVals e = edge_vals<MOVING>(r, ps, tau);
            if (fabsf(e.D) <= kDetMin) continue;
            const int X = (sm.grp.xbits >> i) & 1u;
            const SoftGeom sg = soft_geom<MOVING>(r, ps, e, tau, X);
            if (sg.d <= r2) fn.term(j, r, ps, e, sg, i, tau, X);
          }
        }
      }
      fn.end(j, r_soft);
    }
  }
}

}  // namespace mbr
