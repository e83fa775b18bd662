// mbr_raster.cuh -- per-candidate arithmetic, the pair passes and the work scheduling shared by
// the persistent raster kernels (forward and adjoint).
//
// Work units are (256-pixel patch, split of the sample groups); CTAs draw them from a cost-ordered
// queue and hand them to their warps through a small shared-memory ring, and each warp owns an
// 8 x 4 pixel block of a tile (no block-wide barriers inside a unit).  For each sample group
// (SPT samples that share a record set) a warp walks the tile's bin lists in "pair passes":
//   1. lanes over candidates: each lane tests one face of the list for the group's samples
//      (swept boxes, pixel-reject box) and builds, as bit masks, which (pixel, sample) pairs of
//      the block it can touch;
//   2. a warp prefix scan over the pair counts;
//   3. lanes over pairs: each lane evaluates one (candidate, pixel, sample) pair.
// The core pass (swept bounding box, no soft dilation) evaluates the edge functions of
// Eq. time-dependent2, coverage and the perspective-correct z-test (Sec. 3.1) and keeps the winner
// per (pixel, sample) with a 64-bit atomicMax in shared memory.  The soft pass (r_soft-dilated
// list, uncovered samples only) sums log(1 - exp(-d/delta)) of Eqs. probability-function .. back.
// The forward shades the winners (Eq. fore + Lambert) and accumulates; the adjoint reruns both
// passes and adds one for the soft-term gradients.
#pragma once
#include "mbr_common.cuh"

namespace mbr {

// record field slots (see TriRec)
constexpr int kR_O = 0, kR_E2 = 1, kR_Z = 2, kR_BB = 3, kR_DBB = 4, kR_D = 5, kR_G = 6, kR_A = 7, kR_DZ = 8,
              kR_IL0 = 9, kR_IL1 = 10;
// Soft-coverage terms with exp(-d/delta) <= 2^-25 leave 1 - A == 1 in single precision, so they
// cannot change the product of Eq. back: the soft radius is sqrt(delta * 25 ln 2).
constexpr float kSoftCutoff = 17.328679514f;  // 25 ln 2
constexpr float kCoreMargin = 1e-5f;  // NDC slack of the undilated boxes (covers FP32 rounding)
constexpr int kPersistentThreads = 256;  // threads of a persistent raster CTA (8 warps)

struct BinLists {
  const int32_t* off;    // [G * n_tiles + 1]
  const int32_t* faces;  // CSR face lists
  int32_t cap;           // entries allocated in faces (a replayed plan may count more: clamped)
  __device__ __forceinline__ void range(size_t b, int& beg, int& end) const {
    beg = min(off[b], cap);
    end = min(off[b + 1], cap);
  }
};

struct RasterParams {
  const TriRec* recs;
  const Group* groups;
  BinLists core, soft;       // undilated (coverage) and r_soft-dilated (soft coverage) bins
  const float4* slot_nrm;    // [slots][V]
  const int32_t* faces;      // [F,3]
  const float* albedo;       // [V,3]
  const float* uv;           // [V,2] texture coordinates, or null (textured when uv and tex are set)
  const float* tex;          // [tex_h][tex_w][3] RGB texels, or null
  int32_t tex_w, tex_h;
  float* g_tex;              // adjoint: [tex_h][tex_w][3] texel gradients (zeroed), or null
  int32_t F, V, G;
  int32_t H, W, tiles_x, tiles_y, n_split;
  float r, r2, inv_delta, delta;
  int32_t prob;              // soft-coverage map: 0 exp(-d/delta), 1 sigmoid(-d/delta)
  int32_t persp;             // attribute weights: 0 screen-space w (Eq. fore), 1 perspective-correct
  float lx, ly, lz, ka, kd;
  float inv_T;
  float4* out;               // image: stored (n_split == 1) or accumulated with atomics (zeroed first)
  int32_t dbg_k;             // sub-frame whose winners are written to dbg_ids (or -1)
  int32_t* dbg_ids;
  int32_t moving;            // 1: fast solver (segment records), 0: plain solver (static records)
  int32_t work;              // units of this render: patches * n_split
  const int32_t* order;      // [work] unit visiting order (largest estimated work first), or null
  int32_t* unit_cost;        // forward, if set: [work] measured adjoint work per unit (zeroed before)
  int32_t* fwd_cost;         // forward, if set: [work] its own time per unit, SM cycles / 64 (zeroed before)
  unsigned long long* counts;  // measurement build only: [soft terms, covered samples]
  // adjoint only
  const float4* dl_dimage;   // [H*W]
  float4* g_slot;            // [slots][V][2]: (dx, dy, dnx, dny), (dnz, dz, 0, 0) of the slot states
  float4* g_albedo;          // [V] (dr, dg, db, 0), or null
  // per-sample raster state, written by the forward (when s_stat is set) and read by the adjoint
  float* s_val;              // [T][H][W] covered: winner face id (int bits); else log soft product
  uint8_t* s_stat;           // [T][H][W] kStatCovered, or the count of vanishing soft factors (<= 2)
};

constexpr uint8_t kStatCovered = 0xff;
// A soft factor 1 - A at or below this is "vanishing": it is counted, not summed as a log, so
// that the adjoint's exclusive products prod_{l != j} (1 - A_l) never divide by zero.
constexpr float kTinyFactor = 1e-30f;

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

// Bilinear texture lookup at (u, v) in [0, 1]^2 (u along the width, v along the rows; texel
// centres at (k + 0.5) / size; clamp-to-edge addressing).  Returns the colour, the four taps and
// their weights, and dc/du, dc/dv for the adjoint (zero across a clamped border).
struct TexTap {
  int idx[4];   // texel indices (x + y w): (x0, y0), (x1, y0), (x0, y1), (x1, y1)
  float wt[4];  // bilinear weights
};

__device__ __forceinline__ TexTap tex_lookup(const float* __restrict__ tex, int w, int h, float u, float v,
                                             float c[3], float dcdu[3], float dcdv[3]) {
  const float X = fminf(fmaxf(u * w - 0.5f, -1.f), (float)w), Y = fminf(fmaxf(v * h - 0.5f, -1.f), (float)h);
  const float x0f = floorf(X), y0f = floorf(Y);
  const float fx = X - x0f, fy = Y - y0f;
  const int x0 = (int)x0f, y0 = (int)y0f;
  const int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
  const int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
  TexTap t;
  t.idx[0] = ya * w + xa;
  t.idx[1] = ya * w + xb;
  t.idx[2] = yb * w + xa;
  t.idx[3] = yb * w + xb;
  t.wt[0] = (1.f - fx) * (1.f - fy);
  t.wt[1] = fx * (1.f - fy);
  t.wt[2] = (1.f - fx) * fy;
  t.wt[3] = fx * fy;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float t00 = __ldg(tex + 3 * t.idx[0] + k), t10 = __ldg(tex + 3 * t.idx[1] + k);
    const float t01 = __ldg(tex + 3 * t.idx[2] + k), t11 = __ldg(tex + 3 * t.idx[3] + k);
    c[k] = t.wt[0] * t00 + t.wt[1] * t10 + t.wt[2] * t01 + t.wt[3] * t11;
    dcdu[k] = w * ((1.f - fy) * (t10 - t00) + fy * (t11 - t01));
    dcdv[k] = h * ((1.f - fx) * (t01 - t00) + fx * (t11 - t10));
  }
  return t;
}

// Camera depths of the record's vertices at tau (keyframe lerp for the fast solver).
template <bool MOVING>
__device__ __forceinline__ void depths_at(const float4* r, float tau, float z[3]) {
  z[0] = r[kR_Z].x;
  z[1] = r[kR_Z].y;
  z[2] = r[kR_Z].z;
  if (MOVING) {
    z[0] = fmaf(tau, r[kR_DZ].x, z[0]);
    z[1] = fmaf(tau, r[kR_DZ].y, z[1]);
    z[2] = fmaf(tau, r[kR_DZ].z, z[2]);
  }
}

// Attribute weights of a covered sample from its screen-space barycentrics w: w itself (Eq. fore
// interpolates in screen space), or, with persp, the perspective-correct weights
// (w_i / z_i) / sum_j (w_j / z_j); iz receives 1 / (z_i sum_j w_j / z_j) for the adjoint.
__device__ __forceinline__ void attribute_weights(bool persp, const float w[3], const float z[3], float a[3],
                                                  float iz[3]) {
  if (!persp) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      a[q] = w[q];
      iz[q] = 0.f;
    }
    return;
  }
  float s = 0.f, wz[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    wz[q] = w[q] / z[q];
    s += wz[q];
  }
  const float is = 1.f / s;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    a[q] = wz[q] * is;
    iz[q] = is / z[q];
  }
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
  return __fdividef(__fdividef(e.N0, z0) + __fdividef(e.N1, z1) + __fdividef(e.N2, z2), e.D);
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
    const float invD = __fdividef(1.0f, e.D);
    g.w1 = e.N1 * invD;
    g.w2 = e.N2 * invD;
    g.ppx = fmaf(g.w1, e1Xx, g.w2 * e2Xx);
    g.ppy = fmaf(g.w1, e1Xy, g.w2 * e2Xy);
    g.c = closest_local(e1Xx, e1Xy, e2Xx, e2Xy, g.ppx, g.ppy, X ? r[kR_IL1] : r[kR_IL0]);
    const float e1tx = fmaf(tau, r[kR_D].x, r[kR_O].z), e1ty = fmaf(tau, r[kR_D].y, r[kR_O].w);
    const float e2tx = fmaf(tau, r[kR_D].z, r[kR_E2].x), e2ty = fmaf(tau, r[kR_D].w, r[kR_E2].y);
    const float qtx = fmaf(-tau, r[kR_G].x, s.q0x), qty = fmaf(-tau, r[kR_G].y, s.q0y);
    g.rx = fmaf(g.c.w1, e1tx, fmaf(g.c.w2, e2tx, -qtx));
    g.ry = fmaf(g.c.w1, e1ty, fmaf(g.c.w2, e2ty, -qty));
    g.d = fmaf(g.rx, g.rx, g.ry * g.ry);
  } else {
    g.c = closest_local(r[kR_O].z, r[kR_O].w, r[kR_E2].x, r[kR_E2].y, s.q0x, s.q0y, r[kR_IL0]);
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

// Pixel-centre rectangle in NDC of a warp's 8 x 4 pixel block (clipped to the image).
struct TileBox {
  float u_lo, u_hi, v_lo, v_hi;
  bool empty;
};

// Warp block b of a TW x TH tile is the 8 x 4 pixel block (b % (TW/8), b / (TW/8)); lane l is
// pixel (l % 8, l / 8) of that block.
template <int TW, int TH>
struct PixelMap {
  static_assert(TW % 8 == 0 && TH % 4 == 0, "tile must be a multiple of 8 x 4 pixels");
  static constexpr int kBlocks = (TW / 8) * (TH / 4);
  static __device__ __forceinline__ void pixel(int tx, int ty, int wb, int& px, int& py) {
    const int l = threadIdx.x & 31;
    px = tx * TW + (wb % (TW / 8)) * 8 + (l & 7);
    py = ty * TH + (wb / (TW / 8)) * 4 + (l >> 3);
  }
  static __device__ __forceinline__ TileBox warp_box(int tx, int ty, int wb, int W, int H) {
    const int x0 = tx * TW + (wb % (TW / 8)) * 8, y0 = ty * TH + (wb / (TW / 8)) * 4;
    const int x1 = min(W, x0 + 8) - 1, y1 = min(H, y0 + 4) - 1;
    TileBox t;
    t.empty = x0 >= W || y0 >= H;
    t.u_lo = (2.f * x0 + 1.f) / W - 1.f;
    t.u_hi = (2.f * x1 + 1.f) / W - 1.f;
    t.v_hi = 1.f - (2.f * y0 + 1.f) / H;
    t.v_lo = 1.f - (2.f * y1 + 1.f) / H;
    return t;
  }
};

__device__ __forceinline__ bool in_box(const float4& b, float u, float v) {
  return u >= b.x && u <= b.y && v >= b.z && v <= b.w;
}

// Candidate meta-data for a warp: the samples whose box (dilated by m) meets the warp's pixel
// rectangle, and a pixel-reject box (union of those samples' boxes).  Computed by one lane per
// candidate.
template <bool MOVING>
__device__ __forceinline__ uint32_t candidate_meta(const TriRec* rec, const Group* grp, int n, const TileBox& tb,
                                                   float m, float4& box) {
  const float4 b = __ldg(&rec->f4[kR_BB]);
  float4 db = make_float4(0.f, 0.f, 0.f, 0.f);
  if (MOVING) db = __ldg(&rec->f4[kR_DBB]);
  uint32_t mask = 0;
  float tlo = INFINITY, thi = -INFINITY;
  if (!MOVING) n = 1;
  for (int i = 0; i < n; ++i) {
    const float tau = MOVING ? __ldg(&grp->tau[i]) : 0.f;
    const bool hit = fmaf(tau, db.x, b.x) - m <= tb.u_hi && fmaf(tau, db.y, b.y) + m >= tb.u_lo &&
                     fmaf(tau, db.z, b.z) - m <= tb.v_hi && fmaf(tau, db.w, b.w) + m >= tb.v_lo;
    if (hit) {
      mask |= 1u << i;
      tlo = fminf(tlo, tau);
      thi = fmaxf(thi, tau);
    }
  }
  box = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
  if (mask) {
    box.x = fminf(fmaf(tlo, db.x, b.x), fmaf(thi, db.x, b.x)) - m;
    box.y = fmaxf(fmaf(tlo, db.y, b.y), fmaf(thi, db.y, b.y)) + m;
    box.z = fminf(fmaf(tlo, db.z, b.z), fmaf(thi, db.z, b.z)) - m;
    box.w = fmaxf(fmaf(tlo, db.w, b.w), fmaf(thi, db.w, b.w)) + m;
  }
  return mask;
}

// Load the record fields a pass needs (broadcast loads: every lane reads the same record).
template <bool MOVING>
__device__ __forceinline__ void load_record(const TriRec* src, float4 (&r)[kRecF4], bool with_z, bool with_box) {
  r[kR_O] = __ldg(&src->f4[kR_O]);
  r[kR_E2] = __ldg(&src->f4[kR_E2]);
  if (with_z) r[kR_Z] = __ldg(&src->f4[kR_Z]);
  if (with_box) {
    r[kR_IL0] = __ldg(&src->f4[kR_IL0]);
    if (MOVING) r[kR_IL1] = __ldg(&src->f4[kR_IL1]);
  }
  if (MOVING) {
    if (with_box) {
      r[kR_BB] = __ldg(&src->f4[kR_BB]);
      r[kR_DBB] = __ldg(&src->f4[kR_DBB]);
    }
    r[kR_D] = __ldg(&src->f4[kR_D]);
    r[kR_G] = __ldg(&src->f4[kR_G]);
    r[kR_A] = __ldg(&src->f4[kR_A]);
    if (with_z) r[kR_DZ] = __ldg(&src->f4[kR_DZ]);
  }
}

__device__ __forceinline__ float4 shfl_box(const float4& b, int src) {
  return make_float4(__shfl_sync(0xffffffffu, b.x, src), __shfl_sync(0xffffffffu, b.y, src),
                     __shfl_sync(0xffffffffu, b.z, src), __shfl_sync(0xffffffffu, b.w, src));
}

// ---------------------------------------------------------------- compacted pair passes
// A warp owns an 8 x 4 pixel block (lane p = pixel (p % 8, p / 8)).  The adjoint's soft pass does
// not evaluate a candidate triangle on all 32 lanes when its box touches a few of the pixels; it
// walks the bin list 32 candidates at a time in two steps:
//   generation  lane j takes candidate j: its samples whose box meets the warp's rectangle, and
//               the block pixels its box can touch that take part in the pass; a warp scan lays
//               the (candidate, pixel) pairs out in candidate order;
//   processing  the pairs go to the lanes in batches of 32 consecutive pairs, or in 32 runs of
//               consecutive pairs, one per lane (see for_pairs).

constexpr uint32_t kFullMask = 0xffffffffu;

// Per-warp shared scratch of the passes.
template <int SPT, int ROWS = 6>
struct WarpScratch {
  float logp[SPT][32];              // sum of log(1 - A_j) over the soft factors that do not vanish
  int wface[SPT][32];               // state-free adjoint: recomputed winner face (or -1)
  int nzero[SPT][32];               // vanishing soft factors
  uint32_t pixs[32];                // samples each pixel takes part in, this pass
  float pu[32], pv[32];             // NDC centre of each pixel (written by its own lane)
  float ga[32];                     // adjoint: dL/dalpha / T of each pixel
  int face[32];                     // current chunk of 32 candidates: face ids,
  uint32_t pmask[32];               //   block pixels each may touch,
  uint32_t smask[32];               //   samples each may touch,
  int prefix[33];                   //   pair offsets
  float4 coef[32][ROWS];            // per candidate of a chunk: forward passes: its coefficients at one
                                    // sample time (6 rows); adjoint: its staged record, or a lane's
                                    // contributions to its covered sample's winner (12 rows)
};

// The adjoint's scratch: the staging table and, per candidate of a chunk, its soft-term gradient
// summed over the chunk's pair batches before one set of global atomics.  Table rows: the plain
// solver (SPT 1) stages 5 record fields (rows 0-3 and 9); the fast solver stages 8 rows of
// coefficients per sample with up to two samples per group, its whole record (11 rows) with four.
// The row count is odd, so that the 8 lanes of a 16-byte shared-memory access phase that read
// the same row of different candidates fall in distinct banks.
template <int SPT>
constexpr int bwd_rows() {
  return SPT == 1 ? 11 : (SPT == 2 ? 17 : 13);
}
template <int SPT>
struct BwdScratch : WarpScratch<SPT, bwd_rows<SPT>()> {
  float grow[32][SPT == 1 ? 6 : 12];
};

// Pixel geometry of a warp block.
struct BlockPix {
  int x0, y0, W, H;
  // NDC centre of block pixel p (computed by the owning lane; other lanes read it from the
  // warp's scratch, so every lane sees the same values)
  __device__ __forceinline__ void uv(int p, float& u, float& v) const {
    const int px = x0 + (p & 7), py = y0 + (p >> 3);
    u = (2.f * px + 1.f) / W - 1.f;
    v = 1.f - (2.f * py + 1.f) / H;
  }
};

// Soft-coverage probability A of a triangle at squared distance d (Eq. probability-function)
// and the factor 1 - A it contributes; dA_dd receives dA/dd.  prob 0: A = exp(-d/delta) (the
// paper's map); 1: A = sigmoid(-d/delta) = E / (1 + E) with E = exp(-d/delta) (the SoftRas map
// the paper replaces), so 1 - A = 1 / (1 + E) and dA/dd = -A (1 - A) / delta.  E comes from the
// fast exponential: its relative error (~1e-6) changes alpha = 1 - prod(1 - A_j) by at most
// about that much in absolute terms, because each factor's absolute error passes through the
// product scaled by the other factors (all <= 1).  The sigmoid is below the exponential, so the
// 2^-25 cutoff of the soft radius holds for both maps.
__device__ __forceinline__ float soft_factor(float d, float inv_delta, int prob, float& A, float& dA_dd) {
  const float E = __expf(-d * inv_delta);
  if (prob == 0) {
    A = E;
    dA_dd = -E * inv_delta;
    return 1.f - E;
  }
  const float f = 1.f / (1.f + E);
  A = E * f;
  dA_dd = -A * f * inv_delta;
  return f;
}

// Block pixels whose centres lie in box (xmin, xmax, ymin, ymax).  The boxes are dilated by at
// least kCoreMargin, far above the rounding of this arithmetic, so no pixel inside the
// undilated region is lost.
__device__ __forceinline__ uint32_t box_pixel_mask(const float4& b, const BlockPix& bp) {
  const float hw = 0.5f * bp.W, hh = 0.5f * bp.H;
  const float c0 = fminf(fmaxf(ceilf(fmaf(b.x + 1.f, hw, -0.5f)) - bp.x0, -1.f), 8.f);
  const float c1 = fminf(fmaxf(floorf(fmaf(b.y + 1.f, hw, -0.5f)) - bp.x0, -1.f), 8.f);
  const float r0 = fminf(fmaxf(ceilf(fmaf(1.f - b.w, hh, -0.5f)) - bp.y0, -1.f), 4.f);
  const float r1 = fminf(fmaxf(floorf(fmaf(1.f - b.z, hh, -0.5f)) - bp.y0, -1.f), 4.f);
  const int ic0 = max((int)c0, 0), ic1 = min((int)c1, 7), ir0 = max((int)r0, 0), ir1 = min((int)r1, 3);
  if (ic0 > ic1 || ir0 > ir1) return 0u;
  const uint32_t xm = (0xffu >> (7 - ic1)) & (0xffu << ic0);
  const uint32_t rb = (0xfu >> (3 - ir1)) & (0xfu << ir0);
  const uint32_t spread = (rb & 1u) | ((rb & 2u) << 7) | ((rb & 4u) << 14) | ((rb & 8u) << 21);
  return xm * spread;
}

// position of the r-th (0-based) set bit of m; r < popc(m)
__device__ __forceinline__ int nth_set_bit(uint32_t m, int r) {
  int pos = 0, c;
  c = __popc(m & 0xffffu); if (r >= c) { r -= c; m >>= 16; pos += 16; }
  c = __popc(m & 0xffu);   if (r >= c) { r -= c; m >>= 8;  pos += 8; }
  c = __popc(m & 0xfu);    if (r >= c) { r -= c; m >>= 4;  pos += 4; }
  c = __popc(m & 0x3u);    if (r >= c) { r -= c; m >>= 2;  pos += 2; }
  c = (int)(m & 1u);       if (r >= c) { pos += 1; }
  return pos;
}

// Walk a bin list (warp-collective).  Per chunk of 32 candidates that has pairs: fn.chunk_begin()
// on every lane; with STAGE, fn.stage(record, samples) on lane j for candidate j (what the chunk's
// pairs need of a candidate, read from shared memory instead of global memory); then the pairs;
// finally fn.chunk_end(face, has pairs) on lane j for candidate j.  The pairs go to the lanes in
// one of two ways:
//   batches (RUNS false)  a candidate's pairs are cut into lane slots of K consecutive pairs
//                         (the last one may be short), and slot k of batch b goes to lane k - 32 b:
//                         fn.clear() on every lane, fn.pair(face, p, samples, slot) for each of
//                         the lane's pairs, then fn.batch_end(face or -1, slot); a batch's lanes
//                         of one candidate are consecutive and read its staged values as
//                         broadcasts, and each lane's K pairs share one place in the warp sum;
//   runs (RUNS true)      lane l takes the pairs [l n, (l + 1) n), n = ceil(pairs / 32):
//                         fn.pair_run(face, p, samples, slot) for each, then fn.flush(); a lane's
//                         pairs mostly share a candidate, so its sums stay in registers.
// slot = the candidate's row in the chunk.  allowed[i] = pixels taking part for sample i;
// any_samples = OR of their samples.
template <int SPT, bool MOVING, bool STAGE, bool RUNS, int K, int ROWS, typename Fn>
__device__ __forceinline__ void for_pairs(const TriRec* recs_set, const int32_t* list, int beg, int end,
                                          const Group* grp, int n, const TileBox& tb, const BlockPix& bp, float m,
                                          const uint32_t (&allowed)[SPT], uint32_t any_samples,
                                          WarpScratch<SPT, ROWS>& ws,
                                          Fn&& fn) {
  const int lane = threadIdx.x & 31;
  for (int c0 = beg; c0 < end; c0 += 32) {
    const int j = c0 + lane;
    int f = 0;
    uint32_t sm = 0, pm = 0;
    if (j < end && !tb.empty) {
      f = __ldg(list + j);
      float4 box;
      sm = candidate_meta<MOVING>(recs_set + f, grp, n, tb, m, box) & any_samples;
      if (sm) {
        uint32_t al = 0;
#pragma unroll
        for (int i = 0; i < SPT; ++i)
          if (sm & (1u << i)) al |= allowed[i];
        pm = box_pixel_mask(box, bp) & al;
      }
    }
    int incl = RUNS ? __popc(pm) : (__popc(pm) + K - 1) / K;  // pairs (runs) or lane slots (batches)
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(kFullMask, incl, 31);
    if (total == 0) continue;
    __syncwarp();  // the previous chunk's pairs are read
    ws.face[lane] = f;
    ws.pmask[lane] = pm;
    ws.smask[lane] = sm;
    ws.prefix[lane + 1] = incl;
    if (lane == 0) ws.prefix[0] = 0;
    fn.chunk_begin();
    if (STAGE && pm) fn.stage(recs_set + f, sm);
    __syncwarp();
    if constexpr (RUNS) {
      const int run = (total + 31) >> 5;
      const int k0 = lane * run, k1 = min(k0 + run, total);
      if (k0 < k1) {
        // the run's first pair: the last candidate whose first pair is at or before k0 (it has
        // pairs, since the next prefix is above k0), and its pixels from the (k0 - prefix)-th on
        int jj = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (ws.prefix[jj + step] <= k0) jj += step;
        uint32_t rem = ws.pmask[jj];
        rem &= kFullMask << nth_set_bit(rem, k0 - ws.prefix[jj]);
        for (int k = k0; k < k1; ++k) {
          if (!rem) {  // the next candidate with pairs
            do {
              ++jj;
            } while (ws.pmask[jj] == 0u);
            rem = ws.pmask[jj];
          }
          const int p = __ffs(rem) - 1;
          rem &= rem - 1u;
          const uint32_t smp = ws.smask[jj] & ws.pixs[p];
          if (smp) fn.pair_run(ws.face[jj], p, smp, jj);
        }
        fn.flush();
      }
      __syncwarp();  // the runs' sums are in the chunk's rows
    } else {
      for (int b = 0; b < total; b += 32) {
        const int k = b + lane;
        int face = -1, jj = 0;  // jj: last candidate whose first lane slot is at or before k
        uint32_t rem = 0u;      // the slot's pixels: the candidate's from its K (k - prefix)-th on
        if (k < total) {
#pragma unroll
          for (int step = 16; step > 0; step >>= 1)
            if (ws.prefix[jj + step] <= k) jj += step;
          rem = ws.pmask[jj];
          rem &= kFullMask << nth_set_bit(rem, K * (k - ws.prefix[jj]));
          face = ws.face[jj];
        }
        fn.clear();
#pragma unroll 1
        for (int t = 0; t < K && rem; ++t) {
          const int p = __ffs(rem) - 1;
          rem &= rem - 1u;
          const uint32_t smp = ws.smask[jj] & ws.pixs[p];
          if (smp) fn.pair(face, p, smp, jj);
        }
        fn.batch_end(face, jj);
      }
    }
    fn.chunk_end(f, pm != 0u);
  }
  __syncwarp();
}

// pass 1: z-test winners (Sec. 3.1: coverage by the edge functions of Eq. time-dependent2, then
// the perspective-correct depth; ties to the smaller face id).  Lanes over pixels: the bin list is
// read 32 candidates at a time, lane j holding candidate j's record.  For each sample time tau of
// the group the candidates whose box at tau meets the warp's block are picked by ballot, and each
// of them forms its edge functions at tau once -- for a fixed tau the numerators N1, N2 and the
// denominator D of Eq. time-dependent2 are affine in the pixel position (N1 = cross(p - o, E2(tau))
// + c1 tau + a11 tau^2, N2 = cross(E1(tau), p - o) + c2 tau + a12 tau^2, D = D0 + D1 tau + D2 tau^2,
// with E1, E2 the local edges at tau) -- together with the reciprocal vertex depths and 1 / D, into
// the warp's shared table.  Every lane then tests its own pixel against those candidates in turn
// (broadcast reads) and keeps the nearest covering face per sample in registers: a test is a few
// multiply-adds, with no atomics.  bkey / bface: inverse-depth key (0: none) and face per sample.
// Returns the coverage tests of this lane's pixel.
template <int SPT, bool MOVING, int ROWS>
__device__ __forceinline__ uint32_t core_raster(const TriRec* recs_set, const int32_t* list, int beg, int end,
                                                const float* tau_g, int n, const TileBox& tb, float u, float v,
                                                bool in_img, WarpScratch<SPT, ROWS>& ws, float (&bkey)[SPT],
                                                int (&bface)[SPT]) {
  const int lane = threadIdx.x & 31;
  uint32_t n_tests = 0;
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    bkey[i] = 0.f;
    bface[i] = -1;
  }
  if (tb.empty) return 0;
  for (int c0 = beg; c0 < end; c0 += 32) {
    const int j = c0 + lane;
    const bool valid = j < end;
    const int f = valid ? __ldg(list + j) : 0;
    const TriRec* rec = recs_set + f;
    // the box and the denominator's fields stay in registers; the rest is read when needed
    float4 e2 = make_float4(0.f, 0.f, 0.f, 0.f), b = e2, db = e2, a = e2;
    if (valid) {
      e2 = __ldg(&rec->f4[kR_E2]);
      b = __ldg(&rec->f4[kR_BB]);
      if (MOVING) {
        db = __ldg(&rec->f4[kR_DBB]);
        a = __ldg(&rec->f4[kR_A]);
      }
    }
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
      if (i >= (MOVING ? n : 1)) break;
      const float tau = MOVING ? __ldg(tau_g + i) : 0.f;
      // the candidate's box at tau against the block's pixel rectangle
      const bool hit = valid && fmaf(tau, db.x, b.x) - kCoreMargin <= tb.u_hi &&
                       fmaf(tau, db.y, b.y) + kCoreMargin >= tb.u_lo && fmaf(tau, db.z, b.z) - kCoreMargin <= tb.v_hi &&
                       fmaf(tau, db.w, b.w) + kCoreMargin >= tb.v_lo;
      const float D = fmaf(fmaf(a.w, tau, a.z), tau, e2.z);
      uint32_t M = __ballot_sync(kFullMask, hit && fabsf(D) > kDetMin);
      if (!M) continue;
      if ((M >> lane) & 1u) {
        const float4 o = __ldg(&rec->f4[kR_O]), zz = __ldg(&rec->f4[kR_Z]);
        float4 d = make_float4(0.f, 0.f, 0.f, 0.f), g = d, dz = d;
        if (MOVING) {
          d = __ldg(&rec->f4[kR_D]);
          g = __ldg(&rec->f4[kR_G]);
          dz = __ldg(&rec->f4[kR_DZ]);
        }
        const float E1x = fmaf(tau, d.x, o.z), E1y = fmaf(tau, d.y, o.w);
        const float E2x = fmaf(tau, d.z, e2.x), E2y = fmaf(tau, d.w, e2.y);
        ws.coef[lane][0] = make_float4(o.x, o.y, E2y, -E2x);
        ws.coef[lane][1] = make_float4(-E1y, E1x, tau * fmaf(a.x, tau, g.z), tau * fmaf(a.y, tau, g.w));
        ws.coef[lane][2] = make_float4(D, __fdividef(1.0f, D), __int_as_float(f), 0.f);
        ws.coef[lane][3] = make_float4(__fdividef(1.0f, fmaf(tau, dz.x, zz.x)), __fdividef(1.0f, fmaf(tau, dz.y, zz.y)),
                                       __fdividef(1.0f, fmaf(tau, dz.z, zz.z)), 0.f);
      }
      __syncwarp();
      if (in_img) n_tests += __popc(M);
      while (M) {
        // two candidates per step (independent chains; the second repeats the first when one is left)
        const int ca = __ffs(M) - 1;
        M &= M - 1u;
        const int cb = M ? __ffs(M) - 1 : ca;
        if (M) M &= M - 1u;
        const float4 a0 = ws.coef[ca][0], a1 = ws.coef[ca][1], a2 = ws.coef[ca][2];
        const float4 b0 = ws.coef[cb][0], b1 = ws.coef[cb][1], b2 = ws.coef[cb][2];
        const float qxa = u - a0.x, qya = v - a0.y, qxb = u - b0.x, qyb = v - b0.y;
        const float N1a = fmaf(qxa, a0.z, fmaf(qya, a0.w, a1.z)), N1b = fmaf(qxb, b0.z, fmaf(qyb, b0.w, b1.z));
        const float N2a = fmaf(qxa, a1.x, fmaf(qya, a1.y, a1.w)), N2b = fmaf(qxb, b1.x, fmaf(qyb, b1.y, b1.w));
        const float N0a = a2.x - N1a - N2a, N0b = b2.x - N1b - N2b;
        const bool cova = (N0a >= 0.f && N1a >= 0.f && N2a >= 0.f) || (N0a <= 0.f && N1a <= 0.f && N2a <= 0.f);
        const bool covb = (N0b >= 0.f && N1b >= 0.f && N2b >= 0.f) || (N0b <= 0.f && N1b <= 0.f && N2b <= 0.f);
        if (cova) {
          const float4 a3 = ws.coef[ca][3];
          const float key = fmaxf(fmaf(N0a, a3.x, fmaf(N1a, a3.y, N2a * a3.z)) * a2.y, 1e-30f);  // > 0 when covered
          const int face = __float_as_int(a2.z);
          if (key > bkey[i] || (key == bkey[i] && face < bface[i])) {
            bkey[i] = key;
            bface[i] = face;
          }
        }
        if (covb && cb != ca) {
          const float4 b3 = ws.coef[cb][3];
          const float key = fmaxf(fmaf(N0b, b3.x, fmaf(N1b, b3.y, N2b * b3.z)) * b2.y, 1e-30f);
          const int face = __float_as_int(b2.z);
          if (key > bkey[i] || (key == bkey[i] && face < bface[i])) {
            bkey[i] = key;
            bface[i] = face;
          }
        }
      }
      __syncwarp();  // the table is rewritten for the next sample
    }
  }
  return n_tests;
}

// Soft-coverage geometry of one pair and sample: false if the factor is outside the cutoff.
template <bool MOVING>
__device__ __forceinline__ bool soft_pair_term(const float4 (&r)[kRecF4], const PixelSetup<MOVING>& ps, float u,
                                               float v, float tau, int X, float m, float r2, EdgeVals& e,
                                               SoftGeom& sg) {
  if (MOVING && !in_box_at(r, tau, m, u, v)) return false;
  e = edge_vals<MOVING>(r, ps, tau);
  if (fabsf(e.D) <= kDetMin) return false;
  sg = soft_geom<MOVING>(r, ps, e, tau, X);
  return sg.d <= r2;
}

// The fast solver's soft distance as affine coefficients in q = p - o (o the record origin) at one
// sample time tau and keyframe X (Eqs. euc-dist-approx-1..3): w(tau) = (N1, N2) / D is affine in q
// (N1 = cross(q, E2) + c1 tau + a11 tau^2, N2 = cross(E1, q) + c2 tau + a12 tau^2 with E1, E2 the
// local edges at tau), hence so is the transported point p' = F(X) w(tau); the closest point w* of
// F(X) to p' (three clamped edge projections) gives d = |F(tau) w* - p|^2 with
// F(tau) w* - p = w*_1 E1 + w*_2 E2 - (q - tau g).  The forward's soft pass and the adjoint evaluate
// the term with these same functions, so both take the same single-precision decisions (cutoff,
// vanishing factor).  k[0] = (o, dp'x/dq), k[1] = (p'x(0), dp'y/dq, p'y(0)), k[2] = (e1(X), e2(X)),
// k[3] = (1/|edge(X)|^2, tau g.x), k[4] = (E1, E2), k[5] = (tau g.y); wc = the affine w1, w2.
struct SoftAffine {
  float4 k[6];
  float w1u, w1v, w1c, w2u, w2v, w2c;
};

__device__ __forceinline__ SoftAffine soft_affine(const float4& o, const float4& e2, const float4& d, const float4& g,
                                                  const float4& a, const float4& il, float tau, int X, float D) {
  SoftAffine s;
  const float fx = (float)X;
  const float E1x = fmaf(tau, d.x, o.z), E1y = fmaf(tau, d.y, o.w);
  const float E2x = fmaf(tau, d.z, e2.x), E2y = fmaf(tau, d.w, e2.y);
  const float iD = __fdividef(1.0f, D);
  s.w1u = E2y * iD;
  s.w1v = -E2x * iD;
  s.w1c = tau * fmaf(a.x, tau, g.z) * iD;
  s.w2u = -E1y * iD;
  s.w2v = E1x * iD;
  s.w2c = tau * fmaf(a.y, tau, g.w) * iD;
  const float e1Xx = fmaf(fx, d.x, o.z), e1Xy = fmaf(fx, d.y, o.w);
  const float e2Xx = fmaf(fx, d.z, e2.x), e2Xy = fmaf(fx, d.w, e2.y);
  s.k[0] = make_float4(o.x, o.y, fmaf(s.w1u, e1Xx, s.w2u * e2Xx), fmaf(s.w1v, e1Xx, s.w2v * e2Xx));
  s.k[1] = make_float4(fmaf(s.w1c, e1Xx, s.w2c * e2Xx), fmaf(s.w1u, e1Xy, s.w2u * e2Xy), fmaf(s.w1v, e1Xy, s.w2v * e2Xy),
                       fmaf(s.w1c, e1Xy, s.w2c * e2Xy));
  s.k[2] = make_float4(e1Xx, e1Xy, e2Xx, e2Xy);
  s.k[3] = make_float4(il.x, il.y, il.z, tau * g.x);
  s.k[4] = make_float4(E1x, E1y, E2x, E2y);
  s.k[5] = make_float4(tau * g.y, 0.f, 0.f, 0.f);
  return s;
}

// The distance of the pixel (u, v) from the coefficients; outputs q, p', the closest point and
// r = F(tau) w* - p for the adjoint.
struct SoftEval {
  float qx, qy, ppx, ppy, rx, ry, d;
  Closest c;
};

__device__ __forceinline__ SoftEval soft_affine_eval(const float4 (&k)[6], float u, float v) {
  SoftEval e;
  e.qx = u - k[0].x;
  e.qy = v - k[0].y;
  e.ppx = fmaf(e.qx, k[0].z, fmaf(e.qy, k[0].w, k[1].x));
  e.ppy = fmaf(e.qx, k[1].y, fmaf(e.qy, k[1].z, k[1].w));
  e.c = closest_local(k[2].x, k[2].y, k[2].z, k[2].w, e.ppx, e.ppy, make_float4(k[3].x, k[3].y, k[3].z, 0.f));
  e.rx = fmaf(e.c.w1, k[4].x, fmaf(e.c.w2, k[4].z, k[3].w - e.qx));
  e.ry = fmaf(e.c.w1, k[4].y, fmaf(e.c.w2, k[4].w, k[5].x - e.qy));
  e.d = fmaf(e.rx, e.rx, e.ry * e.ry);
  return e;
}

// pass 2 of the forward: the soft factors 1 - A_j of the uncovered samples (Eqs.
// probability-function .. back), A_j = exp(-d_j / delta), summed as logs per (sample, pixel) in
// registers (factors that vanish are counted apart).  Lanes over pixels, as in pass 1: per sample
// time, the candidates whose box at tau dilated by the soft radius meets the block publish their
// distance coefficients (soft_affine for the fast solver; the plain solver's closest point of F(t)
// to p needs the record's origin, edges and inverse edge lengths) into the warp's table, and every
// lane that takes part (its sample is uncovered) evaluates its own pixel against each of them.
// Only the box and the denominator's fields stay in registers across the samples; a candidate's
// other fields are read when it publishes.  Returns this lane's distance evaluations.
template <int SPT, bool MOVING, int ROWS>
__device__ __forceinline__ uint32_t soft_raster(const TriRec* recs_set, const int32_t* list, int beg, int end,
                                                const float* tau_g, uint32_t xbits, int n, const TileBox& tb, float u,
                                                float v, uint32_t my_s, float m, float r2, float inv_delta, int prob,
                                                WarpScratch<SPT, ROWS>& ws, float (&logp)[SPT], int (&nzero)[SPT],
                                                uint32_t& n_terms, uint32_t& n_touch) {
  const int lane = threadIdx.x & 31;
  uint32_t n_eval = 0;
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    logp[i] = 0.f;
    nzero[i] = 0;
  }
  const uint32_t any_s = __reduce_or_sync(kFullMask, my_s);
  if (tb.empty || !any_s) return 0;
  for (int c0 = beg; c0 < end; c0 += 32) {
    const int j = c0 + lane;
    const bool valid = j < end;
    const int f = valid ? __ldg(list + j) : 0;
    const TriRec* rec = recs_set + f;
    float4 b = make_float4(0.f, 0.f, 0.f, 0.f), db = b, e2 = b, a = b;
    if (valid) {
      b = __ldg(&rec->f4[kR_BB]);
      e2 = __ldg(&rec->f4[kR_E2]);
      if (MOVING) {
        db = __ldg(&rec->f4[kR_DBB]);
        a = __ldg(&rec->f4[kR_A]);
      }
    }
#pragma unroll
    for (int i = 0; i < SPT; ++i) {
      if (i >= (MOVING ? n : 1)) break;
      if (!((any_s >> i) & 1u)) continue;
      const float tau = MOVING ? __ldg(tau_g + i) : 0.f;
      const bool hit = valid && fmaf(tau, db.x, b.x) - m <= tb.u_hi && fmaf(tau, db.y, b.y) + m >= tb.u_lo &&
                       fmaf(tau, db.z, b.z) - m <= tb.v_hi && fmaf(tau, db.w, b.w) + m >= tb.v_lo;
      const float D = MOVING ? fmaf(fmaf(a.w, tau, a.z), tau, e2.z) : e2.z;
      uint32_t M = __ballot_sync(kFullMask, hit && fabsf(D) > kDetMin);
      if (!M) continue;
      if ((M >> lane) & 1u) {
        const float4 o = __ldg(&rec->f4[kR_O]);
        if (MOVING) {
          const int X = (xbits >> i) & 1u;
          const SoftAffine sa = soft_affine(o, e2, __ldg(&rec->f4[kR_D]), __ldg(&rec->f4[kR_G]), a,
                                            __ldg(&rec->f4[X ? kR_IL1 : kR_IL0]), tau, X, D);
#pragma unroll
          for (int q = 0; q < 6; ++q) ws.coef[lane][q] = sa.k[q];
        } else {
          const float4 il0 = __ldg(&rec->f4[kR_IL0]);
          ws.coef[lane][0] = o;
          ws.coef[lane][1] = make_float4(e2.x, e2.y, il0.x, il0.y);
          ws.coef[lane][2] = make_float4(il0.z, 0.f, 0.f, 0.f);
        }
      }
      __syncwarp();
      const bool take = (my_s >> i) & 1u;
      if (lane == 0) n_touch += __popc(M);
      if (take) n_eval += __popc(M);
      while (M) {
        const int c = __ffs(M) - 1;
        M &= M - 1u;
        if (!take) continue;
        float dd;
        if (MOVING) {
          float4 k[6];
#pragma unroll
          for (int q = 0; q < 6; ++q) k[q] = ws.coef[c][q];
          dd = soft_affine_eval(k, u, v).d;
        } else {
          // the plain solver's term exactly as soft_geom forms it: closest point of (0, e1, e2) to q
          const float4 k0 = ws.coef[c][0], k1 = ws.coef[c][1];
          const float ilz = ws.coef[c][2].x;
          dd = closest_local(k0.z, k0.w, k1.x, k1.y, u - k0.x, v - k0.y, make_float4(k1.z, k1.w, ilz, 0.f)).d2;
        }
        if (dd <= r2) {
          float A, dA;
          const float fct = soft_factor(dd, inv_delta, prob, A, dA);
          if (fct > kTinyFactor) logp[i] += __logf(fct);
          else ++nzero[i];
          ++n_terms;
        }
      }
      __syncwarp();  // the table is rewritten for the next sample
    }
  }
  return n_eval;
}

// Persistent scheduling.  A unit is one split of the sample groups (a contiguous range of
// groups) over a 256-pixel patch of one render (one 16 x 16 tile, or four 8 x 8 tiles); it has
// 8 warp blocks of 8 x 4 pixels.  The CTAs of a grid of (SM count x resident CTAs) take units
// from a global atomic counter; inside a CTA the 8 blocks of a unit go to whichever warps ask
// next, through a CTA-local ticket ring in shared memory, so a warp never waits for the slow
// blocks of its unit and the blocks of one unit still share the SM's L1.  Each render's units
// are visited in its cost order (largest estimated work first, from the bin sizes), so the
// expensive silhouette patches do not form a tail.  Renders are ordered by the host (largest
// first); item_off[i] is the first unit of render i.
struct WorkQueue {
  const RasterParams* items;  // [n_items]
  const int32_t* item_off;    // [n_items + 1] unit offsets
  int32_t n_items, n_work;    // n_work = total units
  int32_t* counter;           // zeroed before the launch
  int32_t* status;            // device status word (kStatusSpin if a wait gave up)
  int32_t spin_limit;         // polls (x ~64 ns) before a wait gives up; kSpinLimit normally
  int32_t stall;              // test hook: 1 = claimed units are never published, so every wait
                              // for a publication runs into its limit (nothing faults or hangs)
};

constexpr int kBlocksPerUnit = 8;
constexpr int kRing = 4;              // units a CTA may have in flight
constexpr int kSpinLimit = 1 << 22;   // default bounded wait (x ~64 ns, about 0.27 s): far beyond any real wait


template <int TW, int TH>
struct UnitMap {
  static constexpr int kBlocks = PixelMap<TW, TH>::kBlocks;       // warp blocks per tile
  static constexpr int kTilesPerUnit = kBlocksPerUnit / kBlocks;  // tiles per unit (patch)
  static_assert(kBlocks * kTilesPerUnit == kBlocksPerUnit, "a unit must be 8 warp blocks");
  static __host__ __device__ __forceinline__ int patches(int n_tiles) {
    return (n_tiles + kTilesPerUnit - 1) / kTilesPerUnit;
  }
};

// CTA-local hand-out of the blocks of globally claimed units (shared memory).  Ticket t is block
// t % 8 of the CTA's local unit L = t / 8; the warp holding block 0 claims the global unit and
// publishes it in ring slot L % kRing; a slot is reused only after its 8 tickets have read it.
struct CtaQueue {
  int tick;
  int unit[kRing];
  int ready[kRing];  // L + 1 once unit[] holds local unit L
  int used[kRing];   // tickets that have read the slot (cumulative)
  __device__ __forceinline__ void init() {
    if (threadIdx.x == 0) {
      tick = 0;
      for (int q = 0; q < kRing; ++q) unit[q] = ready[q] = used[q] = 0;
    }
    __syncthreads();
  }
};

__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Next block for this warp (warp-collective).  On success (tile, split, wb) is the block and P
// (this warp's shared copy of the render parameters) is current.  Returns false when the queue
// is exhausted or a bounded wait gave up (status word set; the caller exits).
template <int TW, int TH>
__device__ __forceinline__ bool warp_next(const WorkQueue& Q, CtaQueue& cq, RasterParams& P, int& cur_item,
                                          int& tile, int& split, int& wb) {
  const int lane = threadIdx.x & 31;
  int g = 0, b = 0;
  if (lane == 0) {
    const int t = atomicAdd(&cq.tick, 1);
    const int L = t / kBlocksPerUnit, slot = L % kRing;
    b = t % kBlocksPerUnit;
    bool ok = true;
    if (b == 0) {
      int it = 0;
      const int need = kBlocksPerUnit * (L / kRing);  // readers of the slot's previous units
      while (ld_volatile(&cq.used[slot]) < need) {
        if (++it > Q.spin_limit) { ok = false; break; }
        __nanosleep(64);
      }
      __threadfence_block();
      if (ok) {
        cq.unit[slot] = atomicAdd(Q.counter, 1);
        __threadfence_block();
        if (!Q.stall) *reinterpret_cast<volatile int*>(&cq.ready[slot]) = L + 1;
      }
    } else {
      int it = 0;
      while (ld_volatile(&cq.ready[slot]) != L + 1) {
        if (++it > Q.spin_limit) { ok = false; break; }
        __nanosleep(64);
      }
      __threadfence_block();
    }
    if (ok) {
      g = ld_volatile(&cq.unit[slot]);
      atomicAdd(&cq.used[slot], 1);
    } else {
      atomicOr(Q.status, kStatusSpin);
      g = Q.n_work;
    }
  }
  g = __shfl_sync(0xffffffffu, g, 0);
  b = __shfl_sync(0xffffffffu, b, 0);
  if (g >= Q.n_work) return false;
  int lo = 0, hi = Q.n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(Q.item_off + mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  if (lo != cur_item) {  // uniform across the warp
    __syncwarp();
    const int* src = reinterpret_cast<const int*>(Q.items + lo);
    int* dst = reinterpret_cast<int*>(&P);
    for (int q = lane; q < (int)(sizeof(RasterParams) / 4); q += 32) dst[q] = __ldg(src + q);
    __syncwarp();
    cur_item = lo;
  }
  using M = UnitMap<TW, TH>;
  const int n_tiles = P.tiles_x * P.tiles_y;
  const int n_patches = M::patches(n_tiles);
  int u = g - __ldg(Q.item_off + lo);
  if (P.order) u = __ldg(P.order + u);
  split = u / n_patches;
  tile = (u - split * n_patches) * M::kTilesPerUnit + b / M::kBlocks;
  wb = b % M::kBlocks;
  return true;
}

// per-group values every thread keeps in registers
struct GroupRegs {
  int n, rec_set, slot_a, slot_b, k0;
  uint32_t xbits;
  const float* tau;  // sample times of the group (read through L1 when needed)
  __device__ __forceinline__ void load(const Group* g) {
    n = __ldg(&g->n);
    rec_set = __ldg(&g->rec_set);
    slot_a = __ldg(&g->slot_a);
    slot_b = __ldg(&g->slot_b);
    k0 = __ldg(&g->k0);
    xbits = __ldg(&g->xbits);
    tau = g->tau;
  }
};

}  // namespace mbr
