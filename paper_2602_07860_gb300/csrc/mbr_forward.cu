// mbr_forward.cu -- forward kernels of the sm_103a motion-blurred renderer.
//
//   face_normals_kernel  a0: area-weighted vertex normals (face cross products, atomics)
//   xform_kernel         a1: motion + camera + projection of every vertex at every slot time
//   setup_kernel         a4 setup: per (record set, face) local-frame coefficients (TriRec)
//   bin_*kernel<FILL>    a3: per (group, face) swept bounding box -> core and soft tile bins
//                        (shared-memory histograms per CTA of one group, or global atomics)
//   scan kernels         exclusive scan of the bin counts (CSR offsets)
//   raster_fwd_persistent a4-a8: barycentric solve, coverage, z-test, soft alpha, shading,
//                        temporal average; one float4 store per pixel (or one float4 atomic
//                        add per pixel and group split)
//   unit_*_kernel        visiting order of the raster's work units (largest estimate first)
//   raster_fwd_count     work counters of the raster passes (measurement)
//   count_kernel         N_cand (measurement)
#include <algorithm>
#include <cstdint>

#include "mbr_internal.h"
#include "mbr_raster.cuh"

namespace mbr {

// ---------------------------------------------------------------- a0: vertex normals
__global__ void face_normals_kernel(const float* __restrict__ verts, const int32_t* __restrict__ faces,
                                    int F, int V, float* __restrict__ nacc, int* __restrict__ status) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
  if (a < 0 || b < 0 || c < 0 || a >= V || b >= V || c >= V) {
    atomicOr(status, kStatusBadFace);
    return;
  }
  const float ax = verts[3 * a], ay = verts[3 * a + 1], az = verts[3 * a + 2];
  const float ux = verts[3 * b] - ax, uy = verts[3 * b + 1] - ay, uz = verts[3 * b + 2] - az;
  const float wx = verts[3 * c] - ax, wy = verts[3 * c + 1] - ay, wz = verts[3 * c + 2] - az;
  const float nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
  const int id[3] = {a, b, c};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    atomicAdd(nacc + 3 * id[i], nx);
    atomicAdd(nacc + 3 * id[i] + 1, ny);
    atomicAdd(nacc + 3 * id[i] + 2, nz);
  }
}

// ---------------------------------------------------------------- a1: motion + camera
// grid.y = slot; camera = A [v;1] with A = view o motion(t_slot); ndc = (x, y) / (z tan).
__global__ void xform_kernel(const float* __restrict__ verts, const float* __restrict__ nacc, int V,
                             const SlotXform* __restrict__ xf, float tan_half_fov,
                             float4* __restrict__ pos, float4* __restrict__ nrm) {
  __shared__ SlotXform s;
  const int slot = blockIdx.y;
  if (threadIdx.x < sizeof(SlotXform) / 4)
    reinterpret_cast<float*>(&s)[threadIdx.x] = reinterpret_cast<const float*>(xf + slot)[threadIdx.x];
  __syncthreads();
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const float px = verts[3 * v], py = verts[3 * v + 1], pz = verts[3 * v + 2];
  const float xc = fmaf(s.A[0], px, fmaf(s.A[1], py, fmaf(s.A[2], pz, s.A[3])));
  const float yc = fmaf(s.A[4], px, fmaf(s.A[5], py, fmaf(s.A[6], pz, s.A[7])));
  const float zc = fmaf(s.A[8], px, fmaf(s.A[9], py, fmaf(s.A[10], pz, s.A[11])));
  const float den = zc * tan_half_fov;
  float nx = nacc[3 * v], ny = nacc[3 * v + 1], nz = nacc[3 * v + 2];
  const float len = sqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
  if (len > 0.f) { nx /= len; ny /= len; nz /= len; }
  const size_t o = (size_t)slot * V + v;
  pos[o] = make_float4(xc / den, yc / den, zc, 0.f);
  nrm[o] = make_float4(fmaf(s.R[0], nx, fmaf(s.R[1], ny, s.R[2] * nz)),
                       fmaf(s.R[3], nx, fmaf(s.R[4], ny, s.R[5] * nz)),
                       fmaf(s.R[6], nx, fmaf(s.R[7], ny, s.R[8] * nz)), 0.f);
}

// ---------------------------------------------------------------- a4 setup: triangle records
__global__ void setup_kernel(const float4* __restrict__ pos, const int32_t* __restrict__ faces, int F,
                             int V, const int2* __restrict__ set_slots, int n_sets, float znear,
                             TriRec* __restrict__ recs) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)n_sets * F) return;
  const int set = (int)(idx / F), f = (int)(idx - (size_t)set * F);
  const int2 sl = set_slots[set];
  const int i0 = faces[3 * f], i1 = faces[3 * f + 1], i2 = faces[3 * f + 2];
  if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= V || i1 >= V || i2 >= V) {
    // invalid face: culled (never binned, never dereferenced again)
    TriRec* dst = recs + idx;
    dst->f4[kR_E2] = make_float4(0.f, 0.f, 0.f, __int_as_float(f));
    dst->f4[kR_Z] = make_float4(1.f, 1.f, 1.f, __uint_as_float(kFlagCulled));
    return;
  }
  const float4 a0 = pos[(size_t)sl.x * V + i0], a1 = pos[(size_t)sl.x * V + i1], a2 = pos[(size_t)sl.x * V + i2];
  const float4 b0 = pos[(size_t)sl.y * V + i0], b1 = pos[(size_t)sl.y * V + i1], b2 = pos[(size_t)sl.y * V + i2];
  const float e1x = a1.x - a0.x, e1y = a1.y - a0.y, e2x = a2.x - a0.x, e2y = a2.y - a0.y;
  const float d1x = (b1.x - b0.x) - e1x, d1y = (b1.y - b0.y) - e1y;
  const float d2x = (b2.x - b0.x) - e2x, d2y = (b2.y - b0.y) - e2y;
  const float gx = b0.x - a0.x, gy = b0.y - a0.y;
  uint32_t flags = 0;
  if (a0.z <= znear || a1.z <= znear || a2.z <= znear || b0.z <= znear || b1.z <= znear || b2.z <= znear)
    flags |= kFlagCulled;
  TriRec r;
  r.f4[kR_O] = make_float4(a0.x, a0.y, e1x, e1y);
  r.f4[kR_E2] = make_float4(e2x, e2y, cross2(e1x, e1y, e2x, e2y), __int_as_float(f));
  r.f4[kR_Z] = make_float4(a0.z, a1.z, a2.z, __uint_as_float(flags));
  const float4 ba = make_float4(fminf(a0.x, fminf(a1.x, a2.x)), fmaxf(a0.x, fmaxf(a1.x, a2.x)),
                                fminf(a0.y, fminf(a1.y, a2.y)), fmaxf(a0.y, fmaxf(a1.y, a2.y)));
  const float4 bb = make_float4(fminf(b0.x, fminf(b1.x, b2.x)), fmaxf(b0.x, fmaxf(b1.x, b2.x)),
                                fminf(b0.y, fminf(b1.y, b2.y)), fmaxf(b0.y, fmaxf(b1.y, b2.y)));
  r.f4[kR_BB] = ba;
  r.f4[kR_DBB] = make_float4(bb.x - ba.x, bb.y - ba.y, bb.z - ba.z, bb.w - ba.w);
  r.f4[kR_D] = make_float4(d1x, d1y, d2x, d2y);
  r.f4[kR_G] = make_float4(gx, gy, -cross2(gx, gy, e2x, e2y), -cross2(e1x, e1y, gx, gy));
  r.f4[kR_A] = make_float4(-cross2(gx, gy, d2x, d2y), -cross2(d1x, d1y, gx, gy),
                           cross2(e1x, e1y, d2x, d2y) + cross2(d1x, d1y, e2x, e2y), cross2(d1x, d1y, d2x, d2y));
  r.f4[kR_DZ] = make_float4(b0.z - a0.z, b1.z - a1.z, b2.z - a2.z, 0.f);
  {
    // 1 / |edge|^2 of (v0,v1), (v1,v2), (v2,v0) at both keyframes (0 for a zero-length edge)
    auto inv = [](float x, float y) {
      const float l2 = fmaf(x, x, y * y);
      return l2 > 0.f ? 1.0f / l2 : 0.f;
    };
    const float f1x = e1x + d1x, f1y = e1y + d1y, f2x = e2x + d2x, f2y = e2y + d2y;
    r.f4[kR_IL0] = make_float4(inv(e1x, e1y), inv(e2x - e1x, e2y - e1y), inv(e2x, e2y), 0.f);
    r.f4[kR_IL1] = make_float4(inv(f1x, f1y), inv(f2x - f1x, f2y - f1y), inv(f2x, f2y), 0.f);
  }
  TriRec* dst = recs + idx;
#pragma unroll
  for (int q = 0; q < kRecF4; ++q) dst->f4[q] = r.f4[q];
}

// swept bounding box of a record over [tau_lo, tau_hi] (linear motion: union of the two ends)
__device__ __forceinline__ void swept_bbox(const TriRec& r, float tlo, float thi, float& xmin,
                                           float& xmax, float& ymin, float& ymax) {
  const float ox = r.f4[kR_O].x, oy = r.f4[kR_O].y;
  const float e1x = r.f4[kR_O].z, e1y = r.f4[kR_O].w, e2x = r.f4[kR_E2].x, e2y = r.f4[kR_E2].y;
  const float d1x = r.f4[kR_D].x, d1y = r.f4[kR_D].y, d2x = r.f4[kR_D].z, d2y = r.f4[kR_D].w;
  const float gx = r.f4[kR_G].x, gy = r.f4[kR_G].y;
  xmin = ymin = INFINITY;
  xmax = ymax = -INFINITY;
  const float ts[2] = {tlo, thi};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float t = ts[q];
    const float v0x = fmaf(t, gx, ox), v0y = fmaf(t, gy, oy);
    const float v1x = v0x + fmaf(t, d1x, e1x), v1y = v0y + fmaf(t, d1y, e1y);
    const float v2x = v0x + fmaf(t, d2x, e2x), v2y = v0y + fmaf(t, d2y, e2y);
    xmin = fminf(xmin, fminf(v0x, fminf(v1x, v2x)));
    xmax = fmaxf(xmax, fmaxf(v0x, fmaxf(v1x, v2x)));
    ymin = fminf(ymin, fminf(v0y, fminf(v1y, v2y)));
    ymax = fmaxf(ymax, fmaxf(v0y, fmaxf(v1y, v2y)));
  }
}

// pixel index ranges of the centres inside [xmin, xmax] x [ymin, ymax]; false if empty
__device__ __forceinline__ bool pixel_range(float xmin, float xmax, float ymin, float ymax, int W, int H,
                                            int& i0, int& i1, int& j0, int& j1) {
  i0 = max(0, (int)ceilf((xmin + 1.f) * 0.5f * W - 0.5f));
  i1 = min(W - 1, (int)floorf((xmax + 1.f) * 0.5f * W - 0.5f));
  j0 = max(0, (int)ceilf((1.f - ymax) * 0.5f * H - 0.5f));
  j1 = min(H - 1, (int)floorf((1.f - ymin) * 0.5f * H - 0.5f));
  return i0 <= i1 && j0 <= j1 && isfinite(xmin) && isfinite(ymin);
}

// ---------------------------------------------------------------- a3: tile binning
// One pass computes both bin sets of a render (core: undilated swept box; soft: dilated by
// r_soft) from one swept box per (group, face).  Count pass: per-(group, tile) counts; fill pass:
// face ids into the CSR lists through the cursors (a copy of the offsets).

// tile range of one dilated box; false if it covers no pixel centre
__device__ __forceinline__ bool tile_range(float xmin, float xmax, float ymin, float ymax, float r, int W, int H,
                                           int tw, int th, int& tx0, int& tx1, int& ty0, int& ty1) {
  int i0, i1, j0, j1;
  if (!pixel_range(xmin - r, xmax + r, ymin - r, ymax + r, W, H, i0, i1, j0, j1)) return false;
  tx0 = i0 / tw; tx1 = i1 / tw; ty0 = j0 / th; ty1 = j1 / th;
  return true;
}

template <bool FILL>
__global__ void bin_kernel(const TriRec* __restrict__ recs, int F, const Group* __restrict__ groups, int G, int W,
                           int H, int tw, int th, int tiles_x, int n_tiles, float r_core, float r_soft, BinTargets t,
                           int* __restrict__ status) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)G * F) return;
  const int g = (int)(idx / F), f = (int)(idx - (size_t)g * F);
  const Group& gr = groups[g];
  const TriRec& rec = recs[(size_t)gr.rec_set * F + f];
  if (__float_as_uint(rec.f4[kR_Z].w) & kFlagCulled) return;
  float xmin, xmax, ymin, ymax;
  swept_bbox(rec, gr.tau_lo, gr.tau_hi, xmin, xmax, ymin, ymax);
  const float rr[2] = {r_core, r_soft};
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    int tx0, tx1, ty0, ty1;
    if (!tile_range(xmin, xmax, ymin, ymax, rr[q], W, H, tw, th, tx0, tx1, ty0, ty1)) continue;
    int32_t* base = t.counts_or_cursor[q] + (size_t)g * n_tiles;
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) {
        const int b = ty * tiles_x + tx;
        const int k = atomicAdd(base + b, 1);
        if (FILL) {
          const int slot = t.off[q][(size_t)g * n_tiles + b] + k;
          // the fill pass revisits exactly the counted triples; the check only guards the list
          if (slot < t.off[q][(size_t)g * n_tiles + b + 1] && slot < t.cap[q]) t.list[q][slot] = f;
          else atomicOr(status, kStatusBinOverflow);
        }
      }
  }
}

// Two-level variant (images of up to kSmemBinTiles tiles): a CTA takes 256 faces of ONE group
// (grid.y = group) and counts its (tile, face) entries in shared-memory histograms over the
// tiles (one per bin set); the count pass adds them to the global counts, the fill pass reserves
// one range per (CTA, tile) in the global cursors and places its entries with shared-memory
// atomics.  Global atomics fall from one per entry to one per (CTA, tile) touched.
constexpr int kSmemBinTiles = 4096;

template <bool FILL>
__global__ void bin_smem_kernel(const TriRec* __restrict__ recs, int F, const Group* __restrict__ groups, int W,
                                int H, int tw, int th, int tiles_x, int n_tiles, float r_core, float r_soft,
                                BinTargets t, int* __restrict__ status) {
  extern __shared__ int sh[];  // [2][n_tiles]
  const int g = blockIdx.y;
  for (int i = threadIdx.x; i < 2 * n_tiles; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  bool have[2] = {false, false};
  int tx0[2], tx1[2], ty0[2], ty1[2];
  if (f < F) {
    const Group& gr = groups[g];
    const TriRec& rec = recs[(size_t)gr.rec_set * F + f];
    if (!(__float_as_uint(rec.f4[kR_Z].w) & kFlagCulled)) {
      float xmin, xmax, ymin, ymax;
      swept_bbox(rec, gr.tau_lo, gr.tau_hi, xmin, xmax, ymin, ymax);
      have[0] = tile_range(xmin, xmax, ymin, ymax, r_core, W, H, tw, th, tx0[0], tx1[0], ty0[0], ty1[0]);
      have[1] = tile_range(xmin, xmax, ymin, ymax, r_soft, W, H, tw, th, tx0[1], tx1[1], ty0[1], ty1[1]);
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (have[q])
      for (int ty = ty0[q]; ty <= ty1[q]; ++ty)
        for (int tx = tx0[q]; tx <= tx1[q]; ++tx) atomicAdd(&sh[q * n_tiles + ty * tiles_x + tx], 1);
  __syncthreads();
  if (!FILL) {
    for (int i = threadIdx.x; i < 2 * n_tiles; i += blockDim.x) {
      const int q = i >= n_tiles, b = i - q * n_tiles;
      if (sh[i]) atomicAdd(t.counts_or_cursor[q] + (size_t)g * n_tiles + b, sh[i]);
    }
    return;
  }
  for (int i = threadIdx.x; i < 2 * n_tiles; i += blockDim.x) {
    const int q = i >= n_tiles, b = i - q * n_tiles;
    const size_t gb = (size_t)g * n_tiles + b;
    if (sh[i]) sh[i] = t.off[q][gb] + atomicAdd(t.counts_or_cursor[q] + gb, sh[i]);  // first slot of the range
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (have[q])
      for (int ty = ty0[q]; ty <= ty1[q]; ++ty)
        for (int tx = tx0[q]; tx <= tx1[q]; ++tx) {
          const int b = ty * tiles_x + tx;
          const int slot = atomicAdd(&sh[q * n_tiles + b], 1);
          if (slot < t.off[q][(size_t)g * n_tiles + b + 1] && slot < t.cap[q]) t.list[q][slot] = f;
          else atomicOr(status, kStatusBinOverflow);
        }
}

// ---------------------------------------------------------------- clearing
__global__ void zero_kernel(ZeroList z) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (z.p[k])
      for (size_t i = t0; i < z.n[k]; i += stride) z.p[k][i] = 0;
}

void launch_zero(const ZeroList& z, cudaStream_t st) {
  size_t most = 0;
  for (int k = 0; k < 4; ++k)
    if (z.p[k]) most = std::max(most, z.n[k]);
  if (!most) return;
  const int grid = (int)std::min<size_t>((most + 255) / 256, 1024);
  zero_kernel<<<grid, 256, 0, st>>>(z);
}

// ---------------------------------------------------------------- exclusive scan (CSR offsets)
constexpr int kScanThreads = 1024, kScanPer = 4, kScanBlock = kScanThreads * kScanPer;

__device__ __forceinline__ int block_exclusive_scan(int x, int* s_warp, int& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0;
    int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) s_warp[32] = wi;
  }
  __syncthreads();
  total = s_warp[32];
  const int r = s_warp[wid] + incl - x;
  __syncthreads();
  return r;
}

// The core and soft count arrays are scanned together (grid.y = array).  The apply pass zeroes
// the counts after reading them: they are the fill pass's cursors (slot = offset + cursor).
__global__ void scan_reduce_kernel(ScanPair sp) {
  __shared__ int s_warp[33];
  const int q = blockIdx.y, n = sp.n;
  const int32_t* in = sp.in[q];
  const size_t base = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * kScanPer;
  int x = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k)
    if (base + k < (size_t)n) x += in[base + k];
  int total;
  block_exclusive_scan(x, s_warp, total);
  if (threadIdx.x == 0) sp.sums[q][blockIdx.x] = total;
}

__global__ void scan_sums_kernel(ScanPair sp, int nb) {
  __shared__ int s_warp[33];
  int32_t* sums = sp.sums[blockIdx.y];
  int carry = 0;
  for (int c = 0; c < nb; c += kScanThreads) {
    const int i = c + threadIdx.x;
    const int x = i < nb ? sums[i] : 0;
    int total;
    const int ex = block_exclusive_scan(x, s_warp, total);
    if (i < nb) sums[i] = ex + carry;
    carry += total;
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void scan_apply_kernel(ScanPair sp) {
  __shared__ int s_warp[33];
  const int q = blockIdx.y, n = sp.n;
  int32_t* in = sp.in[q];
  int32_t* out = sp.out[q];
  const int32_t* sums = sp.sums[q];
  const size_t base = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * kScanPer;
  int v[kScanPer];
  int x = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    v[k] = base + k < (size_t)n ? in[base + k] : 0;
    x += v[k];
  }
  int total;
  int ex = block_exclusive_scan(x, s_warp, total) + sums[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    if (base + k < (size_t)n) {
      out[base + k] = ex;
      in[base + k] = 0;
    }
    ex += v[k];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    out[n] = sums[gridDim.x];
    if (sp.total) sp.total[q] = sums[gridDim.x];
  }
}

// ---------------------------------------------------------------- a4-a8: forward raster
// One work item: the 8 x 4 pixel block wb of tile `tile`, sample groups of split `split`; ws is
// the warp's shared scratch.  COUNT (measurement build only): also count soft terms, covered
// samples and pass efficiency into P.counts.  EXT: the variants (texture colours,
// perspective-correct weights, sigmoid probability) are honoured; without it they are compiled
// out, so the paper's default path carries none of their code.
template <int TW, int TH, int SPT, bool MOVING, bool COUNT = false, bool EXT = false>
__device__ __forceinline__ void raster_fwd_block(const RasterParams& P, int tile, int split, int wb,
                                                 WarpScratch<SPT>& ws) {
  const int lane = threadIdx.x & 31;
  const int n_tiles = P.tiles_x * P.tiles_y;
  const int tx = tile % P.tiles_x, ty = tile / P.tiles_x;
  int px, py;
  PixelMap<TW, TH>::pixel(tx, ty, wb, px, py);
  const BlockPix bp{px - (lane & 7), py - (lane >> 3), P.W, P.H};
  const bool in_img = px < P.W && py < P.H;
  float u, v;
  bp.uv(lane, u, v);
  ws.pu[lane] = u;
  ws.pv[lane] = v;
  const TileBox tb = PixelMap<TW, TH>::warp_box(tx, ty, wb, P.W, P.H);
  const int g_begin = (int)((long long)P.G * split / P.n_split);
  const int g_end = (int)((long long)P.G * (split + 1) / P.n_split);
  float acc_r = 0.f, acc_g = 0.f, acc_b = 0.f, acc_a = 0.f;
  uint32_t n_soft = 0, n_cov = 0, n_seval = 0, n_sbatch = 0, n_ctest = 0, n_cbatch = 0;
  int adj_cost = 0;  // lane 0: soft pair batches + samples with a covered pixel (the adjoint's work)
  const long long t_start = clock64();  // this block's own time is the forward's cost measure

  for (int g = g_begin; g < g_end; ++g) {
    const Group* grp = P.groups + g;
    GroupRegs gr;
    gr.load(grp);
    const int n = gr.n;
    const uint32_t all_s = (1u << n) - 1u;
    const TriRec* recs_set = P.recs + (size_t)gr.rec_set * P.F;
    const size_t bi = (size_t)g * n_tiles + tile;
    int cb, ce, sb, se;
    P.core.range(bi, cb, ce);
    P.soft.range(bi, sb, se);

    // ---- pass 1: winners
    float bkey[SPT];
    int bestf[SPT];
    const uint32_t core_tests =
        core_raster<SPT, MOVING>(recs_set, P.core.faces, cb, ce, gr.tau, n, tb, u, v, in_img, ws, bkey, bestf);
    uint32_t uncov = 0;
#pragma unroll
    for (int i = 0; i < SPT; ++i)
      if (i < n && bestf[i] < 0) uncov |= 1u << i;

    // ---- pass 2: soft coverage of the uncovered samples
    float logp[SPT];
    int nzero[SPT];
    const uint32_t my_s = in_img ? uncov : 0u;
    uint32_t s_terms = 0, s_touch = 0;
    const uint32_t s_eval = soft_raster<SPT, MOVING>(recs_set, P.soft.faces, sb, se, gr.tau, gr.xbits, n, tb, u, v, my_s,
                                                     P.r + kCoreMargin, P.r2, P.inv_delta, EXT ? P.prob : 0, ws, logp,
                                                     nzero, s_terms, s_touch);
    adj_cost += (int)s_touch + __popc(__reduce_or_sync(kFullMask, in_img ? (all_s & ~uncov) : 0u));
    if (COUNT) {
      n_ctest += core_tests;
      n_cbatch += (uint32_t)(ce - cb + 31) / 32 * ((threadIdx.x & 31) == 0);
      n_seval += s_eval;
      n_sbatch += s_touch;
      n_soft += s_terms;
      if (in_img) n_cov += (uint32_t)n - (uint32_t)__popc(uncov);
    }

    // ---- shading of the winners (Eq. fore + Lambert) and temporal accumulation (Sec. 3.2)
    if (in_img) {
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        if (i < n) {
          const int f = bestf[i];
          if (P.s_stat) {  // the adjoint's per-sample state
            const size_t o = (size_t)(gr.k0 + i) * ((size_t)P.H * P.W) + (size_t)py * P.W + px;
            P.s_stat[o] = f >= 0 ? kStatCovered : (uint8_t)min(nzero[i], 2);
            P.s_val[o] = f >= 0 ? __int_as_float(f) : logp[i];
          }
          if (P.dbg_ids && gr.k0 + i == P.dbg_k) P.dbg_ids[(size_t)py * P.W + px] = f;
          if (f >= 0) {
            const float tau = MOVING ? __ldg(gr.tau + i) : 0.f;
            const bool persp = EXT && P.persp != 0, textured = EXT && P.tex != nullptr;
            float4 r[kRecF4];
            load_record<MOVING>(recs_set + f, r, persp, false);
            const PixelSetup<MOVING> ps = pixel_setup<MOVING>(r, u, v);
            const EdgeVals e = edge_vals<MOVING>(r, ps, tau);
            const float invD = __fdividef(1.0f, e.D);
            const float wb[3] = {e.N0 * invD, e.N1 * invD, e.N2 * invD};
            float w[3], iz[3], z[3] = {1.f, 1.f, 1.f};
            if (persp) depths_at<MOVING>(r, tau, z);
            attribute_weights(persp, wb, z, w, iz);
            float cr = 0.f, cg = 0.f, cb = 0.f, nx = 0.f, ny = 0.f, nz = 0.f, tu = 0.f, tv = 0.f;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const int vid = __ldg(P.faces + 3 * f + q);
              if (textured) {  // the vertex attribute is a texture coordinate (Eq. fore)
                tu = fmaf(w[q], __ldg(P.uv + 2 * vid), tu);
                tv = fmaf(w[q], __ldg(P.uv + 2 * vid + 1), tv);
              } else {
                cr = fmaf(w[q], __ldg(P.albedo + 3 * vid), cr);
                cg = fmaf(w[q], __ldg(P.albedo + 3 * vid + 1), cg);
                cb = fmaf(w[q], __ldg(P.albedo + 3 * vid + 2), cb);
              }
              float4 na = __ldg(P.slot_nrm + (size_t)gr.slot_a * P.V + vid);
              if (MOVING) {
                const float4 nb = __ldg(P.slot_nrm + (size_t)gr.slot_b * P.V + vid);
                na.x = fmaf(tau, nb.x - na.x, na.x);
                na.y = fmaf(tau, nb.y - na.y, na.y);
                na.z = fmaf(tau, nb.z - na.z, na.z);
              }
              nx = fmaf(w[q], na.x, nx);
              ny = fmaf(w[q], na.y, ny);
              nz = fmaf(w[q], na.z, nz);
            }
            if (textured) {
              float c[3], du[3], dv[3];
              tex_lookup(P.tex, P.tex_w, P.tex_h, tu, tv, c, du, dv);
              cr = c[0];
              cg = c[1];
              cb = c[2];
            }
            const float len = sqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
            const float dot = len > 0.f ? __fdividef(fmaf(nx, P.lx, fmaf(ny, P.ly, nz * P.lz)), len) : 0.f;
            const float shade = fmaf(P.kd, fmaxf(dot, 0.f), P.ka);
            acc_r = fmaf(cr, shade, acc_r);
            acc_g = fmaf(cg, shade, acc_g);
            acc_b = fmaf(cb, shade, acc_b);
            acc_a += 1.f;
          } else {
            acc_a += nzero[i] ? 1.f : 1.f - __expf(logp[i]);
          }
        }
      }
    }
    __syncwarp();  // the scratch is rewritten by the next group
  }
  if (lane == 0 && (P.unit_cost || P.fwd_cost)) {
    const int unit = split * UnitMap<TW, TH>::patches(n_tiles) + tile / UnitMap<TW, TH>::kTilesPerUnit;
    if (P.unit_cost && adj_cost) atomicAdd(P.unit_cost + unit, adj_cost);
    // SM cycles / 64 spent on the block (a unit's 8 blocks sum to far below 2^31)
    const int cyc = (int)min((clock64() - t_start) >> 6, (long long)(1 << 24));
    if (P.fwd_cost && cyc > 0) atomicAdd(P.fwd_cost + unit, cyc);
  }
  if (in_img) {
    const size_t o = (size_t)py * P.W + px;
    const float4 val = make_float4(acc_r * P.inv_T, acc_g * P.inv_T, acc_b * P.inv_T, acc_a * P.inv_T);
    if (P.n_split == 1) P.out[o] = val;
    else atomicAdd(P.out + o, val);  // the image was zeroed; splits add their share of the mean
  }
  if (COUNT) {
    // [soft terms, covered samples, soft evaluations, soft pair batches, coverage tests, core pair batches]
    unsigned long long c[6] = {n_soft, n_cov, n_seval, n_sbatch, n_ctest, n_cbatch};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) c[q] += __shfl_xor_sync(kFullMask, c[q], o);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 6; ++q)
        if (c[q]) atomicAdd(P.counts + q, c[q]);
    }
  }
}

// Persistent forward raster: KIND 0 = plain solver only, 1 = fast solver only, 2 = mixed batch;
// EXT: with the variants (see raster_fwd_block).
template <int TW, int TH, int SPT, int KIND, bool EXT>
__global__ void __launch_bounds__(kPersistentThreads, SPT <= 2 ? 3 : 2) raster_fwd_persistent(WorkQueue Q) {
  __shared__ CtaQueue cq;
  __shared__ RasterParams sp[kPersistentThreads / 32];
  __shared__ WarpScratch<SPT> ws[kPersistentThreads / 32];
  cq.init();
  const int warp = threadIdx.x >> 5;
  RasterParams& P = sp[warp];
  int cur = -1, tile = 0, split = 0, wb = 0;
  while (warp_next<TW, TH>(Q, cq, P, cur, tile, split, wb)) {
    if (tile >= P.tiles_x * P.tiles_y) continue;
    if (KIND == 0 || (KIND == 2 && !P.moving))
      raster_fwd_block<TW, TH, 1, false, false, EXT>(P, tile, split, wb, *reinterpret_cast<WarpScratch<1>*>(ws + warp));
    else
      raster_fwd_block<TW, TH, SPT, true, false, EXT>(P, tile, split, wb, ws[warp]);
  }
}

// Measurement build of the forward (16 x 16 tiles): the same raster, counting into P.counts.
template <int SPT, int KIND>
__global__ void __launch_bounds__(kPersistentThreads, 2) raster_fwd_count(WorkQueue Q) {
  __shared__ CtaQueue cq;
  __shared__ RasterParams sp[kPersistentThreads / 32];
  __shared__ WarpScratch<SPT> ws[kPersistentThreads / 32];
  cq.init();
  const int warp = threadIdx.x >> 5;
  RasterParams& P = sp[warp];
  int cur = -1, tile = 0, split = 0, wb = 0;
  while (warp_next<16, 16>(Q, cq, P, cur, tile, split, wb)) {
    if (tile >= P.tiles_x * P.tiles_y) continue;
    if (KIND == 0)
      raster_fwd_block<16, 16, 1, false, true>(P, tile, split, wb, *reinterpret_cast<WarpScratch<1>*>(ws + warp));
    else
      raster_fwd_block<16, 16, SPT, true, true>(P, tile, split, wb, ws[warp]);
  }
}

// ---------------------------------------------------------------- unit cost order (LPT)
// Estimated work of a unit: its bin entries over the split's groups and the patch's tiles, the
// soft entries weighted x2 (a soft term costs more than a coverage test).  Units are bucketed by
// half-octaves of the estimate and visited from the largest bucket down.
constexpr int kOrderBuckets = 64;

// bucket of a cost estimate: half-octaves, largest visited first
__device__ __forceinline__ int cost_bucket(long long cost) {
  if (cost <= 0) return 0;
  const int lg = 63 - __clzll(cost);                          // floor(log2(cost))
  const int half = lg > 0 ? (int)((cost >> (lg - 1)) & 1) : 0;  // next bit: upper half-octave
  return min(kOrderBuckets - 1, 1 + 2 * lg + half);
}

__device__ __forceinline__ int unit_bucket(const int32_t* __restrict__ core_off, const int32_t* __restrict__ soft_off,
                                           int G, int n_tiles, int tpu, int n_patches, int n_split, int u) {
  const int split = u / n_patches, patch = u - split * n_patches;
  const int g0 = (int)((long long)G * split / n_split), g1 = (int)((long long)G * (split + 1) / n_split);
  long long cost = 0;
  for (int g = g0; g < g1; ++g)
    for (int q = 0; q < tpu; ++q) {
      const int t = patch * tpu + q;
      if (t >= n_tiles) break;
      const size_t b = (size_t)g * n_tiles + t;
      cost += (long long)(core_off[b + 1] - core_off[b]) + 2LL * (soft_off[b + 1] - soft_off[b]);
    }
  return cost_bucket(cost);
}

// One CTA: bucket every unit by its cost (from the bins, or measured when cost_in is set), count
// the buckets in shared memory, scan them largest first, scatter the units.  cost_zero and
// cost_zero2 (if set) are cleared on the way (the forward raster accumulates its measured costs
// there); cost_zero may be cost_in.
constexpr int kOrderThreads = 1024;

__global__ void __launch_bounds__(kOrderThreads) unit_order_kernel(
    const int32_t* __restrict__ core_off, const int32_t* __restrict__ soft_off, int G, int n_tiles, int tpu,
    int n_patches, int n_split, const int32_t* cost_in, int32_t* cost_zero, int32_t* cost_zero2, int n_units,
    int32_t* __restrict__ bucket, int32_t* __restrict__ order) {
  __shared__ int s_hist[kOrderBuckets];
  if (threadIdx.x < kOrderBuckets) s_hist[threadIdx.x] = 0;
  __syncthreads();
  for (int u = threadIdx.x; u < n_units; u += kOrderThreads) {
    const int k = cost_in ? cost_bucket(cost_in[u])
                          : unit_bucket(core_off, soft_off, G, n_tiles, tpu, n_patches, n_split, u);
    bucket[u] = k;
    atomicAdd(&s_hist[k], 1);
    if (cost_zero) cost_zero[u] = 0;  // may be cost_in: this thread has read it
    if (cost_zero2) cost_zero2[u] = 0;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // lane l owns buckets 63 - 2l and 62 - 2l (descending order)
    const int lane = threadIdx.x;
    const int a = s_hist[kOrderBuckets - 1 - 2 * lane], b = s_hist[kOrderBuckets - 2 - 2 * lane];
    int incl = a + b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int ex = incl - a - b;
    s_hist[kOrderBuckets - 1 - 2 * lane] = ex;
    s_hist[kOrderBuckets - 2 - 2 * lane] = ex + a;
  }
  __syncthreads();
  for (int u = threadIdx.x; u < n_units; u += kOrderThreads) order[atomicAdd(&s_hist[bucket[u]], 1)] = u;
}

// ---------------------------------------------------------------- N_cand (measurement)
__global__ void count_kernel(const TriRec* __restrict__ recs, int F, const Group* __restrict__ groups, int G,
                             int W, int H, float r, unsigned long long* __restrict__ out) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long c = 0;
  if (idx < (size_t)G * F) {
    const int g = (int)(idx / F), f = (int)(idx - (size_t)g * F);
    const Group& gr = groups[g];
    const TriRec& rec = recs[(size_t)gr.rec_set * F + f];
    const bool culled = (__float_as_uint(rec.f4[kR_Z].w) & kFlagCulled) != 0;
    for (int i = 0; i < gr.n && !culled; ++i) {
      float xmin, xmax, ymin, ymax;
      swept_bbox(rec, gr.tau[i], gr.tau[i], xmin, xmax, ymin, ymax);
      int i0, i1, j0, j1;
      if (pixel_range(xmin - r, xmax + r, ymin - r, ymax + r, W, H, i0, i1, j0, j1))
        c += (unsigned long long)(i1 - i0 + 1) * (unsigned long long)(j1 - j0 + 1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// ---------------------------------------------------------------- FP32 peak (measurement)
// Independent FMA chains: each thread runs kChains chains of a = a * m + c, kUnroll steps per
// iteration, so every warp has kChains independent FMAs in flight and the FMA pipe, not the
// dependency latency, sets the rate.  m and c keep the values near 1 (no overflow, no denormals);
// the result is stored only if it equals an impossible value, so the chains cannot be removed.
constexpr int kPeakChains = 8, kPeakUnroll = 16, kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(int iters, float m, float c, float* sink) {
  float a[kPeakChains];
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) a[q] = 1.0f + 1e-3f * (float)(threadIdx.x + q);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u) {
#pragma unroll
      for (int q = 0; q < kPeakChains; ++q) a[q] = fmaf(a[q], m, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) s += a[q];
  if (s == -1.0f) sink[blockIdx.x] = s;  // never true for these chains
}

// ---------------------------------------------------------------- launch wrappers
void launch_face_normals(const float* verts, const int32_t* faces, int F, int V, float* nacc, int* status,
                         cudaStream_t st) {
  if (F > 0) face_normals_kernel<<<(F + 255) / 256, 256, 0, st>>>(verts, faces, F, V, nacc, status);
}

void launch_xform(const float* verts, const float* nacc, int V, const SlotXform* xf, int n_slots, float th,
                  float4* pos, float4* nrm, cudaStream_t st) {
  dim3 grid((V + 255) / 256, n_slots);
  xform_kernel<<<grid, 256, 0, st>>>(verts, nacc, V, xf, th, pos, nrm);
}

void launch_setup(const float4* pos, const int32_t* faces, int F, int V, const int2* set_slots, int n_sets,
                  float znear, TriRec* recs, cudaStream_t st) {
  const size_t n = (size_t)n_sets * F;
  if (n) setup_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pos, faces, F, V, set_slots, n_sets, znear, recs);
}

void launch_bin(bool fill, const TriRec* recs, int F, const Group* groups, int G, int W, int H, int tw, int th,
                int tiles_x, int n_tiles, float r_core, float r_soft, const BinTargets& t, int* status,
                cudaStream_t st) {
  const size_t n = (size_t)G * F;
  if (!n) return;
  if (n_tiles <= kSmemBinTiles && G <= 65535) {
    const dim3 grid((unsigned)((F + 255) / 256), (unsigned)G);
    const size_t smem = sizeof(int) * 2 * (size_t)n_tiles;
    if (fill)
      bin_smem_kernel<true><<<grid, 256, smem, st>>>(recs, F, groups, W, H, tw, th, tiles_x, n_tiles, r_core, r_soft,
                                                     t, status);
    else
      bin_smem_kernel<false><<<grid, 256, smem, st>>>(recs, F, groups, W, H, tw, th, tiles_x, n_tiles, r_core, r_soft,
                                                      t, status);
    return;
  }
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (fill)
    bin_kernel<true><<<blocks, 256, 0, st>>>(recs, F, groups, G, W, H, tw, th, tiles_x, n_tiles, r_core, r_soft, t,
                                             status);
  else
    bin_kernel<false><<<blocks, 256, 0, st>>>(recs, F, groups, G, W, H, tw, th, tiles_x, n_tiles, r_core, r_soft, t,
                                              status);
}

size_t scan_temp_ints(int n) { return (size_t)(n + kScanBlock - 1) / kScanBlock + 1; }

int launch_scan_pair(const ScanPair& sp, cudaStream_t st) {
  const int nb = (sp.n + kScanBlock - 1) / kScanBlock;
  if (nb == 0) return 0;  // callers only scan non-empty bin arrays
  scan_reduce_kernel<<<dim3(nb, 2), kScanThreads, 0, st>>>(sp);
  scan_sums_kernel<<<dim3(1, 2), kScanThreads, 0, st>>>(sp, nb);
  scan_apply_kernel<<<dim3(nb, 2), kScanThreads, 0, st>>>(sp);
  return 3;
}

template <int TW, int TH, int KIND, bool EXT>
static void launch_fwd_spt(const WorkQueue& Q, int spt, int grid, cudaStream_t st) {
  if (spt <= 2)
    raster_fwd_persistent<TW, TH, 2, KIND, EXT><<<grid, kPersistentThreads, 0, st>>>(Q);
  else
    raster_fwd_persistent<TW, TH, 4, KIND, EXT><<<grid, kPersistentThreads, 0, st>>>(Q);
}

template <int TW, int TH, bool EXT>
static void launch_fwd_tile(const WorkQueue& Q, int spt, int kind, int grid, cudaStream_t st) {
  if (kind == 0)
    raster_fwd_persistent<TW, TH, 1, 0, EXT><<<grid, kPersistentThreads, 0, st>>>(Q);
  else if (kind == 1)
    launch_fwd_spt<TW, TH, 1, EXT>(Q, spt, grid, st);
  else
    launch_fwd_spt<TW, TH, 2, EXT>(Q, spt, grid, st);
}

template <typename K>
static int occupancy_of(K kernel) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kPersistentThreads, 0) != cudaSuccess) n = 1;
  return n < 1 ? 1 : n;
}

template <int TW, int TH, bool EXT>
static int occ_fwd(int spt, int kind) {
  if (kind == 0) return occupancy_of(raster_fwd_persistent<TW, TH, 1, 0, EXT>);
  if (kind == 1)
    return spt <= 2 ? occupancy_of(raster_fwd_persistent<TW, TH, 2, 1, EXT>)
                    : occupancy_of(raster_fwd_persistent<TW, TH, 4, 1, EXT>);
  return spt <= 2 ? occupancy_of(raster_fwd_persistent<TW, TH, 2, 2, EXT>)
                  : occupancy_of(raster_fwd_persistent<TW, TH, 4, 2, EXT>);
}

// kind: kKindPlain / kKindFast / kKindMixed, plus kKindExt for the variant kernels
int persistent_grid_fwd(int num_sms, int tile, int spt, int kind) {
  const int k = kind & kKindMask;
  int occ;
  if (kind & kKindExt) occ = tile == 8 ? occ_fwd<8, 8, true>(spt, k) : occ_fwd<16, 16, true>(spt, k);
  else occ = tile == 8 ? occ_fwd<8, 8, false>(spt, k) : occ_fwd<16, 16, false>(spt, k);
  return num_sms * occ;
}

void launch_raster_fwd(const WorkQueue& Q, int tile, int spt, int kind, int grid, cudaStream_t st) {
  if (Q.n_work <= 0) return;
  const int k = kind & kKindMask;
  if (kind & kKindExt) {
    if (tile == 8) launch_fwd_tile<8, 8, true>(Q, spt, k, grid, st);
    else launch_fwd_tile<16, 16, true>(Q, spt, k, grid, st);
  } else {
    if (tile == 8) launch_fwd_tile<8, 8, false>(Q, spt, k, grid, st);
    else launch_fwd_tile<16, 16, false>(Q, spt, k, grid, st);
  }
}

double launch_fma_peak(int num_sms, int iters, float* sink, cudaStream_t st) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel, kPeakThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int grid = num_sms * per_sm;
  fma_peak_kernel<<<grid, kPeakThreads, 0, st>>>(iters, 0.999999f, 1e-6f, sink);
  return 2.0 * kPeakChains * kPeakUnroll * (double)iters * grid * kPeakThreads;  // FMA = 2 flops
}

size_t unit_order_ints(int n_units) { return (size_t)n_units; }

void launch_unit_order(const int32_t* core_off, const int32_t* soft_off, int G, int n_tiles, int tile, int n_split,
                       int n_units, int32_t* order, int32_t* scratch, int32_t* cost_zero, int32_t* cost_zero2,
                       cudaStream_t st) {
  if (n_units <= 0) return;
  const int tpu = tile == 8 ? UnitMap<8, 8>::kTilesPerUnit : UnitMap<16, 16>::kTilesPerUnit;
  const int n_patches = (n_tiles + tpu - 1) / tpu;
  unit_order_kernel<<<1, kOrderThreads, 0, st>>>(core_off, soft_off, G, n_tiles, tpu, n_patches, n_split, nullptr,
                                                 cost_zero, cost_zero2, n_units, scratch, order);
}

void launch_unit_order_measured(const int32_t* cost, int n_units, int32_t* order, int32_t* scratch,
                                int32_t* cost_zero, int32_t* cost_zero2, cudaStream_t st) {
  if (n_units <= 0) return;
  unit_order_kernel<<<1, kOrderThreads, 0, st>>>(nullptr, nullptr, 0, 0, 1, 1, 1, cost, cost_zero, cost_zero2,
                                                 n_units, scratch, order);
}

void launch_raster_count(const WorkQueue& Q, int spt, int kind, int grid, cudaStream_t st) {
  if (Q.n_work <= 0) return;
  if ((kind & kKindMask) == 0) raster_fwd_count<1, 0><<<grid, kPersistentThreads, 0, st>>>(Q);
  else if (spt <= 2) raster_fwd_count<2, 1><<<grid, kPersistentThreads, 0, st>>>(Q);
  else raster_fwd_count<4, 1><<<grid, kPersistentThreads, 0, st>>>(Q);
}

void launch_count(const TriRec* recs, int F, const Group* groups, int G, int W, int H, float r,
                  unsigned long long* out, cudaStream_t st) {
  const size_t n = (size_t)G * F;
  if (n) count_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(recs, F, groups, G, W, H, r, out);
}

}  // namespace mbr
