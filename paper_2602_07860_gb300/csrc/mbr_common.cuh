// mbr_common.cuh -- shared device-side definitions of the sm_103a renderer kernels.
//
// Data layout in HBM (per call, owned by the context):
//   slot_pos[slot][V]  float4 (ndc x, ndc y, camera z, 0)   -- vertex state at a slot time
//   slot_nrm[slot][V]  float4 (world normal xyz, 0)
//   recs[set][F]       TriRec (11 x float4)                   -- per (record set, face) setup
//   groups[G]          Group                                  -- samples sharing a record set
//   bins               CSR over (group, tile): face ids       -- tile binning
// A "slot" is a time at which vertices are placed exactly: the S+1 keyframes s/S of the fast
// solver or the T sub-frame times of the plain solver.  A "record set" is what a group's
// samples share: one linear segment (fast: keyframes s, s+1) or one sub-frame (plain).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mbr {

constexpr int kMaxSpt = 4;            // samples per group (max)
constexpr float kDetMin = 1e-10f;     // |det F| at or below: triangle skipped at that sample
constexpr int kRecF4 = 11;            // float4s per triangle record

// Per (record set, face) triangle record.  Local frame: origin o = v0 at the set's first
// keyframe; e1 = v1 - v0, e2 = v2 - v0 at that keyframe; d1, d2 = change of e1, e2 over the
// segment; g = displacement of v0 over the segment.  With q0 = p - o the edge functions are
//   N1(tau) = cross(q0 - tau g, e2 + tau d2),  N2(tau) = cross(e1 + tau d1, q0 - tau g),
//   D(tau)  = cross(e1 + tau d1, e2 + tau d2), N0 = D - N1 - N2,
// i.e. the numerators / denominator of Eq. time-dependent2 written about a moving local origin
// (the coefficients are the appendix's A_1..A_3, a_1..a_3 up to the change of origin).
//   f4[0] = (ox, oy, e1x, e1y)        f4[1] = (e2x, e2y, D0, face bits)
//   f4[2] = (z0_0, z0_1, z0_2, flags) f4[3] = bounding box at the first keyframe
//                                              (xmin, xmax, ymin, ymax)
//   f4[4] = change of that box over the segment (the box of the lerped triangle at tau lies in
//           the lerp of the two keyframe boxes)
//   f4[5] = (d1x, d1y, d2x, d2y)      f4[6] = (gx, gy, c1, c2)
//   f4[7] = (a11, a12, D1, D2)        f4[8] = (dz0, dz1, dz2, 0)
//   f4[9], f4[10] = 1 / |edge|^2 of the edges (v0,v1), (v1,v2), (v2,v0) at the first / second
//           keyframe (0 for a zero-length edge) -- the closest-point search of the soft term
// with c1 = -cross(g, e2), c2 = -cross(e1, g), a11 = -cross(g, d2), a12 = -cross(d1, g),
// D0 = cross(e1, e2), D1 = cross(e1, d2) + cross(d1, e2), D2 = cross(d1, d2).
// Static (plain) records only use f4[0..3].
struct TriRec {
  float4 f4[kRecF4];
};

constexpr uint32_t kFlagCulled = 1u;  // a vertex at camera z <= znear: skipped for the whole set

// device status word bits (read back by the host after the binning sync)
constexpr int kStatusBadFace = 1;       // a face index outside [0, V)
constexpr int kStatusBinOverflow = 2;   // fill pass disagreed with the count pass
constexpr int kStatusSpin = 4;          // a raster CTA gave up a bounded wait (result incomplete)

struct Group {
  int32_t rec_set;     // record set of the group's samples
  int32_t slot_a;      // slot of the set's first keyframe (normals lerp from slot_a to slot_b)
  int32_t slot_b;
  int32_t n;           // samples in this group (1..kMaxSpt)
  int32_t k0;          // sub-frame index of the first sample (samples are k0 .. k0+n-1)
  uint32_t xbits;      // bit i set: keyframe X = 1 for sample i (Eq. euc-dist-approx-2)
  float tau_lo, tau_hi;  // local-time range of the samples (swept bounding box for binning)
  float tau[kMaxSpt];
};

struct SlotXform {      // one slot: world -> camera affine map and world normal rotation
  float A[12];          // camera = A [v; 1]  (view composed with the motion at the slot time)
  float R[9];           // world normal at the slot = R n_base
  float t;              // slot time
  float pad[2];
};

__device__ __forceinline__ float cross2(float ax, float ay, float bx, float by) {
  return fmaf(ax, by, -ay * bx);
}

__device__ __forceinline__ int float_as_int_bits(float f) { return __float_as_int(f); }

// Closest point of the triangle (0, e1, e2) (local frame of vertex 0) to point (px, py), by the
// appendix's three clamped edge projections in the order (v0,v1), (v1,v2), (v2,v0), keeping the
// first minimum.  Returns squared distance; outputs barycentrics (w0, w1, w2), the region
// (0..2 interior of edge, 3 + i vertex i), the edge slots (ei, ej) and the clamped parameter t.
struct Closest {
  float d2, w0, w1, w2, t;
  int region, ei, ej;
};

__device__ __forceinline__ Closest closest_local(float e1x, float e1y, float e2x, float e2y,
                                                float px, float py, const float4& inv_len2) {
  Closest c;
  c.d2 = INFINITY;
  c.w0 = c.w1 = c.w2 = 0.f;
  c.t = 0.f;
  c.region = 0;
  c.ei = 0;
  c.ej = 1;
  const float vx[3] = {0.f, e1x, e2x};
  const float vy[3] = {0.f, e1y, e2y};
  const float iL[3] = {inv_len2.x, inv_len2.y, inv_len2.z};
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const int i = e, j = (e + 1) % 3;
    const float ax = vx[i], ay = vy[i];
    const float ex = vx[j] - ax, ey = vy[j] - ay;
    const float rx = px - ax, ry = py - ay;
    float t = fmaf(rx, ex, ry * ey) * iL[e];
    int reg = e;
    float qx, qy;
    if (t <= 0.f) {
      t = 0.f; qx = ax; qy = ay; reg = 3 + i;
    } else if (t >= 1.f) {
      t = 1.f; qx = vx[j]; qy = vy[j]; reg = 3 + j;
    } else {
      qx = fmaf(t, ex, ax); qy = fmaf(t, ey, ay);
    }
    const float dx = px - qx, dy = py - qy;
    const float d2 = fmaf(dx, dx, dy * dy);
    if (d2 < c.d2) {
      c.d2 = d2;
      c.region = reg;
      c.ei = i;
      c.ej = j;
      c.t = t;
      float w[3] = {0.f, 0.f, 0.f};
      w[i] = 1.f - t;
      w[j] = t;
      c.w0 = w[0]; c.w1 = w[1]; c.w2 = w[2];
    }
  }
  return c;
}

}  // namespace mbr
