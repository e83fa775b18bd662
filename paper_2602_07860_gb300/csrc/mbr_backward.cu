// mbr_backward.cu -- adjoint kernels of the sm_103a motion-blurred renderer (a9).
//
//   raster_bwd_persistent back-propagates dL/dimage from the forward raster's per-sample
//                      state: through shading (Eq. fore + Lambert) and the
//                      barycentric edge functions of the stored winners, and through the
//                      soft-coverage product (Eqs. probability-function .. back, exclusive
//                      products) of the uncovered samples, into gradients on the slot vertex
//                      states (ndc x, y and world normal); soft-term gradients are warp-reduced
//                      per candidate before the atomics
//   slot_chain_kernel  slot-state gradients -> base vertex gradients through projection, camera
//                      and motion; base-normal gradient -> area-weighted-normal gradient
//   normals_bwd_kernel adjoint of the face cross products of the vertex normals (a0)
#include <algorithm>
#include <cstdint>

#include "mbr_internal.h"
#include "mbr_raster.cuh"

namespace mbr {

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// gradient of the edge functions N_q (at tau, local frame) w.r.t. the three vertex positions:
// N0 = cross(a1, a2), N1 = cross(a2, a0), N2 = cross(a0, a1) with a_i = v_i(tau) - p.
__device__ __forceinline__ void edge_backward(float gN0, float gN1, float gN2, const float ax[3],
                                              const float ay[3], float gx[3], float gy[3]) {
  // d cross(a, b) / da = (b.y, -b.x), / db = (-a.y, a.x)
  gx[0] = gN1 * -ay[2] + gN2 * ay[1];
  gy[0] = gN1 * ax[2] + gN2 * -ax[1];
  gx[1] = gN0 * ay[2] + gN2 * -ay[0];
  gy[1] = gN0 * -ax[2] + gN2 * ax[0];
  gx[2] = gN0 * -ay[1] + gN1 * ay[0];
  gy[2] = gN0 * ax[1] + gN1 * -ax[0];
}

// vertex positions relative to the pixel at tau: a_i = v_i(tau) - p
template <bool MOVING>
__device__ __forceinline__ void rel_vertices(const float4* r, const PixelSetup<MOVING>& ps, float tau,
                                             float ax[3], float ay[3]) {
  const float qtx = MOVING ? fmaf(-tau, r[kR_G].x, ps.q0x) : ps.q0x;
  const float qty = MOVING ? fmaf(-tau, r[kR_G].y, ps.q0y) : ps.q0y;
  const float e1x = MOVING ? fmaf(tau, r[kR_D].x, r[kR_O].z) : r[kR_O].z;
  const float e1y = MOVING ? fmaf(tau, r[kR_D].y, r[kR_O].w) : r[kR_O].w;
  const float e2x = MOVING ? fmaf(tau, r[kR_D].z, r[kR_E2].x) : r[kR_E2].x;
  const float e2y = MOVING ? fmaf(tau, r[kR_D].w, r[kR_E2].y) : r[kR_E2].y;
  ax[0] = -qtx; ay[0] = -qty;
  ax[1] = e1x - qtx; ay[1] = e1y - qty;
  ax[2] = e2x - qtx; ay[2] = e2y - qty;
}

// Gradient of one soft factor's distance d w.r.t. the vertex positions, scaled by gd = dL/dd:
// accumulated into the slot-a (keyframe 0 / sub-frame) and slot-b (keyframe 1) sums.
// Plain solver: exact distance, d d / d v_i = 2 (F w* - p) w*_i (envelope).
__device__ __forceinline__ void soft_grad_plain(const Closest& c, float rx, float ry, float gd, float (&gax)[3],
                                                float (&gay)[3]) {
  const float grx = 2.f * rx * gd, gry = 2.f * ry * gd;  // d/d(F w* - p)
  const float ws_[3] = {c.w0, c.w1, c.w2};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    gax[q] = fmaf(ws_[q], grx, gax[q]);
    gay[q] = fmaf(ws_[q], gry, gay[q]);
  }
}

// Fast solver: d = |F(tau) w* - p|^2 with w* the closest point in F(X) to p' = F(X) w(tau) (Eqs.
// euc-dist-approx-1..3), differentiated through w*, p' and w(tau) = N / D.  k: the term's
// coefficients at tau (soft_affine: F(X)'s edges in k[2], F(tau)'s in k[4], tau g in k[3].w and
// k[5].x); ev: its evaluation at the pixel; (w1, w2) = w(tau); iD = 1 / D(tau).
__device__ __forceinline__ void soft_grad_fast(const float4 (&k)[6], const SoftEval& ev, float w1, float w2, float iD,
                                               float tau, int X, float gd, float (&gax)[3], float (&gay)[3],
                                               float (&gbx)[3], float (&gby)[3]) {
  const float grx = 2.f * ev.rx * gd, gry = 2.f * ev.ry * gd;  // d/d(F(tau) w* - p)
  const float ws_[3] = {ev.c.w0, ev.c.w1, ev.c.w2};
  float gtx[3], gty[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    gtx[q] = ws_[q] * grx;
    gty[q] = ws_[q] * gry;
  }
  // local vertex positions at tau and at keyframe X
  const float Vtx[3] = {0.f, k[4].x, k[4].z}, Vty[3] = {0.f, k[4].y, k[4].w};
  const float VXx[3] = {0.f, k[2].x, k[2].z}, VXy[3] = {0.f, k[2].y, k[2].w};
  float gXx[3] = {0.f, 0.f, 0.f}, gXy[3] = {0.f, 0.f, 0.f};
  float gpx = 0.f, gpy = 0.f;
  if (ev.c.region < 3) {
    // w*_i = 1 - t, w*_j = t, t = ((p' - V_i) . E) / |E|^2 on edge (i, j) of F(X)
    const int ei = ev.c.ei, ej = ev.c.ej;
    float gti = 0.f, gtj = 0.f, Ex = 0.f, Ey = 0.f, Rx = 0.f, Ry = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q == ei) {
        gti = Vtx[q] * grx + Vty[q] * gry;
        Rx = ev.ppx - VXx[q];
        Ry = ev.ppy - VXy[q];
        Ex -= VXx[q];
        Ey -= VXy[q];
      }
      if (q == ej) {
        gtj = Vtx[q] * grx + Vty[q] * gry;
        Ex += VXx[q];
        Ey += VXy[q];
      }
    }
    const float L2 = fmaf(Ex, Ex, Ey * Ey);
    const float gt = __fdividef(gtj - gti, L2), t = ev.c.t;
    gpx = gt * Ex;
    gpy = gt * Ey;
    const float gix = gt * (-Ex - Rx + 2.f * t * Ex), giy = gt * (-Ey - Ry + 2.f * t * Ey);
    const float gjx = gt * (Rx - 2.f * t * Ex), gjy = gt * (Ry - 2.f * t * Ey);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (q == ei) { gXx[q] += gix; gXy[q] += giy; }
      if (q == ej) { gXx[q] += gjx; gXy[q] += gjy; }
    }
  }
  // p' = F(X) w(tau)
  const float w0 = 1.f - w1 - w2;
  const float wv[3] = {w0, w1, w2};
  float gw[3];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    gXx[q] = fmaf(wv[q], gpx, gXx[q]);
    gXy[q] = fmaf(wv[q], gpy, gXy[q]);
    gw[q] = VXx[q] * gpx + VXy[q] * gpy;
  }
  // w = N / D with D = N0 + N1 + N2; the N_i are cross products of the vertices relative to the
  // pixel at tau, a_i = v_i(tau) - p (local frame: v_0(tau) - p = -(q - tau g))
  const float sw = wv[0] * gw[0] + wv[1] * gw[1] + wv[2] * gw[2];
  const float qtx = ev.qx - k[3].w, qty = ev.qy - k[5].x;
  const float ax[3] = {-qtx, Vtx[1] - qtx, Vtx[2] - qtx}, ay[3] = {-qty, Vty[1] - qty, Vty[2] - qty};
  float ex[3], ey[3];
  edge_backward((gw[0] - sw) * iD, (gw[1] - sw) * iD, (gw[2] - sw) * iD, ax, ay, ex, ey);
  // F(tau) = lerp of the two keyframes; F(X) is keyframe X
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    gtx[q] += ex[q];
    gty[q] += ey[q];
    gax[q] = fmaf(1.f - tau, gtx[q], gax[q]);
    gay[q] = fmaf(1.f - tau, gty[q], gay[q]);
    gbx[q] = fmaf(tau, gtx[q], gbx[q]);
    gby[q] = fmaf(tau, gty[q], gby[q]);
    if (X == 0) {
      gax[q] += gXx[q];
      gay[q] += gXy[q];
    } else {
      gbx[q] += gXx[q];
      gby[q] += gXy[q];
    }
  }
}

// pairs per lane slot of the fast solver's batches
constexpr int kPairsPerLane = 2;

// pass 3 of the adjoint: gradient of alpha = 1 - prod_j (1 - A_j) w.r.t. the vertex positions of
// every soft candidate, summed per candidate into its row of the chunk in shared memory; each row
// is added to the slot gradients once, when its chunk is done.
//   fast solver (batches)  a batch's pairs of one face sit on consecutive lanes: a segmented warp
//                          sum (as many halving steps as the batch's longest run needs) gives one
//                          head per face and batch, which adds the run's total to the row;
//   plain solver (runs)    each lane sums its run of pairs in registers while they belong to one
//                          candidate and adds the sum to the candidate's row when the candidate
//                          changes (shared-memory atomics: a candidate's pairs may span runs).
// The fast solver reads eight staged rows per term, which a batch's lanes of one candidate read as
// broadcasts; the plain solver's terms are short, so the warp sum would dominate them.
template <int SPT, bool MOVING>
struct BwdSoftGradPairs {
  const TriRec* recs_set;
  const Group* grp;
  BlockPix bp;
  BwdScratch<SPT>* ws;
  uint32_t xbits;
  float m, r2, inv_delta;
  int prob;
  const int32_t* faces;
  float4* gslot_a;
  float4* gslot_b;
  float gax[3], gay[3], gbx[3], gby[3];  // this lane's sums
  int cur;                               // runs: the candidate they belong to (-1: none)
  // with at most two samples per group the fast solver's pairs read the term's coefficients at
  // each sample time, formed once per candidate when its chunk is laid out (8 rows per sample:
  // soft_affine's k[0..4], (k[5].x, 1 / D, w1u, w1v), (w1c, w2u, w2v, w2c), the box at tau dilated
  // by m); otherwise they read the staged record and form the coefficients per pair
  static constexpr bool kAff = MOVING && SPT == 2;
  __device__ __forceinline__ void stage(const TriRec* rec, uint32_t sm) {
    const int lane = threadIdx.x & 31;
    if constexpr (kAff) {
      const float4 o = __ldg(&rec->f4[kR_O]), e2 = __ldg(&rec->f4[kR_E2]), d = __ldg(&rec->f4[kR_D]);
      const float4 g = __ldg(&rec->f4[kR_G]), a = __ldg(&rec->f4[kR_A]);
      const float4 b = __ldg(&rec->f4[kR_BB]), db = __ldg(&rec->f4[kR_DBB]);
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        if (!((sm >> i) & 1u)) continue;
        const float tau = __ldg(&grp->tau[i]);
        const int X = (xbits >> i) & 1u;
        const float D = fmaf(fmaf(a.w, tau, a.z), tau, e2.z);
        float4* row = ws->coef[lane] + 8 * i;
        if (!(fabsf(D) > kDetMin)) {
          row[7] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);  // no pixel passes
          continue;
        }
        const SoftAffine sa = soft_affine(o, e2, d, g, a, __ldg(&rec->f4[X ? kR_IL1 : kR_IL0]), tau, X, D);
#pragma unroll
        for (int q = 0; q < 5; ++q) row[q] = sa.k[q];
        row[5] = make_float4(sa.k[5].x, __fdividef(1.0f, D), sa.w1u, sa.w1v);
        row[6] = make_float4(sa.w1c, sa.w2u, sa.w2v, sa.w2c);
        row[7] = make_float4(fmaf(tau, db.x, b.x) - m, fmaf(tau, db.y, b.y) + m, fmaf(tau, db.z, b.z) - m,
                             fmaf(tau, db.w, b.w) + m);
      }
    } else {
#pragma unroll
      for (int q = 0; q < kRecF4; ++q)
        if (MOVING || q == kR_O || q == kR_E2 || q == kR_Z || q == kR_BB || q == kR_IL0) ws->coef[lane][q] = __ldg(&rec->f4[q]);
    }
  }
  // the factor's share of dL/dd: gd = dL/dalpha * prod_{l != j} (1 - A_l) * dA_j/dd
  __device__ __forceinline__ float factor_grad(float d, float ga, int i, int p) const {
    float A, dA;
    const float f = soft_factor(d, inv_delta, prob, A, dA);
    const float S = ws->logp[i][p];
    const int nz = ws->nzero[i][p];
    // the product of the other factors, each <= 1 (the bound keeps a factor that rounds to 0
    // from turning it into infinity)
    float excl;
    if (nz == 0) excl = fminf(__expf(S - __logf(f)), 1.f);
    else excl = (nz == 1 && f <= kTinyFactor) ? __expf(S) : 0.f;
    return ga * excl * dA;
  }
  // batches: the sums start from zero in every batch and take the lane's pairs
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int q = 0; q < 3; ++q) gax[q] = gay[q] = gbx[q] = gby[q] = 0.f;
  }
  __device__ __forceinline__ void pair(int face, int p, uint32_t smp, int slot) { accumulate(p, smp, slot); }
  // runs: the sums carry over while the candidate stays the same
  __device__ __forceinline__ void pair_run(int face, int p, uint32_t smp, int slot) {
    if (slot != cur) {
      flush();
      cur = slot;
    }
    accumulate(p, smp, slot);
  }
  // the soft terms of one pair (candidate slot of the chunk, block pixel p, samples smp), added
  // to this lane's sums
  __device__ __forceinline__ void accumulate(int p, uint32_t smp, int slot) {
    const float u = ws->pu[p], v = ws->pv[p];
    const float ga = ws->ga[p];
    if constexpr (kAff) {
      while (smp) {
        const int i = __ffs(smp) - 1;
        smp &= smp - 1u;
        const float4* row = ws->coef[slot] + 8 * i;
        const float4 bx = row[7];
        if (!(u >= bx.x && u <= bx.y && v >= bx.z && v <= bx.w)) continue;
        float4 k[6];
#pragma unroll
        for (int q = 0; q < 5; ++q) k[q] = row[q];
        const float4 r5 = row[5];
        k[5] = make_float4(r5.x, 0.f, 0.f, 0.f);
        // the term exactly as the forward's soft pass evaluates it (same coefficients)
        const SoftEval ev = soft_affine_eval(k, u, v);
        if (!(ev.d <= r2)) continue;
        const float gd = factor_grad(ev.d, ga, i, p);
        if (gd == 0.f) continue;
        const float4 r6 = row[6];
        const float w1 = fmaf(ev.qx, r5.z, fmaf(ev.qy, r5.w, r6.x));
        const float w2 = fmaf(ev.qx, r6.y, fmaf(ev.qy, r6.z, r6.w));
        soft_grad_fast(k, ev, w1, w2, r5.y, __ldg(&grp->tau[i]), (xbits >> i) & 1u, gd, gax, gay, gbx, gby);
      }
      return;
    }
    // the candidate's record, staged in shared memory when its chunk was laid out
    float4 r[kRecF4];
    r[kR_O] = ws->coef[slot][kR_O];
    r[kR_E2] = ws->coef[slot][kR_E2];
    r[kR_IL0] = ws->coef[slot][kR_IL0];
    if (MOVING) {
      r[kR_IL1] = ws->coef[slot][kR_IL1];
      r[kR_BB] = ws->coef[slot][kR_BB];
      r[kR_DBB] = ws->coef[slot][kR_DBB];
      r[kR_D] = ws->coef[slot][kR_D];
      r[kR_G] = ws->coef[slot][kR_G];
      r[kR_A] = ws->coef[slot][kR_A];
    }
    const PixelSetup<MOVING> ps = pixel_setup<MOVING>(r, u, v);
    while (smp) {
      const int i = __ffs(smp) - 1;
      smp &= smp - 1u;
      const float tau = MOVING ? __ldg(&grp->tau[i]) : 0.f;
      const int X = (xbits >> i) & 1u;
      if (MOVING) {
        // the term exactly as the forward's soft pass evaluates it (soft_affine)
        if (!in_box_at(r, tau, m, u, v)) continue;
        const float D = fmaf(fmaf(r[kR_A].w, tau, r[kR_A].z), tau, r[kR_E2].z);
        if (!(fabsf(D) > kDetMin)) continue;
        const SoftAffine sa = soft_affine(r[kR_O], r[kR_E2], r[kR_D], r[kR_G], r[kR_A], X ? r[kR_IL1] : r[kR_IL0], tau,
                                          X, D);
        const SoftEval ev = soft_affine_eval(sa.k, u, v);
        if (!(ev.d <= r2)) continue;
        const float gd = factor_grad(ev.d, ga, i, p);
        if (gd == 0.f) continue;
        const float w1 = fmaf(ev.qx, sa.w1u, fmaf(ev.qy, sa.w1v, sa.w1c));
        const float w2 = fmaf(ev.qx, sa.w2u, fmaf(ev.qy, sa.w2v, sa.w2c));
        soft_grad_fast(sa.k, ev, w1, w2, __fdividef(1.0f, D), tau, X, gd, gax, gay, gbx, gby);
      } else {
        EdgeVals e;
        SoftGeom sg;
        if (!soft_pair_term<MOVING>(r, ps, u, v, tau, X, m, r2, e, sg)) continue;
        const float gd = factor_grad(sg.d, ga, i, p);
        if (gd == 0.f) continue;
        soft_grad_plain(sg.c, sg.rx, sg.ry, gd, gax, gay);
      }
    }
  }
  // runs: this lane's sums of the current candidate into its row of the chunk
  __device__ __forceinline__ void flush() {
    if (cur >= 0) {
      float* row = ws->grow[cur];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (gax[q] != 0.f) atomicAdd(row + 2 * q, gax[q]);
        if (gay[q] != 0.f) atomicAdd(row + 2 * q + 1, gay[q]);
        if (MOVING && gbx[q] != 0.f) atomicAdd(row + 6 + 2 * q, gbx[q]);
        if (MOVING && gby[q] != 0.f) atomicAdd(row + 6 + 2 * q + 1, gby[q]);
        gax[q] = gay[q] = gbx[q] = gby[q] = 0.f;
      }
    }
    cur = -1;
  }
  __device__ __forceinline__ void chunk_begin() {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < (MOVING ? 12 : 6); ++k) ws->grow[lane][k] = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) gax[q] = gay[q] = gbx[q] = gby[q] = 0.f;
    cur = -1;
    __syncwarp();
  }
  // the batch's pairs of one face sit on consecutive lanes: a segmented warp sum (as many halving
  // steps as the batch's longest run needs); the first lane of each run adds the run's total to the
  // face's row of the chunk (one head per face and batch, so no two lanes add to one row)
  __device__ __forceinline__ void batch_end(int face, int slot) {
    const int lane = threadIdx.x & 31;
    bool mine = false;
#pragma unroll
    for (int q = 0; q < 3; ++q) mine |= gax[q] != 0.f || gay[q] != 0.f || (MOVING && (gbx[q] != 0.f || gby[q] != 0.f));
    if (!__any_sync(kFullMask, mine)) return;
    const int prev = __shfl_up_sync(kFullMask, face, 1);
    const bool head = face >= 0 && (lane == 0 || prev != face);
    const uint32_t heads = __ballot_sync(kFullMask, head);
    const uint32_t above = lane == 31 ? 0u : (heads & (kFullMask << (lane + 1)));
    const int seg_end = above ? __ffs(above) - 1 : 32;
    // lanes without a pair (face < 0) trail the batch: a run ends at the last lane with a pair
    const int n_valid = __popc(__ballot_sync(kFullMask, face >= 0));
    const int longest = __reduce_max_sync(kFullMask, head ? min(seg_end, n_valid) - lane : 0);
    constexpr int NV = MOVING ? 12 : 6;
    float vals[NV];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      vals[2 * q] = gax[q];
      vals[2 * q + 1] = gay[q];
      if (MOVING) {
        vals[6 + 2 * q] = gbx[q];
        vals[6 + 2 * q + 1] = gby[q];
      }
    }
#pragma unroll 1
    for (int o = 1; o < longest; o <<= 1) {
      const bool take = lane + o < seg_end;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const float y = __shfl_down_sync(kFullMask, vals[q], o);
        if (take) vals[q] += y;
      }
    }
    if (head) {
#pragma unroll
      for (int q = 0; q < NV; ++q) ws->grow[slot][q] += vals[q];
    }
    __syncwarp();  // the next batch's heads read the rows
  }
  // candidate j's gradient summed over the chunk's pairs: one set of atomics per face
  __device__ __forceinline__ void chunk_end(int face, bool had_pairs) {
    const int lane = threadIdx.x & 31;
    constexpr int NV = MOVING ? 12 : 6;
    if (had_pairs) {
      float vals[NV];
      bool any = false;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        vals[q] = ws->grow[lane][q];
        any |= vals[q] != 0.f;
      }
      if (any) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int vid = __ldg(faces + 3 * face + q);
          atomicAdd(reinterpret_cast<float2*>(gslot_a + (size_t)vid * 2), make_float2(vals[2 * q], vals[2 * q + 1]));
          if (MOVING)
            atomicAdd(reinterpret_cast<float2*>(gslot_b + (size_t)vid * 2),
                      make_float2(vals[6 + 2 * q], vals[6 + 2 * q + 1]));
        }
      }
    }
    __syncwarp();
  }
};

// Adjoint of one covered sample: shading (Eq. fore + Lambert) and w = N / D through the edge
// functions to the slot states of the winner's vertices.  Lanes that share a winner face are
// summed in shared memory (ws_rows, one row per lane) and their lowest lane adds them, so each
// distinct face of the warp costs one set of vector atomics.  Warp-collective: every lane calls it; lanes without a covered sample pass
// has = false.  EXT: texture colours and perspective-correct weights are honoured (see
// raster_fwd_block); without it they are compiled out.
template <bool MOVING, bool EXT, int R>
__device__ __forceinline__ void covered_adjoint(const RasterParams& P, const TriRec* recs_set, int slot_a, int slot_b,
                                                bool has, int f, float tau, float u, float v, float gr, float gg,
                                                float gb, float4 (*ws_rows)[R]) {
  // per-vertex contributions: slot a (dx, dy, dnx, dny | dnz, dz), slot b (same), albedo (r, g, b)
  float4 ca[3], cb[3], cal[3];
  float ca_z[3], cb_z[3], ca_dz[3], cb_dz[3];
  int vid[3] = {0, 0, 0};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    ca[q] = cb[q] = cal[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    ca_z[q] = cb_z[q] = ca_dz[q] = cb_dz[q] = 0.f;
  }
  if (has) {
    const bool persp = EXT && P.persp != 0;
    const bool textured = EXT && P.tex != nullptr;  // vertex attribute: a texture coordinate (Eq. fore)
    float4 r[kRecF4];
    load_record<MOVING>(recs_set + f, r, persp, false);
    const PixelSetup<MOVING> ps = pixel_setup<MOVING>(r, u, v);
    const EdgeVals e = edge_vals<MOVING>(r, ps, tau);
    const float invD = __fdividef(1.0f, e.D);
    const float wb[3] = {e.N0 * invD, e.N1 * invD, e.N2 * invD};  // screen-space barycentrics
    float w[3], iz[3], z[3] = {1.f, 1.f, 1.f};                     // attribute weights
    if (persp) depths_at<MOVING>(r, tau, z);
    attribute_weights(persp, wb, z, w, iz);
    float al[3][3], nv[3][3];
    float cr = 0.f, cg = 0.f, cbl = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      vid[q] = __ldg(P.faces + 3 * f + q);
      if (textured) {
        al[q][0] = __ldg(P.uv + 2 * vid[q]);
        al[q][1] = __ldg(P.uv + 2 * vid[q] + 1);
        al[q][2] = 0.f;
      } else {
        al[q][0] = __ldg(P.albedo + 3 * vid[q]);
        al[q][1] = __ldg(P.albedo + 3 * vid[q] + 1);
        al[q][2] = __ldg(P.albedo + 3 * vid[q] + 2);
      }
      float4 na = __ldg(P.slot_nrm + (size_t)slot_a * P.V + vid[q]);
      if (MOVING) {
        const float4 nb = __ldg(P.slot_nrm + (size_t)slot_b * P.V + vid[q]);
        na.x = fmaf(tau, nb.x - na.x, na.x);
        na.y = fmaf(tau, nb.y - na.y, na.y);
        na.z = fmaf(tau, nb.z - na.z, na.z);
      }
      nv[q][0] = na.x; nv[q][1] = na.y; nv[q][2] = na.z;
      cr = fmaf(w[q], al[q][0], cr);
      cg = fmaf(w[q], al[q][1], cg);
      cbl = fmaf(w[q], al[q][2], cbl);
      nx = fmaf(w[q], na.x, nx);
      ny = fmaf(w[q], na.y, ny);
      nz = fmaf(w[q], na.z, nz);
    }
    float du[3] = {0.f, 0.f, 0.f}, dv[3] = {0.f, 0.f, 0.f};
    TexTap tap;
    if (textured) {  // cr.. held the interpolated (u, v)
      float c[3];
      tap = tex_lookup(P.tex, P.tex_w, P.tex_h, cr, cg, c, du, dv);
      cr = c[0];
      cg = c[1];
      cbl = c[2];
    }
    const float len = sqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
    const float dot = len > 0.f ? __fdividef(fmaf(nx, P.lx, fmaf(ny, P.ly, nz * P.lz)), len) : 0.f;
    const float shade = fmaf(P.kd, fmaxf(dot, 0.f), P.ka);
    // I = c shade
    const float gcr = gr * shade, gcg = gg * shade, gcb = gb * shade;
    const float gshade = gr * cr + gg * cg + gb * cbl;
    float gw[3];
    if (textured) {
      // c = texture(sum_q w_q uv_q): dL/dw_q = uv_q . (dL/du, dL/dv); texel gradients by the taps
      const float gu = du[0] * gcr + du[1] * gcg + du[2] * gcb, gv = dv[0] * gcr + dv[1] * gcg + dv[2] * gcb;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        gw[q] = al[q][0] * gu + al[q][1] * gv;
        cal[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (P.g_tex) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          atomicAdd(P.g_tex + 3 * tap.idx[k], tap.wt[k] * gcr);
          atomicAdd(P.g_tex + 3 * tap.idx[k] + 1, tap.wt[k] * gcg);
          atomicAdd(P.g_tex + 3 * tap.idx[k] + 2, tap.wt[k] * gcb);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        gw[q] = al[q][0] * gcr + al[q][1] * gcg + al[q][2] * gcb;
        cal[q] = make_float4(w[q] * gcr, w[q] * gcg, w[q] * gcb, 0.f);
      }
    }
    if (len > 0.f && dot > 0.f) {
      const float il = __fdividef(1.f, len);
      const float hx = nx * il, hy = ny * il, hz = nz * il;
      const float gx = P.kd * gshade * P.lx, gy = P.kd * gshade * P.ly, gz = P.kd * gshade * P.lz;
      const float hg = hx * gx + hy * gy + hz * gz;
      const float gnx = (gx - hx * hg) * il, gny = (gy - hy * hg) * il, gnz = (gz - hz * hg) * il;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        gw[q] += nv[q][0] * gnx + nv[q][1] * gny + nv[q][2] * gnz;
        const float sa = MOVING ? (1.f - tau) * w[q] : w[q];
        ca[q].z = sa * gnx;
        ca[q].w = sa * gny;
        ca_z[q] = sa * gnz;
        if (MOVING) {
          cb[q].z = tau * w[q] * gnx;
          cb[q].w = tau * w[q] * gny;
          cb_z[q] = tau * w[q] * gnz;
        }
      }
    }
    // attribute weights -> screen barycentrics (and vertex depths, perspective-correct weights
    // a_i = (w_i / z_i) / S: dL/dw_k = (g_k - sum_i g_i a_i) / (z_k S), dL/dz_k = -(w_k / z_k) dL/dw_k)
    if (persp) {
      const float sa = w[0] * gw[0] + w[1] * gw[1] + w[2] * gw[2];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        gw[q] = (gw[q] - sa) * iz[q];
        const float gz = -(wb[q] / z[q]) * gw[q];
        ca_dz[q] = MOVING ? (1.f - tau) * gz : gz;
        if (MOVING) cb_dz[q] = tau * gz;
      }
    }
    // w = N / D -> vertex positions at tau
    const float sw = wb[0] * gw[0] + wb[1] * gw[1] + wb[2] * gw[2];
    float ax[3], ay[3], ex[3], ey[3];
    rel_vertices<MOVING>(r, ps, tau, ax, ay);
    edge_backward((gw[0] - sw) * invD, (gw[1] - sw) * invD, (gw[2] - sw) * invD, ax, ay, ex, ey);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const float sa = MOVING ? 1.f - tau : 1.f;
      ca[q].x = sa * ex[q];
      ca[q].y = sa * ey[q];
      if (MOVING) {
        cb[q].x = tau * ex[q];
        cb[q].y = tau * ey[q];
      }
    }
  }
  float4* ga_ = P.g_slot + (size_t)slot_a * P.V * 2;
  float4* gb_ = P.g_slot + (size_t)slot_b * P.V * 2;
  // Lanes with the same winner face add their contributions in shared memory first: the lowest
  // lane of each group sums the group's rows and issues the face's atomics, so a face costs one
  // set of vector atomics per warp and sample instead of one per covered lane.
  const uint32_t hmask = __ballot_sync(0xffffffffu, has);
  if (!hmask) return;
  const int lane = threadIdx.x & 31;
  const uint32_t grp = __match_any_sync(0xffffffffu, has ? f : -1 - lane);
  const bool lead = has && (__ffs(grp) - 1) == lane;
  constexpr int kDzA = MOVING ? 39 : 24, kDzB = 42;  // slot depth gradients (EXT only)
  constexpr int NV = EXT ? (MOVING ? 45 : 27) : (MOVING ? 39 : 24);
  static_assert(NV <= 4 * R, "a lane's contributions must fit its row");
  const bool shared_sum = __any_sync(0xffffffffu, has && __popc(grp) > 1);
  if (shared_sum) {
    float x[NV];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      x[5 * q] = ca[q].x; x[5 * q + 1] = ca[q].y; x[5 * q + 2] = ca[q].z; x[5 * q + 3] = ca[q].w;
      x[5 * q + 4] = ca_z[q];
      x[15 + 3 * q] = cal[q].x; x[16 + 3 * q] = cal[q].y; x[17 + 3 * q] = cal[q].z;
      if (MOVING) {
        x[24 + 5 * q] = cb[q].x; x[25 + 5 * q] = cb[q].y; x[26 + 5 * q] = cb[q].z; x[27 + 5 * q] = cb[q].w;
        x[28 + 5 * q] = cb_z[q];
        if (EXT) x[kDzB + q] = cb_dz[q];
      }
      if (EXT) x[kDzA + q] = ca_dz[q];
    }
    float* row = reinterpret_cast<float*>(ws_rows + lane);
    __syncwarp();
    if (has) {
#pragma unroll
      for (int k = 0; k < NV; ++k) row[k] = x[k];
    }
    __syncwarp();
    if (lead) {
      uint32_t others = grp & (grp - 1u);
      while (others) {
        const float* src = reinterpret_cast<const float*>(ws_rows + (__ffs(others) - 1));
        others &= others - 1u;
#pragma unroll
        for (int k = 0; k < NV; ++k) x[k] += src[k];
      }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        ca[q] = make_float4(x[5 * q], x[5 * q + 1], x[5 * q + 2], x[5 * q + 3]);
        ca_z[q] = x[5 * q + 4];
        cal[q] = make_float4(x[15 + 3 * q], x[16 + 3 * q], x[17 + 3 * q], 0.f);
        if (MOVING) {
          cb[q] = make_float4(x[24 + 5 * q], x[25 + 5 * q], x[26 + 5 * q], x[27 + 5 * q]);
          cb_z[q] = x[28 + 5 * q];
          if (EXT) cb_dz[q] = x[kDzB + q];
        }
        if (EXT) ca_dz[q] = x[kDzA + q];
      }
    }
    __syncwarp();  // the rows are read before they are reused
  }
  if (lead) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      atomicAdd(ga_ + (size_t)vid[q] * 2, ca[q]);
      atomicAdd(reinterpret_cast<float2*>(ga_ + (size_t)vid[q] * 2 + 1), make_float2(ca_z[q], ca_dz[q]));
      if (MOVING) {
        atomicAdd(gb_ + (size_t)vid[q] * 2, cb[q]);
        atomicAdd(reinterpret_cast<float2*>(gb_ + (size_t)vid[q] * 2 + 1), make_float2(cb_z[q], cb_dz[q]));
      }
      if (P.g_albedo && !(EXT && P.tex)) atomicAdd(P.g_albedo + vid[q], cal[q]);
    }
  }
}

// The adjoint raster reads the per-sample state of the forward raster (winner face of a covered
// sample; log soft product and vanishing-factor count of an uncovered one) and does not repeat
// the forward's coverage or soft-product passes.  Per block and sample group: the shading and
// barycentric adjoint of the covered samples' winners, then the soft-factor gradients (pass 3)
// of the uncovered samples that carry dL/dalpha.  Both parts run in one kernel: the covered part
// is latency-bound (dependent loads and atomics) and fills the issue slots of the soft part.
struct BwdBlock {
  int lane, n_tiles, px, py;
  BlockPix bp;
  bool in_img;
  float u, v;
  TileBox tb;
  int g_begin, g_end;
  float gr, gg, gb, ga;
};

template <int TW, int TH>
__device__ __forceinline__ BwdBlock bwd_block_setup(const RasterParams& P, int tile, int split, int wb) {
  BwdBlock B;
  B.lane = threadIdx.x & 31;
  B.n_tiles = P.tiles_x * P.tiles_y;
  const int tx = tile % P.tiles_x, ty = tile / P.tiles_x;
  PixelMap<TW, TH>::pixel(tx, ty, wb, B.px, B.py);
  B.bp = BlockPix{B.px - (B.lane & 7), B.py - (B.lane >> 3), P.W, P.H};
  B.in_img = B.px < P.W && B.py < P.H;
  B.bp.uv(B.lane, B.u, B.v);
  B.tb = PixelMap<TW, TH>::warp_box(tx, ty, wb, P.W, P.H);
  B.g_begin = (int)((long long)P.G * split / P.n_split);
  B.g_end = (int)((long long)P.G * (split + 1) / P.n_split);
  float4 G4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (B.in_img) G4 = __ldg(P.dl_dimage + (size_t)B.py * P.W + B.px);
  B.gr = G4.x * P.inv_T;
  B.gg = G4.y * P.inv_T;
  B.gb = G4.z * P.inv_T;
  B.ga = G4.w * P.inv_T;
  return B;
}

// The state-free adjoint's per-group state (the forward kept none): the group's winners and the
// soft log products of its uncovered samples that carry dL/dalpha, recomputed by the forward's own
// passes.  Out of line, so that the stored-state path carries none of its registers.  Writes the
// winners to ws.wface and the soft state to ws.logp / ws.nzero; returns this pixel's uncovered
// samples that carry dL/dalpha.
template <int SPT, bool MOVING, bool EXT>
__device__ __noinline__ uint32_t recompute_group_state(const RasterParams& P, const TriRec* recs_set,
                                                       const GroupRegs& gq, int g, int tile, const BwdBlock& B,
                                                       bool alpha, int sb, int se, BwdScratch<SPT>& ws) {
  const int lane = threadIdx.x & 31;
  const int n = gq.n;
  int cb, ce;
  P.core.range((size_t)g * B.n_tiles + tile, cb, ce);
  float bkey[SPT];
  int win[SPT];
  core_raster<SPT, MOVING>(recs_set, P.core.faces, cb, ce, gq.tau, n, B.tb, B.u, B.v, B.in_img, ws, bkey, win);
  uint32_t my_s = 0u;
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    if (!(i < n && B.in_img)) win[i] = -1;
    else if (win[i] < 0 && alpha) my_s |= 1u << i;
    ws.wface[i][lane] = win[i];
  }
  float lp[SPT];
  int nz[SPT];
  uint32_t t0 = 0, t1 = 0;
  soft_raster<SPT, MOVING>(recs_set, P.soft.faces, sb, se, gq.tau, gq.xbits, n, B.tb, B.u, B.v, my_s,
                           P.r + kCoreMargin, P.r2, P.inv_delta, EXT ? P.prob : 0, ws, lp, nz, t0, t1);
#pragma unroll
  for (int i = 0; i < SPT; ++i) {
    ws.logp[i][lane] = lp[i];
    ws.nzero[i][lane] = nz[i];
  }
  __syncwarp();
  return my_s;
}

// the adjoint of one 8 x 4 block over its split of the sample groups (EXT: see covered_adjoint)
template <int TW, int TH, int SPT, bool MOVING, bool EXT>
__device__ __forceinline__ void raster_bwd_block(const RasterParams& P, int tile, int split, int wb,
                                                 BwdScratch<SPT>& ws) {
  const BwdBlock B = bwd_block_setup<TW, TH>(P, tile, split, wb);
  const bool rgb = B.in_img && (B.gr != 0.f || B.gg != 0.f || B.gb != 0.f);  // colour gradient
  const bool alpha = B.in_img && B.ga != 0.f;                                // alpha gradient
  const bool any_rgb = __any_sync(kFullMask, rgb);
  if (!any_rgb && !__any_sync(kFullMask, alpha)) return;
  const int lane = B.lane;
  ws.pu[lane] = B.u;
  ws.pv[lane] = B.v;
  ws.ga[lane] = B.ga;
  const size_t plane = (size_t)P.H * P.W, pix = (size_t)B.py * P.W + B.px;

  for (int g = B.g_begin; g < B.g_end; ++g) {
    const Group* grp = P.groups + g;
    GroupRegs gq;
    gq.load(grp);
    const int n = gq.n;
    const TriRec* recs_set = P.recs + (size_t)gq.rec_set * P.F;
    int win[SPT];
    uint32_t my_s = 0u;
    int sb, se;
    P.soft.range((size_t)g * B.n_tiles + tile, sb, se);
    if (P.s_stat) {
      // the forward's state of the group's samples at this pixel
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        win[i] = -1;
        if (i < n && B.in_img) {
          const size_t o = (size_t)(gq.k0 + i) * plane + pix;
          // both words at once (the value's meaning follows from the status)
          const uint8_t st = __ldg(P.s_stat + o);
          const float sv = __ldg(P.s_val + o);
          if (st == kStatCovered) {
            win[i] = __float_as_int(sv);
          } else if (alpha) {
            my_s |= 1u << i;
            ws.nzero[i][lane] = st;
            ws.logp[i][lane] = sv;
          }
        }
      }
    } else {
      // state-free adjoint: recompute the group's winners and the soft products of its uncovered
      // samples that carry dL/dalpha, exactly as the forward raster does (same passes, same order)
      my_s = recompute_group_state<SPT, MOVING, EXT>(P, recs_set, gq, g, tile, B, alpha, sb, se, ws);
#pragma unroll
      for (int i = 0; i < SPT; ++i) win[i] = ws.wface[i][lane];
      __syncwarp();
    }

    // ---- covered samples: shading adjoint and barycentric adjoint of the winner
    if (any_rgb) {
#pragma unroll 1
      for (int i = 0; i < n; ++i) {
        int f = -1;
#pragma unroll
        for (int q = 0; q < SPT; ++q)
          if (q == i) f = win[q];
        const bool has = rgb && f >= 0;
        const float tau = MOVING ? __ldg(gq.tau + i) : 0.f;
        covered_adjoint<MOVING, EXT>(P, recs_set, gq.slot_a, gq.slot_b, has, has ? f : 0, tau, B.u, B.v, B.gr,
                                     B.gg, B.gb, ws.coef);
      }
    }

    // ---- uncovered samples: soft-factor gradients (pass 3)
    const uint32_t any_s = __reduce_or_sync(kFullMask, my_s);
    if (se > sb && any_s) {
      uint32_t allowed[SPT];
#pragma unroll
      for (int i = 0; i < SPT; ++i) allowed[i] = __ballot_sync(kFullMask, (my_s >> i) & 1u);
      ws.pixs[lane] = my_s;
      __syncwarp();
      const float m = P.r + kCoreMargin;
      BwdSoftGradPairs<SPT, MOVING> p3;
      p3.recs_set = recs_set;
      p3.grp = grp;
      p3.bp = B.bp;
      p3.ws = &ws;
      p3.xbits = gq.xbits;
      p3.m = m;
      p3.r2 = P.r2;
      p3.inv_delta = P.inv_delta;
      p3.prob = EXT ? P.prob : 0;
      p3.faces = P.faces;
      p3.gslot_a = P.g_slot + (size_t)gq.slot_a * P.V * 2;
      p3.gslot_b = P.g_slot + (size_t)gq.slot_b * P.V * 2;
      for_pairs<SPT, MOVING, true, !MOVING, kPairsPerLane>(recs_set, P.soft.faces, sb, se, grp, n, B.tb, B.bp, m, allowed,
                                                          any_s, ws, p3);
    }
    __syncwarp();  // the scratch is rewritten by the next group
  }
}

// Persistent adjoint raster: KIND 0 = plain solver only, 1 = fast solver only, 2 = mixed batch;
// EXT: with the variants.
template <int TW, int TH, int SPT, int KIND, bool EXT>
__global__ void __launch_bounds__(kPersistentThreads, KIND == 0 ? 3 : 2) raster_bwd_persistent(WorkQueue Q) {
  __shared__ CtaQueue cq;
  __shared__ RasterParams sp[kPersistentThreads / 32];
  __shared__ BwdScratch<SPT> ws[kPersistentThreads / 32];
  cq.init();
  const int warp = threadIdx.x >> 5;
  RasterParams& P = sp[warp];
  int cur = -1, tile = 0, split = 0, wb = 0;
  while (warp_next<TW, TH>(Q, cq, P, cur, tile, split, wb)) {
    if (tile >= P.tiles_x * P.tiles_y) continue;
    if constexpr (KIND == 0) {
      raster_bwd_block<TW, TH, 1, false, EXT>(P, tile, split, wb, ws[warp]);
    } else {
      if (KIND == 2 && !P.moving)
        raster_bwd_block<TW, TH, 1, false, EXT>(P, tile, split, wb, *reinterpret_cast<BwdScratch<1>*>(ws + warp));
      else
        raster_bwd_block<TW, TH, SPT, true, EXT>(P, tile, split, wb, ws[warp]);
    }
  }
}

// ---------------------------------------------------------------- slot gradients -> vertices
// one warp per vertex, lanes over slots (no atomics); writes dL/dv and dL/dm (m = normal sum)
__global__ void slot_chain_kernel(const float* __restrict__ verts, const float* __restrict__ nacc, int V,
                                  const SlotXform* __restrict__ xf, int n_slots, float th,
                                  const float4* __restrict__ g_slot, const float4* __restrict__ g_alb4,
                                  float* __restrict__ g_verts, float* __restrict__ g_m,
                                  float* __restrict__ g_albedo) {
  // one warp per vertex: lanes take the slots, then a warp sum (V is small, slots are many)
  const int v = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (v >= V) return;  // warp-uniform
  if (g_albedo && lane == 0) {
    const float4 a = g_alb4[v];
    g_albedo[3 * v] = a.x;
    g_albedo[3 * v + 1] = a.y;
    g_albedo[3 * v + 2] = a.z;
  }
  const float px = verts[3 * v], py = verts[3 * v + 1], pz = verts[3 * v + 2];
  float gvx = 0.f, gvy = 0.f, gvz = 0.f, gnx = 0.f, gny = 0.f, gnz = 0.f;
  for (int s = lane; s < n_slots; s += 32) {
    const float4 ga = g_slot[((size_t)s * V + v) * 2];
    const float4 gz4 = g_slot[((size_t)s * V + v) * 2 + 1];
    const float g0 = ga.x, g1 = ga.y, g2 = ga.z, g3 = ga.w, g4 = gz4.x, g5 = gz4.y;
    if (g0 == 0.f && g1 == 0.f && g2 == 0.f && g3 == 0.f && g4 == 0.f && g5 == 0.f) continue;
    const float* A = xf[s].A;
    const float* R = xf[s].R;
    const float xc = fmaf(A[0], px, fmaf(A[1], py, fmaf(A[2], pz, A[3])));
    const float yc = fmaf(A[4], px, fmaf(A[5], py, fmaf(A[6], pz, A[7])));
    const float zc = fmaf(A[8], px, fmaf(A[9], py, fmaf(A[10], pz, A[11])));
    const float den = zc * th;
    // x = xc / (zc th), y = yc / (zc th)
    const float dxc = g0 / den, dyc = g1 / den;
    const float dzc = g5 - (g0 * xc + g1 * yc) / (den * zc);  // camera z: direct (depth) + projection
    gvx += A[0] * dxc + A[4] * dyc + A[8] * dzc;
    gvy += A[1] * dxc + A[5] * dyc + A[9] * dzc;
    gvz += A[2] * dxc + A[6] * dyc + A[10] * dzc;
    gnx += R[0] * g2 + R[3] * g3 + R[6] * g4;
    gny += R[1] * g2 + R[4] * g3 + R[7] * g4;
    gnz += R[2] * g2 + R[5] * g3 + R[8] * g4;
  }
  gvx = warp_sum(gvx);
  gvy = warp_sum(gvy);
  gvz = warp_sum(gvz);
  gnx = warp_sum(gnx);
  gny = warp_sum(gny);
  gnz = warp_sum(gnz);
  if (lane != 0) return;
  g_verts[3 * v] = gvx;
  g_verts[3 * v + 1] = gvy;
  g_verts[3 * v + 2] = gvz;
  // n = m / |m|: dL/dm = (g - n (n.g)) / |m|
  const float mx = nacc[3 * v], my = nacc[3 * v + 1], mz = nacc[3 * v + 2];
  const float len = sqrtf(fmaf(mx, mx, fmaf(my, my, mz * mz)));
  float ox = 0.f, oy = 0.f, oz = 0.f;
  if (len > 0.f) {
    const float il = 1.f / len;
    const float hx = mx * il, hy = my * il, hz = mz * il;
    const float hg = hx * gnx + hy * gny + hz * gnz;
    ox = (gnx - hx * hg) * il;
    oy = (gny - hy * hg) * il;
    oz = (gnz - hz * hg) * il;
  }
  g_m[3 * v] = ox;
  g_m[3 * v + 1] = oy;
  g_m[3 * v + 2] = oz;
}

// m_v += (b - a) x (c - a) for every face f = (a, b, c):  dL/db = (c - a) x G, dL/dc = G x (b - a)
__global__ void normals_bwd_kernel(const float* __restrict__ verts, const int32_t* __restrict__ faces, int F, int V,
                                   const float* __restrict__ g_m, float* __restrict__ g_verts) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
  if (a < 0 || b < 0 || c < 0 || a >= V || b >= V || c >= V) return;
  const float Gx = g_m[3 * a] + g_m[3 * b] + g_m[3 * c];
  const float Gy = g_m[3 * a + 1] + g_m[3 * b + 1] + g_m[3 * c + 1];
  const float Gz = g_m[3 * a + 2] + g_m[3 * b + 2] + g_m[3 * c + 2];
  if (Gx == 0.f && Gy == 0.f && Gz == 0.f) return;
  const float ax = verts[3 * a], ay = verts[3 * a + 1], az = verts[3 * a + 2];
  const float ux = verts[3 * b] - ax, uy = verts[3 * b + 1] - ay, uz = verts[3 * b + 2] - az;
  const float wx = verts[3 * c] - ax, wy = verts[3 * c + 1] - ay, wz = verts[3 * c + 2] - az;
  const float bx = wy * Gz - wz * Gy, by = wz * Gx - wx * Gz, bz = wx * Gy - wy * Gx;
  const float cx = Gy * uz - Gz * uy, cy = Gz * ux - Gx * uz, cz = Gx * uy - Gy * ux;
  atomicAdd(g_verts + 3 * b, bx);
  atomicAdd(g_verts + 3 * b + 1, by);
  atomicAdd(g_verts + 3 * b + 2, bz);
  atomicAdd(g_verts + 3 * c, cx);
  atomicAdd(g_verts + 3 * c + 1, cy);
  atomicAdd(g_verts + 3 * c + 2, cz);
  atomicAdd(g_verts + 3 * a, -(bx + cx));
  atomicAdd(g_verts + 3 * a + 1, -(by + cy));
  atomicAdd(g_verts + 3 * a + 2, -(bz + cz));
}

template <int TW, int TH, int KIND, bool EXT>
static void launch_bwd_spt(const WorkQueue& Q, int spt, int grid, cudaStream_t st) {
  if (spt <= 2)
    raster_bwd_persistent<TW, TH, 2, KIND, EXT><<<grid, kPersistentThreads, 0, st>>>(Q);
  else
    raster_bwd_persistent<TW, TH, 4, KIND, EXT><<<grid, kPersistentThreads, 0, st>>>(Q);
}

template <int TW, int TH, bool EXT>
static void launch_bwd_tile(const WorkQueue& Q, int spt, int kind, int grid, cudaStream_t st) {
  if (kind == 0)
    raster_bwd_persistent<TW, TH, 1, 0, EXT><<<grid, kPersistentThreads, 0, st>>>(Q);
  else if (kind == 1)
    launch_bwd_spt<TW, TH, 1, EXT>(Q, spt, grid, st);
  else
    launch_bwd_spt<TW, TH, 2, EXT>(Q, spt, grid, st);
}

void launch_raster_bwd(const WorkQueue& Q, int tile, int spt, int kind, int grid, cudaStream_t st) {
  if (Q.n_work <= 0) return;
  const int k = kind & kKindMask;
  if (kind & kKindExt) {
    if (tile == 8) launch_bwd_tile<8, 8, true>(Q, spt, k, grid, st);
    else launch_bwd_tile<16, 16, true>(Q, spt, k, grid, st);
  } else {
    if (tile == 8) launch_bwd_tile<8, 8, false>(Q, spt, k, grid, st);
    else launch_bwd_tile<16, 16, false>(Q, spt, k, grid, st);
  }
}

template <typename K>
static int occupancy_of(K kernel) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kPersistentThreads, 0) != cudaSuccess) n = 1;
  return n < 1 ? 1 : n;
}

template <int TW, int TH, bool EXT>
static int occ_bwd(int spt, int kind) {
  if (kind == 0) return occupancy_of(raster_bwd_persistent<TW, TH, 1, 0, EXT>);
  if (kind == 1)
    return spt <= 2 ? occupancy_of(raster_bwd_persistent<TW, TH, 2, 1, EXT>)
                    : occupancy_of(raster_bwd_persistent<TW, TH, 4, 1, EXT>);
  return spt <= 2 ? occupancy_of(raster_bwd_persistent<TW, TH, 2, 2, EXT>)
                  : occupancy_of(raster_bwd_persistent<TW, TH, 4, 2, EXT>);
}

int persistent_grid_bwd(int num_sms, int tile, int spt, int kind) {
  const int k = kind & kKindMask;
  int occ;
  if (kind & kKindExt) occ = tile == 8 ? occ_bwd<8, 8, true>(spt, k) : occ_bwd<16, 16, true>(spt, k);
  else occ = tile == 8 ? occ_bwd<8, 8, false>(spt, k) : occ_bwd<16, 16, false>(spt, k);
  return num_sms * occ;
}

void launch_slot_chain(const float* verts, const float* nacc, int V, const SlotXform* xf, int n_slots, float th,
                       const float4* g_slot, const float4* g_alb4, float* g_verts, float* g_m, float* g_albedo,
                       cudaStream_t st) {
  if (V > 0)
    slot_chain_kernel<<<(unsigned)(((size_t)V * 32 + 255) / 256), 256, 0, st>>>(verts, nacc, V, xf, n_slots, th, g_slot, g_alb4, g_verts, g_m,
                                                       g_albedo);
}

void launch_normals_bwd(const float* verts, const int32_t* faces, int F, int V, const float* g_m, float* g_verts,
                        cudaStream_t st) {
  if (F > 0) normals_bwd_kernel<<<(F + 255) / 256, 256, 0, st>>>(verts, faces, F, V, g_m, g_verts);
}

}  // namespace mbr
