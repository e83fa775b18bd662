// mbr_api.cu -- host side of the C ABI declared in include/mbr.h.
//
// Per call: validate arguments -> time map (Secs. 3.2-3.3, exact integer arithmetic) -> per-slot
// motion + camera matrices (double precision, one 3x4 per slot time) -> kernels on the caller's
// stream: normals, transform, triangle setup, tile binning (count, scan, one stream sync to
// size the face lists, fill), raster, finalize.  Backward reruns the same front half and the
// adjoint raster, then chains slot gradients to vertices.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/mbr.h"
#include "mbr_internal.h"
#include "mbr_raster.cuh"

using namespace mbr;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

// one CSR binning of (group, tile) -> face lists
struct BinSet {
  DevBuf counts, offsets, cursor, list, scan_tmp;
};

}  // namespace

struct mbr_ctx {
  int device = 0;
  int num_sms = 1;
  std::string err;
  // tuning
  int tile = 16, spt = 8, splits = 0;
  // scratch
  DevBuf nacc, pos, nrm, recs, tables, partial, gslot, galb, gm, cnt64, status;
  BinSet core, soft;  // undilated bins (coverage) and r_soft-dilated bins (soft coverage)
  void* host_stage = nullptr;
  size_t host_stage_cap = 0;
  int32_t* host_total = nullptr;
  // measurement: one event pair per raster kind (0 forward, 1 adjoint), harvested lazily
  bool profiling = false;
  cudaEvent_t ev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool pending[2] = {false, false};
  mbr_stats stats{};
};

namespace {

constexpr double kPi = 3.14159265358979323846;

int fail(mbr_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CUDA_TRY(ctx, expr)                                                                     \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? MBR_ERR_OOM : MBR_ERR_CUDA, "%s: %s", \
                  #expr, cudaGetErrorString(e_));                                               \
  } while (0)

// grow-only device buffer; old contents are discarded
int ensure(mbr_ctx* c, DevBuf& b, size_t bytes, cudaStream_t st) {
  if (bytes <= b.cap) return MBR_OK;
  if (b.p) {
    CUDA_TRY(c, cudaStreamSynchronize(st));
    CUDA_TRY(c, cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = std::max<size_t>(bytes + bytes / 4, 256);
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    b.p = nullptr;
    return fail(c, MBR_ERR_OOM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
  }
  b.cap = want;
  return MBR_OK;
}

int ensure_host(mbr_ctx* c, size_t bytes) {
  if (bytes <= c->host_stage_cap) return MBR_OK;
  if (c->host_stage) cudaFreeHost(c->host_stage);
  c->host_stage = nullptr;
  c->host_stage_cap = 0;
  size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
  if (cudaMallocHost(&c->host_stage, want) != cudaSuccess) {
    c->host_stage = nullptr;
    return fail(c, MBR_ERR_OOM, "cudaMallocHost(%zu) failed", want);
  }
  c->host_stage_cap = want;
  return MBR_OK;
}

// ------------------------------------------------------------------ time map (Secs. 3.2-3.3)
int num_segments(const mbr_motion* m) {
  if (m->segments > 0) return m->segments;
  if (m->kind == MBR_TRANSLATE) return 1;
  const double x = 12.0 * std::fabs((double)m->omega) / (2.0 * kPi);
  const int n = (int)std::ceil(x - 1e-4);  // tolerance: omega = 2 pi rounded to float is 12 segments
  return n < 1 ? 1 : n;
}

// t_k = num / den exactly
void time_fraction(int rule, int T, int k, long long& num, long long& den) {
  if (rule == MBR_TIME_MIDPOINT) {
    num = 2LL * k + 1;
    den = 2LL * T;
  } else if (T == 1) {
    num = 1;
    den = 2;
  } else {
    num = k;
    den = (long long)T - 1;
  }
}

// Rodrigues rotation matrix of angle th about unit axis k (right-handed)
void rotation(const double k[3], double th, double R[9]) {
  const double c = std::cos(th), s = std::sin(th), C = 1.0 - c;
  R[0] = c + k[0] * k[0] * C;        R[1] = k[0] * k[1] * C - k[2] * s; R[2] = k[0] * k[2] * C + k[1] * s;
  R[3] = k[1] * k[0] * C + k[2] * s; R[4] = c + k[1] * k[1] * C;        R[5] = k[1] * k[2] * C - k[0] * s;
  R[6] = k[2] * k[0] * C - k[1] * s; R[7] = k[2] * k[1] * C + k[0] * s; R[8] = c + k[2] * k[2] * C;
}

SlotXform slot_xform(const mbr_motion* m, const mbr_camera* cam, double t) {
  double Rm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, b[3] = {0, 0, 0};
  if (m->kind == MBR_TRANSLATE) {
    for (int i = 0; i < 3; ++i) b[i] = (double)m->offset[i] + t * (double)m->dir[i];
  } else {
    double k[3] = {m->axis[0], m->axis[1], m->axis[2]};
    const double n = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    for (double& x : k) x /= n;
    rotation(k, (double)m->omega * t, Rm);
  }
  SlotXform x;
  std::memset(&x, 0, sizeof(x));
  for (int r = 0; r < 3; ++r) {
    const float* V = cam->view + 4 * r;
    for (int c = 0; c < 3; ++c)
      x.A[4 * r + c] = (float)(V[0] * Rm[c] + V[1] * Rm[3 + c] + V[2] * Rm[6 + c]);
    x.A[4 * r + 3] = (float)(V[0] * b[0] + V[1] * b[1] + V[2] * b[2] + V[3]);
  }
  for (int i = 0; i < 9; ++i) x.R[i] = (float)Rm[i];
  x.t = (float)t;
  return x;
}

int validate(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam, int T, int H,
             int W, int solver) {
  if (!c) return MBR_ERR_ARG;
  if (!mesh || !motion || !cam) return fail(c, MBR_ERR_ARG, "null mesh/motion/camera");
  if (mesh->V < 1 || mesh->F < 0) return fail(c, MBR_ERR_ARG, "bad mesh sizes V=%d F=%d", mesh->V, mesh->F);
  if (!mesh->verts || !mesh->albedo || (mesh->F > 0 && !mesh->faces))
    return fail(c, MBR_ERR_ARG, "null mesh buffer");
  if (T < 1 || T > (1 << 20)) return fail(c, MBR_ERR_ARG, "bad T=%d", T);
  if (H < 1 || W < 1 || H > 16384 || W > 16384) return fail(c, MBR_ERR_ARG, "bad image size %dx%d", H, W);
  if (solver != MBR_PLAIN && solver != MBR_FAST) return fail(c, MBR_ERR_ARG, "bad solver %d", solver);
  if (motion->kind != MBR_TRANSLATE && motion->kind != MBR_ROTATE)
    return fail(c, MBR_ERR_ARG, "bad motion kind %d", motion->kind);
  if (motion->segments < 0 || motion->segments > 1000000) return fail(c, MBR_ERR_ARG, "bad segments");
  if (motion->kind == MBR_ROTATE &&
      !(motion->axis[0] * motion->axis[0] + motion->axis[1] * motion->axis[1] + motion->axis[2] * motion->axis[2] > 0.f))
    return fail(c, MBR_ERR_ARG, "zero rotation axis");
  if (!(cam->tan_half_fov > 0.f) || !(cam->delta > 0.f)) return fail(c, MBR_ERR_ARG, "bad camera fov/delta");
  if (cam->time_rule != MBR_TIME_PAPER && cam->time_rule != MBR_TIME_MIDPOINT)
    return fail(c, MBR_ERR_ARG, "bad time rule");
  const long long T_ = T;
  if (solver == MBR_FAST && (long long)num_segments(motion) > 4 * T_ + 64)
    return fail(c, MBR_ERR_ARG, "segments %d far exceed T=%d", num_segments(motion), T);
  return MBR_OK;
}

// kernels launched by the front half: normals, transform, setup (+ bins: count, 3 scan, fill)
constexpr int kFrontLaunches = 3, kBinLaunches = 5;

// add the duration of a recorded event pair to the sums (waits for its end event)
int harvest(mbr_ctx* c, int kind) {
  if (!c->pending[kind]) return MBR_OK;
  CUDA_TRY(c, cudaEventSynchronize(c->ev[kind][1]));
  float ms = 0.f;
  CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev[kind][0], c->ev[kind][1]));
  if (kind == 0) {
    c->stats.raster_fwd_ms += ms;
    c->stats.raster_fwd_count += 1;
  } else {
    c->stats.raster_bwd_ms += ms;
    c->stats.raster_bwd_count += 1;
  }
  c->pending[kind] = false;
  return MBR_OK;
}

int time_begin(mbr_ctx* c, int kind, cudaStream_t st) {
  if (!c->profiling) return MBR_OK;
  int rc = harvest(c, kind);
  if (rc) return rc;
  if (!c->ev[kind][0]) {
    CUDA_TRY(c, cudaEventCreate(&c->ev[kind][0]));
    CUDA_TRY(c, cudaEventCreate(&c->ev[kind][1]));
  }
  CUDA_TRY(c, cudaEventRecord(c->ev[kind][0], st));
  return MBR_OK;
}

int time_end(mbr_ctx* c, int kind, cudaStream_t st) {
  if (!c->profiling) return MBR_OK;
  CUDA_TRY(c, cudaEventRecord(c->ev[kind][1], st));
  c->pending[kind] = true;
  return MBR_OK;
}

// Everything the raster kernels need; built by prepare().
struct Prepared {
  int S = 1, n_slots = 0, n_sets = 0, G = 0;
  int tiles_x = 0, tiles_y = 0, n_tiles = 0, n_split = 1;
  bool moving = false;
  int spt = 1;
  SlotXform* d_xf = nullptr;
  Group* d_groups = nullptr;
  float r = 0.f;
};

int build_tables(mbr_ctx* c, const mbr_motion* motion, const mbr_camera* cam, int T, int solver,
                 std::vector<SlotXform>& xf, std::vector<int2>& sets, std::vector<Group>& groups, Prepared& pp) {
  const int S = solver == MBR_FAST ? num_segments(motion) : 1;
  pp.S = S;
  pp.moving = solver == MBR_FAST;
  pp.spt = pp.moving ? std::max(1, std::min(kMaxSpt, c->spt)) : 1;
  xf.clear();
  sets.clear();
  groups.clear();
  if (solver == MBR_FAST) {
    for (int s = 0; s <= S; ++s) xf.push_back(slot_xform(motion, cam, (double)s / S));
    for (int s = 0; s < S; ++s) sets.push_back(make_int2(s, s + 1));
    // samples of segment s are a contiguous range of k; chunk them by spt
    int k = 0;
    while (k < T) {
      long long num, den;
      time_fraction(cam->time_rule, T, k, num, den);
      long long sg = (num * S) / den;
      if (sg > S - 1) sg = S - 1;
      Group g;
      std::memset(&g, 0, sizeof(g));
      g.rec_set = (int)sg;
      g.slot_a = (int)sg;
      g.slot_b = (int)sg + 1;
      g.k0 = k;
      g.tau_lo = INFINITY;
      g.tau_hi = -INFINITY;
      while (k < T && g.n < pp.spt) {
        time_fraction(cam->time_rule, T, k, num, den);
        long long s2 = (num * S) / den;
        if (s2 > S - 1) s2 = S - 1;
        if (s2 != sg) break;
        const long long rem = num * S - sg * den;  // tau = rem / den
        const float tau = (float)((double)rem / (double)den);
        g.tau[g.n] = tau;
        if (2 * rem > den) g.xbits |= 1u << g.n;  // keyframe X = 1 iff tau > 1/2
        g.tau_lo = std::min(g.tau_lo, tau);
        g.tau_hi = std::max(g.tau_hi, tau);
        ++g.n;
        ++k;
      }
      groups.push_back(g);
    }
  } else {
    for (int k = 0; k < T; ++k) {
      long long num, den;
      time_fraction(cam->time_rule, T, k, num, den);
      xf.push_back(slot_xform(motion, cam, (double)num / (double)den));
      sets.push_back(make_int2(k, k));
      Group g;
      std::memset(&g, 0, sizeof(g));
      g.rec_set = k;
      g.slot_a = g.slot_b = k;
      g.n = 1;
      g.k0 = k;
      g.tau[0] = 0.f;
      g.tau_lo = g.tau_hi = 0.f;
      groups.push_back(g);
    }
  }
  pp.n_slots = (int)xf.size();
  pp.n_sets = (int)sets.size();
  pp.G = (int)groups.size();
  return MBR_OK;
}

// front half shared by forward, backward and the candidate count.  do_bins = false stops after
// the triangle setup.
int prepare(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam, int T, int H,
            int W, int solver, cudaStream_t st, bool do_bins, Prepared& pp) {
  std::vector<SlotXform> xf;
  std::vector<int2> sets;
  std::vector<Group> groups;
  int rc = build_tables(c, motion, cam, T, solver, xf, sets, groups, pp);
  if (rc) return rc;
  const int V = mesh->V, F = mesh->F;
  // tables -> one pinned staging buffer -> one async copy
  const size_t xf_b = xf.size() * sizeof(SlotXform), sets_b = sets.size() * sizeof(int2),
               g_b = groups.size() * sizeof(Group);
  const size_t off_sets = (xf_b + 255) & ~size_t(255), off_g = (off_sets + sets_b + 255) & ~size_t(255);
  const size_t tab_b = off_g + g_b;
  if ((rc = ensure_host(c, tab_b))) return rc;
  if ((rc = ensure(c, c->tables, tab_b, st))) return rc;
  char* h = (char*)c->host_stage;
  std::memcpy(h, xf.data(), xf_b);
  std::memcpy(h + off_sets, sets.data(), sets_b);
  std::memcpy(h + off_g, groups.data(), g_b);
  CUDA_TRY(c, cudaMemcpyAsync(c->tables.p, h, tab_b, cudaMemcpyHostToDevice, st));
  char* dt = (char*)c->tables.p;
  pp.d_xf = (SlotXform*)dt;
  const int2* d_sets = (const int2*)(dt + off_sets);
  pp.d_groups = (Group*)(dt + off_g);

  // a0 normals, a1 transform, a4 setup
  if ((rc = ensure(c, c->nacc, sizeof(float) * 3 * V, st))) return rc;
  if ((rc = ensure(c, c->pos, sizeof(float4) * (size_t)pp.n_slots * V, st))) return rc;
  if ((rc = ensure(c, c->nrm, sizeof(float4) * (size_t)pp.n_slots * V, st))) return rc;
  if ((rc = ensure(c, c->recs, sizeof(TriRec) * (size_t)pp.n_sets * std::max(F, 1), st))) return rc;
  if ((rc = ensure(c, c->status, sizeof(int32_t), st))) return rc;
  int* d_status = (int*)c->status.p;
  CUDA_TRY(c, cudaMemsetAsync(d_status, 0, sizeof(int32_t), st));
  CUDA_TRY(c, cudaMemsetAsync(c->nacc.p, 0, sizeof(float) * 3 * V, st));
  launch_face_normals(mesh->verts, mesh->faces, F, V, (float*)c->nacc.p, d_status, st);
  launch_xform(mesh->verts, (const float*)c->nacc.p, V, pp.d_xf, pp.n_slots, cam->tan_half_fov,
               (float4*)c->pos.p, (float4*)c->nrm.p, st);
  launch_setup((const float4*)c->pos.p, mesh->faces, F, V, d_sets, pp.n_sets, cam->znear, (TriRec*)c->recs.p, st);
  CUDA_TRY(c, cudaGetLastError());
  pp.r = (float)std::sqrt((double)cam->delta * (double)kSoftCutoff);
  c->stats.launches += (F > 0 ? 1 : 0) + 1 + (F > 0 ? 1 : 0);
  c->stats.groups = pp.G;
  if (!do_bins) {
    CUDA_TRY(c, cudaMemcpyAsync(c->host_total + 1, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    if (c->host_total[1] & kStatusBadFace) return fail(c, MBR_ERR_ARG, "face index outside [0, V)");
    return MBR_OK;
  }

  // a3 binning: core and soft bins: count -> scan (both) -> one sync for the totals -> fill
  const int tw = c->tile, th = c->tile;
  pp.tiles_x = (W + tw - 1) / tw;
  pp.tiles_y = (H + th - 1) / th;
  pp.n_tiles = pp.tiles_x * pp.tiles_y;
  const long long nb = (long long)pp.G * pp.n_tiles;
  if (nb > (1LL << 30)) return fail(c, MBR_ERR_ARG, "too many (group, tile) bins: %lld", nb);
  BinSet* sets2[2] = {&c->core, &c->soft};
  const float margins[2] = {kCoreMargin, pp.r + kCoreMargin};
  for (int q = 0; q < 2; ++q) {
    BinSet& bs = *sets2[q];
    if ((rc = ensure(c, bs.counts, sizeof(int32_t) * (size_t)nb, st))) return rc;
    if ((rc = ensure(c, bs.offsets, sizeof(int32_t) * (size_t)(nb + 1), st))) return rc;
    if ((rc = ensure(c, bs.scan_tmp, sizeof(int32_t) * scan_temp_ints((int)nb), st))) return rc;
    CUDA_TRY(c, cudaMemsetAsync(bs.counts.p, 0, sizeof(int32_t) * (size_t)nb, st));
    launch_bin(false, (const TriRec*)c->recs.p, F, pp.d_groups, pp.G, W, H, tw, th, pp.tiles_x, pp.n_tiles,
               margins[q], (int32_t*)bs.counts.p, nullptr, nullptr, d_status, st);
    launch_scan((const int32_t*)bs.counts.p, (int)nb, (int32_t*)bs.offsets.p, (int32_t*)bs.scan_tmp.p, st);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(c->host_total + 2 * q, (int32_t*)bs.offsets.p + nb, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->host_total + 1, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (c->host_total[1] & kStatusBadFace) return fail(c, MBR_ERR_ARG, "face index outside [0, V)");
  long long totals[2] = {c->host_total[0], c->host_total[2]};
  for (int q = 0; q < 2; ++q) {
    BinSet& bs = *sets2[q];
    if (totals[q] < 0) return fail(c, MBR_ERR_DEVICE, "bin total overflow");
    if ((rc = ensure(c, bs.list, sizeof(int32_t) * (size_t)std::max<long long>(totals[q], 1), st))) return rc;
    if ((rc = ensure(c, bs.cursor, sizeof(int32_t) * (size_t)nb, st))) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(bs.cursor.p, bs.offsets.p, sizeof(int32_t) * (size_t)nb, cudaMemcpyDeviceToDevice,
                                st));
    launch_bin(true, (const TriRec*)c->recs.p, F, pp.d_groups, pp.G, W, H, tw, th, pp.tiles_x, pp.n_tiles,
               margins[q], (int32_t*)bs.cursor.p, (int32_t*)bs.list.p, (const int32_t*)bs.offsets.p, d_status, st);
    CUDA_TRY(c, cudaGetLastError());
  }
  c->stats.launches += 2 * ((F > 0 ? 2 : 0) + 3);
  c->stats.bin_entries = totals[0] + totals[1];
  // work split over sub-frame groups so that small images still fill the SMs
  int ns = c->splits;
  if (ns <= 0) ns = (8 * c->num_sms + pp.n_tiles - 1) / pp.n_tiles;
  pp.n_split = std::max(1, std::min(ns, pp.G));
  return MBR_OK;
}

RasterParams raster_params(mbr_ctx* c, const mbr_mesh* mesh, const mbr_camera* cam, int T, int H, int W,
                           const Prepared& pp) {
  RasterParams P;
  std::memset(&P, 0, sizeof(P));
  P.recs = (const TriRec*)c->recs.p;
  P.groups = pp.d_groups;
  P.core.off = (const int32_t*)c->core.offsets.p;
  P.core.faces = (const int32_t*)c->core.list.p;
  P.soft.off = (const int32_t*)c->soft.offsets.p;
  P.soft.faces = (const int32_t*)c->soft.list.p;
  P.slot_nrm = (const float4*)c->nrm.p;
  P.faces = mesh->faces;
  P.albedo = mesh->albedo;
  P.F = mesh->F;
  P.V = mesh->V;
  P.G = pp.G;
  P.H = H;
  P.W = W;
  P.tiles_x = pp.tiles_x;
  P.tiles_y = pp.tiles_y;
  P.n_split = pp.n_split;
  P.r = pp.r;
  P.r2 = pp.r * pp.r;
  P.delta = cam->delta;
  P.inv_delta = 1.0f / cam->delta;
  double L[3] = {cam->light_dir[0], cam->light_dir[1], cam->light_dir[2]};
  const double ln = std::sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
  if (ln > 0) for (double& x : L) x /= ln;
  P.lx = (float)L[0];
  P.ly = (float)L[1];
  P.lz = (float)L[2];
  P.ka = cam->k_ambient;
  P.kd = cam->k_diffuse;
  P.inv_T = (float)(1.0 / T);
  P.dbg_k = -1;
  return P;
}

int forward_impl(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam, int T, int H,
                 int W, int solver, float* image, int dbg_k, int32_t* dbg_ids, cudaStream_t st) {
  int rc = validate(c, mesh, motion, cam, T, H, W, solver);
  if (rc) return rc;
  if (!image && !dbg_ids) return fail(c, MBR_ERR_ARG, "null image");
  Prepared pp;
  if ((rc = prepare(c, mesh, motion, cam, T, H, W, solver, st, true, pp))) return rc;
  RasterParams P = raster_params(c, mesh, cam, T, H, W, pp);
  const size_t npix = (size_t)H * W;
  if (dbg_ids) {
    P.dbg_k = dbg_k;
    P.dbg_ids = dbg_ids;
  }
  if (pp.n_split > 1 || !image) {
    if ((rc = ensure(c, c->partial, sizeof(float4) * npix * pp.n_split, st))) return rc;
    P.out = (float4*)c->partial.p;
  } else {
    P.out = (float4*)image;
  }
  if ((rc = time_begin(c, 0, st))) return rc;
  launch_raster_fwd(P, c->tile, pp.spt, pp.moving, st);
  CUDA_TRY(c, cudaGetLastError());
  if ((rc = time_end(c, 0, st))) return rc;
  c->stats.launches += 1;
  c->stats.n_split = pp.n_split;
  if (pp.n_split > 1 && image) {
    launch_finalize((const float4*)c->partial.p, pp.n_split, npix, P.inv_T, (float4*)image, st);
    CUDA_TRY(c, cudaGetLastError());
    c->stats.launches += 1;
  }
  return MBR_OK;
}

}  // namespace

extern "C" {

int mbr_create(mbr_ctx** out) {
  if (!out) return MBR_ERR_ARG;
  *out = nullptr;
  mbr_ctx* c = new (std::nothrow) mbr_ctx();
  if (!c) return MBR_ERR_OOM;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return MBR_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
  if (c->num_sms < 1) c->num_sms = 1;
  if (cudaMallocHost(&c->host_total, sizeof(int32_t) * 4) != cudaSuccess) {
    delete c;
    return MBR_ERR_OOM;
  }
  *out = c;
  return MBR_OK;
}

void mbr_destroy(mbr_ctx* c) {
  if (!c) return;
  DevBuf* bufs[] = {&c->nacc, &c->pos, &c->nrm, &c->recs, &c->tables, &c->partial, &c->gslot, &c->galb, &c->gm,
                    &c->cnt64,
                    &c->status, &c->core.counts, &c->core.offsets, &c->core.cursor, &c->core.list,
                    &c->core.scan_tmp, &c->soft.counts, &c->soft.offsets, &c->soft.cursor, &c->soft.list,
                    &c->soft.scan_tmp};
  cudaDeviceSynchronize();
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->host_stage) cudaFreeHost(c->host_stage);
  if (c->host_total) cudaFreeHost(c->host_total);
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < 2; ++q)
      if (c->ev[k][q]) cudaEventDestroy(c->ev[k][q]);
  delete c;
}

int mbr_set_profiling(mbr_ctx* c, int32_t on) {
  if (!c) return MBR_ERR_ARG;
  c->pending[0] = c->pending[1] = false;
  c->profiling = on != 0;
  c->stats.raster_fwd_ms = c->stats.raster_bwd_ms = 0.0;
  c->stats.raster_fwd_count = c->stats.raster_bwd_count = 0;
  return MBR_OK;
}

int mbr_get_stats(mbr_ctx* c, mbr_stats* out) {
  if (!c || !out) return MBR_ERR_ARG;
  int rc = harvest(c, 0);
  if (!rc) rc = harvest(c, 1);
  if (rc) return rc;
  *out = c->stats;
  return MBR_OK;
}

const char* mbr_last_error(mbr_ctx* c) { return c ? c->err.c_str() : "null context"; }

int mbr_set_tuning(mbr_ctx* c, int32_t tile, int32_t spt, int32_t splits) {
  if (!c) return MBR_ERR_ARG;
  if (tile != 8 && tile != 16) return fail(c, MBR_ERR_ARG, "tile must be 8 or 16");
  if (spt < 1 || spt > kMaxSpt) return fail(c, MBR_ERR_ARG, "spt must be in [1, %d]", kMaxSpt);
  if (splits < 0) return fail(c, MBR_ERR_ARG, "splits must be >= 0");
  c->tile = tile;
  c->spt = spt;
  c->splits = splits;
  return MBR_OK;
}

int mbr_render_blur(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam, int32_t T,
                    int32_t H, int32_t W, int32_t solver, float* image, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  return forward_impl(c, mesh, motion, cam, T, H, W, solver, image, -1, nullptr, (cudaStream_t)stream);
}

int mbr_debug_winners(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam, int32_t T,
                      int32_t H, int32_t W, int32_t solver, int32_t k, int32_t* ids, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  if (!ids) return fail(c, MBR_ERR_ARG, "null ids");
  if (k < 0 || k >= T) return fail(c, MBR_ERR_ARG, "sub-frame %d out of range", k);
  return forward_impl(c, mesh, motion, cam, T, H, W, solver, nullptr, k, ids, (cudaStream_t)stream);
}

int mbr_render_blur_backward(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam,
                             int32_t T, int32_t H, int32_t W, int32_t solver, const float* dl_dimage,
                             float* dl_dverts, float* dl_dalbedo, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  cudaStream_t st = (cudaStream_t)stream;
  int rc = validate(c, mesh, motion, cam, T, H, W, solver);
  if (rc) return rc;
  if (!dl_dimage || !dl_dverts) return fail(c, MBR_ERR_ARG, "null gradient buffer");
  Prepared pp;
  if ((rc = prepare(c, mesh, motion, cam, T, H, W, solver, st, true, pp))) return rc;
  RasterParams P = raster_params(c, mesh, cam, T, H, W, pp);
  const int V = mesh->V;
  const size_t gbytes = sizeof(float4) * 2 * (size_t)V * pp.n_slots;
  if ((rc = ensure(c, c->gslot, gbytes, st))) return rc;
  if ((rc = ensure(c, c->gm, sizeof(float) * 3 * V, st))) return rc;
  if ((rc = ensure(c, c->galb, sizeof(float4) * V, st))) return rc;
  CUDA_TRY(c, cudaMemsetAsync(c->gslot.p, 0, gbytes, st));
  if (dl_dalbedo) CUDA_TRY(c, cudaMemsetAsync(c->galb.p, 0, sizeof(float4) * V, st));
  P.dl_dimage = (const float4*)dl_dimage;
  P.g_slot = (float4*)c->gslot.p;
  P.g_albedo = dl_dalbedo ? (float4*)c->galb.p : nullptr;
  if ((rc = time_begin(c, 1, st))) return rc;
  launch_raster_bwd(P, c->tile, pp.spt, pp.moving, st);
  CUDA_TRY(c, cudaGetLastError());
  if ((rc = time_end(c, 1, st))) return rc;
  c->stats.launches += 1 + 1 + (mesh->F > 0 ? 1 : 0);
  c->stats.n_split = pp.n_split;
  launch_slot_chain(mesh->verts, (const float*)c->nacc.p, V, pp.d_xf, pp.n_slots, cam->tan_half_fov,
                    (const float4*)c->gslot.p, (const float4*)c->galb.p, dl_dverts, (float*)c->gm.p, dl_dalbedo, st);
  launch_normals_bwd(mesh->verts, mesh->faces, mesh->F, V, (const float*)c->gm.p, dl_dverts, st);
  CUDA_TRY(c, cudaGetLastError());
  return MBR_OK;
}

int mbr_count_candidates(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam,
                         int32_t T, int32_t H, int32_t W, int32_t solver, int64_t* out, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  cudaStream_t st = (cudaStream_t)stream;
  int rc = validate(c, mesh, motion, cam, T, H, W, solver);
  if (rc) return rc;
  if (!out) return fail(c, MBR_ERR_ARG, "null out");
  Prepared pp;
  if ((rc = prepare(c, mesh, motion, cam, T, H, W, solver, st, false, pp))) return rc;
  if ((rc = ensure(c, c->cnt64, sizeof(unsigned long long), st))) return rc;
  CUDA_TRY(c, cudaMemsetAsync(c->cnt64.p, 0, sizeof(unsigned long long), st));
  // N_cand keeps its definition: boxes dilated by sqrt(delta ln 1e12)
  const float r_count = (float)std::sqrt((double)cam->delta * std::log(1e12));
  launch_count((const TriRec*)c->recs.p, mesh->F, pp.d_groups, pp.G, W, H, r_count,
               (unsigned long long*)c->cnt64.p, st);
  c->stats.launches += mesh->F > 0 ? 1 : 0;
  CUDA_TRY(c, cudaGetLastError());
  unsigned long long h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, c->cnt64.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  *out = (int64_t)h;
  return MBR_OK;
}

int mbr_render_blur_batch(mbr_ctx* c, int32_t n, const mbr_item* items, int32_t with_backward, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  if (n < 0 || (n > 0 && !items)) return fail(c, MBR_ERR_ARG, "bad batch");
  for (int i = 0; i < n; ++i) {
    const mbr_item& it = items[i];
    int rc = forward_impl(c, &it.mesh, &it.motion, &it.camera, it.T, it.H, it.W, it.solver, it.image, -1, nullptr,
                          (cudaStream_t)stream);
    if (rc) return rc;
    if (with_backward) {
      rc = mbr_render_blur_backward(c, &it.mesh, &it.motion, &it.camera, it.T, it.H, it.W, it.solver, it.dl_dimage,
                                    it.dl_dverts, it.dl_dalbedo, stream);
      if (rc) return rc;
    }
  }
  return MBR_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free forward render
// mbr_render_blur_noalloc: the forward pipeline of mbr_render_blur, with every scratch buffer
// carved out of one file-scope device array instead of context-owned allocations.  The device
// address of the array is looked up once per device (cudaGetSymbolAddress) and passed to the
// kernels like any other pointer; in host code the array's name is only a stand-in.

constexpr size_t kStaticScratchBytes = size_t(32) << 20;  // per device, held until process exit
static __device__ __align__(256) unsigned char g_mbr_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices] = {};

struct Arena {
  char* base;
  size_t cap, used;
  void* take(size_t bytes) {
    const size_t o = (used + 255) & ~size_t(255);
    if (o > cap || bytes > cap - o) return nullptr;
    used = o + bytes;
    return base + o;
  }
};

int noalloc_forward(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam, int T, int H,
                    int W, int solver, float* image, cudaStream_t st) {
  int rc = validate(c, mesh, motion, cam, T, H, W, solver);
  if (rc) return rc;
  if (!image) return fail(c, MBR_ERR_ARG, "null image");
  int dev = 0;
  CUDA_TRY(c, cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(c, MBR_ERR_ARG, "device %d out of range", dev);
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
      void* p = nullptr;
      CUDA_TRY(c, cudaGetSymbolAddress(&p, g_mbr_static_scratch));
      g_static_addr[dev] = p;
    }
    base = g_static_addr[dev];
  }

  std::vector<SlotXform> xf;
  std::vector<int2> sets;
  std::vector<Group> groups;
  Prepared pp;
  if ((rc = build_tables(c, motion, cam, T, solver, xf, sets, groups, pp))) return rc;
  const int V = mesh->V, F = mesh->F, tw = 16, th = 16;
  pp.tiles_x = (W + tw - 1) / tw;
  pp.tiles_y = (H + th - 1) / th;
  pp.n_tiles = pp.tiles_x * pp.tiles_y;
  pp.n_split = 1;
  pp.r = (float)std::sqrt((double)cam->delta * (double)kSoftCutoff);
  const long long nb = (long long)pp.G * pp.n_tiles;

  // fixed part of the arena
  Arena A{(char*)base, kStaticScratchBytes, 0};
  int* d_status = (int*)A.take(sizeof(int32_t));
  float* nacc = (float*)A.take(sizeof(float) * 3 * (size_t)V);
  float4* pos = (float4*)A.take(sizeof(float4) * (size_t)pp.n_slots * V);
  float4* nrm = (float4*)A.take(sizeof(float4) * (size_t)pp.n_slots * V);
  TriRec* recs = (TriRec*)A.take(sizeof(TriRec) * (size_t)pp.n_sets * std::max(F, 1));
  SlotXform* d_xf = (SlotXform*)A.take(sizeof(SlotXform) * xf.size());
  int2* d_sets = (int2*)A.take(sizeof(int2) * sets.size());
  Group* d_groups = (Group*)A.take(sizeof(Group) * groups.size());
  int32_t *counts[2], *offs[2], *tmp[2], *cursor[2], *list[2];
  for (int q = 0; q < 2; ++q) {
    counts[q] = (int32_t*)A.take(sizeof(int32_t) * (size_t)nb);
    offs[q] = (int32_t*)A.take(sizeof(int32_t) * (size_t)(nb + 1));
    tmp[q] = (int32_t*)A.take(sizeof(int32_t) * scan_temp_ints((int)nb));
    cursor[q] = (int32_t*)A.take(sizeof(int32_t) * (size_t)nb);
  }
  if (!d_status || !nacc || !pos || !nrm || !recs || !d_xf || !d_sets || !d_groups || !counts[1] || !offs[1] ||
      !tmp[1] || !cursor[1] || nb > (1LL << 30))
    return fail(c, MBR_ERR_ARG,
                "render needs more than the %zu MiB static scratch (V=%d F=%d T=%d %dx%d); use mbr_render_blur",
                kStaticScratchBytes >> 20, V, F, T, W, H);
  pp.d_xf = d_xf;
  pp.d_groups = d_groups;
  CUDA_TRY(c, cudaMemcpyAsync(d_xf, xf.data(), sizeof(SlotXform) * xf.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, cudaMemcpyAsync(d_sets, sets.data(), sizeof(int2) * sets.size(), cudaMemcpyHostToDevice, st));
  CUDA_TRY(c, cudaMemcpyAsync(d_groups, groups.data(), sizeof(Group) * groups.size(), cudaMemcpyHostToDevice, st));

  // the array keeps the previous call's contents: clear everything that accumulates
  CUDA_TRY(c, cudaMemsetAsync(d_status, 0, sizeof(int32_t), st));
  CUDA_TRY(c, cudaMemsetAsync(nacc, 0, sizeof(float) * 3 * V, st));
  launch_face_normals(mesh->verts, mesh->faces, F, V, nacc, d_status, st);
  launch_xform(mesh->verts, nacc, V, d_xf, pp.n_slots, cam->tan_half_fov, pos, nrm, st);
  launch_setup(pos, mesh->faces, F, V, d_sets, pp.n_sets, cam->znear, recs, st);
  const float margins[2] = {kCoreMargin, pp.r + kCoreMargin};
  int32_t host[3] = {0, 0, 0};
  for (int q = 0; q < 2; ++q) {
    CUDA_TRY(c, cudaMemsetAsync(counts[q], 0, sizeof(int32_t) * (size_t)nb, st));
    launch_bin(false, recs, F, d_groups, pp.G, W, H, tw, th, pp.tiles_x, pp.n_tiles, margins[q], counts[q], nullptr,
               nullptr, d_status, st);
    launch_scan(counts[q], (int)nb, offs[q], tmp[q], st);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(host + q, offs[q] + nb, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(c, cudaMemcpyAsync(host + 2, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (host[2] & kStatusBadFace) return fail(c, MBR_ERR_ARG, "face index outside [0, V)");
  for (int q = 0; q < 2; ++q) {
    list[q] = (int32_t*)A.take(sizeof(int32_t) * (size_t)std::max(host[q], 1));
    if (host[q] < 0 || !list[q])
      return fail(c, MBR_ERR_ARG, "tile lists (%d + %d entries) exceed the %zu MiB static scratch; use mbr_render_blur",
                  host[0], host[1], kStaticScratchBytes >> 20);
  }
  for (int q = 0; q < 2; ++q) {
    CUDA_TRY(c, cudaMemcpyAsync(cursor[q], offs[q], sizeof(int32_t) * (size_t)nb, cudaMemcpyDeviceToDevice, st));
    launch_bin(true, recs, F, d_groups, pp.G, W, H, tw, th, pp.tiles_x, pp.n_tiles, margins[q], cursor[q], list[q],
               offs[q], d_status, st);
  }
  CUDA_TRY(c, cudaGetLastError());

  // raster, writing the caller's image directly (one split, no partial sums)
  c->recs.p = recs;
  c->nrm.p = nrm;
  c->core.offsets.p = offs[0];
  c->core.list.p = list[0];
  c->soft.offsets.p = offs[1];
  c->soft.list.p = list[1];
  RasterParams P = raster_params(c, mesh, cam, T, H, W, pp);
  P.out = (float4*)image;
  launch_raster_fwd(P, tw, pp.spt, pp.moving, st);
  CUDA_TRY(c, cudaGetLastError());
  return MBR_OK;
}

}  // namespace

extern "C" int mbr_render_blur_noalloc(const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* camera,
                                       int32_t T, int32_t H, int32_t W, int32_t solver, float* image,
                                       void* cuda_stream, char* err, int32_t err_len) {
  mbr_ctx local;  // default tuning and an error sink; its buffers are pointed into the static array
  const int rc = noalloc_forward(&local, mesh, motion, camera, T, H, W, solver, image, (cudaStream_t)cuda_stream);
  if (err && err_len > 0) {
    std::strncpy(err, local.err.c_str(), (size_t)err_len - 1);
    err[err_len - 1] = '\0';
  }
  return rc;
}
