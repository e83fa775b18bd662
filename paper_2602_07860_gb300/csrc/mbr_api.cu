// mbr_api.cu -- host side of the C ABI declared in include/mbr.h.
//
// Per call: validate arguments -> time map (Secs. 3.2-3.3, exact integer arithmetic) -> per-slot
// motion + camera matrices (double precision, one 3x4 per slot time) -> kernels on the caller's
// stream: normals, transform, triangle setup, tile binning (count, scan, one stream sync to
// size the face lists, fill), unit cost order, raster.  Backward reruns the same front half and the
// adjoint raster, then chains slot gradients to vertices.
#include <algorithm>
#include <atomic>
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
  DevBuf offsets, list, scan_tmp;
};

struct BatchState;  // batched renders (defined with mbr_render_blur_batch)
struct Prepared;    // front half of one render (defined below)
struct FwdCostKey {  // unit layout whose measured forward costs the order buffer holds
  bool valid = false;
  int n_units = 0, G = 0, n_tiles = 0, n_split = 0, tile = 0;
  const void* buf = nullptr;
};

// arguments of the last mbr_render_blur, whose front half the adjoint may reuse
struct LastForward {
  bool valid = false;
  mbr_mesh mesh;
  mbr_motion motion;
  mbr_camera cam;
  int T = 0, H = 0, W = 0, solver = 0, tile = 0, spt = 0, splits = 0;
  long long state_budget = 0;
};

}  // namespace

struct mbr_ctx {
  int device = 0;
  int num_sms = 1;
  std::string err;
  // tuning
  int tile = 16, spt = 2, splits = 0;
  long long state_budget = 1LL << 30;  // the forward keeps per-sample state for the adjoint up to this size
  // scratch
  DevBuf nacc, pos, nrm, recs, tables, partial, gslot, galb, gm, cnt64, status, order, bstate, bin_counts;
  DevBuf sdf_cnt, sdf_off, sdf_tmp;  // SDF extraction: edge flags + triangle counts, their scans
  FwdCostKey fcost;  // unit layout of the last forward whose per-unit cost is in the order buffer
  BinSet core, soft;  // undilated bins (coverage) and r_soft-dilated bins (soft coverage)
  void* host_stage = nullptr;
  size_t host_stage_cap = 0;
  int32_t* host_total = nullptr;
  // persistent-raster work queue of single renders: params + offsets + counter (device), and a
  // pinned host copy of the params
  DevBuf queue;
  void* host_queue = nullptr;
  size_t host_queue_cap = 0;
  cudaEvent_t queue_copied = nullptr;  // recorded after each copy out of host_queue
  // batch plans (mbr_render_blur_batch): arena per plan, captured graph, pinned staging
  BatchState* batch = nullptr;
  // the last forward's front half (records, bins, unit order, normals stay in the buffers above)
  LastForward last;
  Prepared* last_pp = nullptr;
  // measurement: one event pair per raster kind (0 forward, 1 adjoint), harvested lazily
  bool profiling = false;
  cudaEvent_t ev[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool pending[2] = {false, false};
  mbr_stats stats{};
};

namespace {

constexpr double kPi = 3.14159265358979323846;

// bounded-wait test hook (mbr_debug_wait_limit): applies to raster launches issued after it is set
std::atomic<int32_t> g_wait_polls{0}, g_wait_stall{0}, g_wait_check{0};

void set_wait_fields(WorkQueue& Q) {
  const int32_t polls = g_wait_polls.load();
  Q.spin_limit = polls > 0 ? polls : kSpinLimit;
  Q.stall = g_wait_stall.load() ? 1 : 0;
}

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
    if (n > 0) {
      for (double& x : k) x /= n;
      rotation(k, (double)m->omega * t, Rm);
    }
    if (m->kind == MBR_PARABOLIC)
      for (int i = 0; i < 3; ++i) b[i] = (double)m->offset[i] + t * (double)m->dir[i] + t * t * (double)m->acc[i];
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
  if (mesh->texture && (!mesh->uv || mesh->tex_h < 1 || mesh->tex_w < 1 || mesh->tex_h > 65536 || mesh->tex_w > 65536))
    return fail(c, MBR_ERR_ARG, "a texture needs uv coordinates and a size in [1, 65536]");
  if (T < 1 || T > (1 << 20)) return fail(c, MBR_ERR_ARG, "bad T=%d", T);
  if (H < 1 || W < 1 || H > 16384 || W > 16384) return fail(c, MBR_ERR_ARG, "bad image size %dx%d", H, W);
  if (solver != MBR_PLAIN && solver != MBR_FAST) return fail(c, MBR_ERR_ARG, "bad solver %d", solver);
  if (motion->kind != MBR_TRANSLATE && motion->kind != MBR_ROTATE && motion->kind != MBR_PARABOLIC)
    return fail(c, MBR_ERR_ARG, "bad motion kind %d", motion->kind);
  if (motion->segments < 0 || motion->segments > 1000000) return fail(c, MBR_ERR_ARG, "bad segments");
  if ((motion->kind == MBR_ROTATE || (motion->kind == MBR_PARABOLIC && motion->omega != 0.f)) &&
      !(motion->axis[0] * motion->axis[0] + motion->axis[1] * motion->axis[1] + motion->axis[2] * motion->axis[2] > 0.f))
    return fail(c, MBR_ERR_ARG, "zero rotation axis");
  if (!(cam->tan_half_fov > 0.f) || !(cam->delta > 0.f)) return fail(c, MBR_ERR_ARG, "bad camera fov/delta");
  if (cam->prob != MBR_PROB_EXP && cam->prob != MBR_PROB_SIGMOID) return fail(c, MBR_ERR_ARG, "bad probability map");
  if (cam->interp != MBR_INTERP_SCREEN && cam->interp != MBR_INTERP_PERSPECTIVE)
    return fail(c, MBR_ERR_ARG, "bad attribute interpolation");
  if (cam->time_rule != MBR_TIME_PAPER && cam->time_rule != MBR_TIME_MIDPOINT)
    return fail(c, MBR_ERR_ARG, "bad time rule");
  const long long T_ = T;
  if (solver == MBR_FAST && (long long)num_segments(motion) > 4 * T_ + 64)
    return fail(c, MBR_ERR_ARG, "segments %d far exceed T=%d", num_segments(motion), T);
  return MBR_OK;
}

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
  int core_cap = 0, soft_cap = 0;  // bin list capacities
  int n_units = 0;                  // raster work units: patches x n_split
  int32_t* d_order = nullptr;       // their visiting order (estimate from the bins)
  int32_t* d_order_bwd = nullptr;   // the adjoint's visiting order (from the forward's measured cost)
  int32_t* d_cost = nullptr;        // the forward's measured adjoint cost per unit
  int32_t* d_fcost = nullptr;       // the forward's measured own cost per unit
  int32_t* d_order_tmp = nullptr;   // scratch of the order kernels
  bool stored = false;              // the forward kept the per-sample state (else the adjoint recomputes it)
};

// the forward keeps the adjoint's per-sample state (5 bytes per pixel and sub-frame) within the budget
bool keeps_state(const mbr_ctx* c, int T, int H, int W) {
  return (double)T * H * W * 5.0 <= (double)c->state_budget;
}

// order buffer of a render: order | adjoint order | adjoint cost | forward cost | scratch
size_t order_buffer_ints(int n_units) { return (size_t)4 * n_units + unit_order_ints(n_units); }

void carve_orders(int32_t* base, Prepared& pp) {
  pp.d_order = base;
  pp.d_order_bwd = base + pp.n_units;
  pp.d_cost = base + 2 * (size_t)pp.n_units;
  pp.d_fcost = base + 3 * (size_t)pp.n_units;
  pp.d_order_tmp = base + 4 * (size_t)pp.n_units;
}

// a render that uses a variant (texture colours, perspective-correct weights, sigmoid map) runs
// the raster kernels compiled with them; the paper's default path runs kernels without their code
bool uses_variants(const mbr_mesh* mesh, const mbr_camera* cam) {
  return mesh->texture != nullptr || cam->interp != MBR_INTERP_SCREEN || cam->prob != MBR_PROB_EXP;
}

int raster_kind(const Prepared& pp, const mbr_mesh* mesh, const mbr_camera* cam) {
  return (pp.moving ? 1 : 0) | (uses_variants(mesh, cam) ? kKindExt : 0);
}

// units of a render: 256-pixel patches x group splits
int patches_of(int tile, int n_tiles) {
  return tile == 8 ? UnitMap<8, 8>::patches(n_tiles) : UnitMap<16, 16>::patches(n_tiles);
}

// Group splits: enough units (about 64 per SM) for the largest-first order to balance the SMs;
// more splits add one float4 atomic per pixel and split in the forward.
int choose_splits(const mbr_ctx* c, int G, int n_patches) {
  int ns = c->splits;
  if (ns <= 0) ns = (int)std::min<long long>(G, (64LL * c->num_sms + n_patches - 1) / std::max(1, n_patches));
  return std::max(1, std::min(ns, std::max(G, 1)));
}

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
  c->last.valid = false;  // the buffers are about to be rewritten
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
  int* d_status = (int*)c->status.p;  // [0] this call, [1] raster launches (sticky until read)
  // one launch clears this call's status word, the normal accumulators and both bin count arrays
  ZeroList zl{};
  zl.p[0] = d_status;
  zl.n[0] = 1;
  zl.p[1] = (int32_t*)c->nacc.p;
  zl.n[1] = (size_t)3 * V;
  const int tw = c->tile, th = c->tile;
  long long nb = 0;
  if (do_bins) {
    pp.tiles_x = (W + tw - 1) / tw;
    pp.tiles_y = (H + th - 1) / th;
    pp.n_tiles = pp.tiles_x * pp.tiles_y;
    nb = (long long)pp.G * pp.n_tiles;
    if (nb > (1LL << 30)) return fail(c, MBR_ERR_ARG, "too many (group, tile) bins: %lld", nb);
    // both count arrays in one buffer; after the scan they are the fill cursors
    if ((rc = ensure(c, c->bin_counts, sizeof(int32_t) * 2 * (size_t)nb, st))) return rc;
    zl.p[2] = (int32_t*)c->bin_counts.p;
    zl.n[2] = 2 * (size_t)nb;
  }
  launch_zero(zl, st);
  launch_face_normals(mesh->verts, mesh->faces, F, V, (float*)c->nacc.p, d_status, st);
  launch_xform(mesh->verts, (const float*)c->nacc.p, V, pp.d_xf, pp.n_slots, cam->tan_half_fov,
               (float4*)c->pos.p, (float4*)c->nrm.p, st);
  launch_setup((const float4*)c->pos.p, mesh->faces, F, V, d_sets, pp.n_sets, cam->znear, (TriRec*)c->recs.p, st);
  CUDA_TRY(c, cudaGetLastError());
  pp.r = (float)std::sqrt((double)cam->delta * (double)kSoftCutoff);
  c->stats.launches += 1 + (F > 0 ? 1 : 0) + 1 + (F > 0 ? 1 : 0);  // clear, normals, transform, setup
  c->stats.groups = pp.G;
  if (!do_bins) {
    CUDA_TRY(c, cudaMemcpyAsync(c->host_total, d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    if (c->host_total[0] & kStatusBadFace) return fail(c, MBR_ERR_ARG, "face index outside [0, V)");
    return MBR_OK;
  }

  // a3 binning: core and soft bins: count -> scan (both) -> one sync for the totals -> fill (the
  // count arrays were cleared above)
  BinSet* sets2[2] = {&c->core, &c->soft};
  const float r_core = kCoreMargin, r_soft = pp.r + kCoreMargin;
  BinTargets bt{};
  ScanPair sp{};
  for (int q = 0; q < 2; ++q) {
    BinSet& bs = *sets2[q];
    if ((rc = ensure(c, bs.offsets, sizeof(int32_t) * (size_t)(nb + 1), st))) return rc;
    if ((rc = ensure(c, bs.scan_tmp, sizeof(int32_t) * scan_temp_ints((int)nb), st))) return rc;
    bt.counts_or_cursor[q] = (int32_t*)c->bin_counts.p + q * (size_t)nb;
    sp.in[q] = bt.counts_or_cursor[q];
    sp.out[q] = (int32_t*)bs.offsets.p;
    sp.sums[q] = (int32_t*)bs.scan_tmp.p;
  }
  sp.total = d_status + 2;  // [2] core, [3] soft list totals
  sp.n = (int)nb;
  launch_bin(false, (const TriRec*)c->recs.p, F, pp.d_groups, pp.G, W, H, tw, th, pp.tiles_x, pp.n_tiles, r_core,
             r_soft, bt, d_status, st);
  const int scan_launches = launch_scan_pair(sp, st);
  CUDA_TRY(c, cudaGetLastError());
  // one read-back: [0] this call's status, [1] raster launches' status, [2], [3] list totals
  CUDA_TRY(c, cudaMemcpyAsync(c->host_total, d_status, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (c->host_total[0] & kStatusBadFace) return fail(c, MBR_ERR_ARG, "face index outside [0, V)");
  if (c->host_total[1] & kStatusSpin) {
    CUDA_TRY(c, cudaMemsetAsync(d_status + 1, 0, sizeof(int32_t), st));
    return fail(c, MBR_ERR_TIMEOUT, "a raster launch of an earlier call gave up a bounded wait (its output is incomplete)");
  }
  long long totals[2] = {c->host_total[2], c->host_total[3]};
  for (int q = 0; q < 2; ++q) {
    BinSet& bs = *sets2[q];
    if (totals[q] < 0) return fail(c, MBR_ERR_DEVICE, "bin total overflow");
    if ((rc = ensure(c, bs.list, sizeof(int32_t) * (size_t)std::max<long long>(totals[q], 1), st))) return rc;
    bt.list[q] = (int32_t*)bs.list.p;
    bt.off[q] = (const int32_t*)bs.offsets.p;
    bt.cap[q] = (int)totals[q];
  }
  launch_bin(true, (const TriRec*)c->recs.p, F, pp.d_groups, pp.G, W, H, tw, th, pp.tiles_x, pp.n_tiles, r_core,
             r_soft, bt, d_status, st);
  CUDA_TRY(c, cudaGetLastError());
  c->stats.launches += (F > 0 ? 2 : 0) + scan_launches;
  c->stats.bin_entries = totals[0] + totals[1];
  pp.core_cap = (int)totals[0];
  pp.soft_cap = (int)totals[1];
  // work units: patches x group splits, visited largest estimate first
  const int n_patches = patches_of(tw, pp.n_tiles);
  pp.n_split = choose_splits(c, pp.G, n_patches);
  pp.n_units = n_patches * pp.n_split;
  if ((rc = ensure(c, c->order, sizeof(int32_t) * order_buffer_ints(pp.n_units), st))) return rc;
  carve_orders((int32_t*)c->order.p, pp);
  // The previous forward of the same unit layout measured each unit's work: visit the units in
  // that order (an optimisation loop's geometry moves little between calls); otherwise estimate
  // from the bin sizes.  Either way both cost arrays are cleared for this render's measurements.
  const FwdCostKey& K = c->fcost;
  if (K.valid && K.buf == c->order.p && K.n_units == pp.n_units && K.G == pp.G && K.n_tiles == pp.n_tiles &&
      K.n_split == pp.n_split && K.tile == tw)
    launch_unit_order_measured(pp.d_fcost, pp.n_units, pp.d_order, pp.d_order_tmp, pp.d_fcost, pp.d_cost, st);
  else
    launch_unit_order((const int32_t*)c->core.offsets.p, (const int32_t*)c->soft.offsets.p, pp.G, pp.n_tiles, tw,
                      pp.n_split, pp.n_units, pp.d_order, pp.d_order_tmp, pp.d_cost, pp.d_fcost, st);
  c->fcost.valid = false;  // until this render's forward has measured
  CUDA_TRY(c, cudaGetLastError());
  c->stats.launches += 1;
  return MBR_OK;
}

// device buffers one render's raster reads (the context's own, a batch slice or the static scratch)
struct RasterBufs {
  const void* recs;
  const void* nrm;
  const void* off[2];   // core, soft bin offsets
  const void* list[2];  // core, soft face lists
};

RasterBufs ctx_bufs(const mbr_ctx* c) {
  return RasterBufs{c->recs.p, c->nrm.p, {c->core.offsets.p, c->soft.offsets.p}, {c->core.list.p, c->soft.list.p}};
}

RasterParams raster_params(const mbr_ctx* c, const RasterBufs& b, const mbr_mesh* mesh, const mbr_camera* cam, int T,
                           int H, int W, const Prepared& pp) {
  RasterParams P;
  std::memset(&P, 0, sizeof(P));
  P.recs = (const TriRec*)b.recs;
  P.groups = pp.d_groups;
  P.core.off = (const int32_t*)b.off[0];
  P.core.faces = (const int32_t*)b.list[0];
  P.soft.off = (const int32_t*)b.off[1];
  P.soft.faces = (const int32_t*)b.list[1];
  P.core.cap = pp.core_cap;
  P.soft.cap = pp.soft_cap;
  P.slot_nrm = (const float4*)b.nrm;
  P.faces = mesh->faces;
  P.albedo = mesh->albedo;
  if (mesh->texture) {
    P.uv = mesh->uv;
    P.tex = mesh->texture;
    P.tex_w = mesh->tex_w;
    P.tex_h = mesh->tex_h;
  }
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
  P.prob = cam->prob;
  P.persp = cam->interp == MBR_INTERP_PERSPECTIVE ? 1 : 0;
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
  P.moving = pp.moving ? 1 : 0;
  P.work = pp.n_units;
  P.order = pp.d_order;
  return P;
}

// Upload the params of the renders and their work offsets; the queue's counter is zeroed on st.
int upload_queue(mbr_ctx* c, const RasterParams* items, int n, cudaStream_t st, WorkQueue& Q) {
  const size_t par_b = sizeof(RasterParams) * n, off_b = sizeof(int32_t) * (n + 1);
  const size_t off_at = (par_b + 255) & ~size_t(255), cnt_at = (off_at + off_b + 255) & ~size_t(255);
  const size_t total = cnt_at + 256;
  int rc;
  if ((rc = ensure(c, c->queue, total, st))) return rc;
  // the previous copy out of the pinned staging buffer may still be queued (a reused front half
  // skips the binning sync): wait for it before rewriting the buffer
  if (c->queue_copied) CUDA_TRY(c, cudaEventSynchronize(c->queue_copied));
  if (total > c->host_queue_cap) {
    CUDA_TRY(c, cudaStreamSynchronize(st));
    if (c->host_queue) cudaFreeHost(c->host_queue);
    c->host_queue = nullptr;
    c->host_queue_cap = 0;
    if (cudaMallocHost(&c->host_queue, total + total / 4) != cudaSuccess)
      return fail(c, MBR_ERR_OOM, "cudaMallocHost(%zu) failed", total);
    c->host_queue_cap = total + total / 4;
  }
  char* h = (char*)c->host_queue;
  std::memcpy(h, items, par_b);
  int32_t* off = (int32_t*)(h + off_at);
  off[0] = 0;
  for (int i = 0; i < n; ++i) off[i + 1] = off[i] + items[i].work;
  *(int32_t*)(h + cnt_at) = 0;  // the queue's counter travels with the parameters
  char* d = (char*)c->queue.p;
  CUDA_TRY(c, cudaMemcpyAsync(d, h, cnt_at + sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (!c->queue_copied) CUDA_TRY(c, cudaEventCreateWithFlags(&c->queue_copied, cudaEventDisableTiming));
  CUDA_TRY(c, cudaEventRecord(c->queue_copied, st));
  Q.items = (const RasterParams*)d;
  Q.item_off = (const int32_t*)(d + off_at);
  Q.n_items = n;
  Q.n_work = off[n];
  Q.counter = (int32_t*)(d + cnt_at);
  Q.status = (int32_t*)c->status.p + 1;
  set_wait_fields(Q);
  return MBR_OK;
}

// With the wait hook's check_now set: wait for the raster just launched and report a wait that gave
// up from this call (normally the next call's binning sync reports it).  word is the sticky status
// word of the raster's queue; it is cleared when reported.
int check_waits_now(mbr_ctx* c, int32_t* word, cudaStream_t st) {
  if (!g_wait_check.load()) return MBR_OK;
  int32_t h = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&h, word, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (h & kStatusSpin) {
    CUDA_TRY(c, cudaMemsetAsync(word, 0, sizeof(int32_t), st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    return fail(c, MBR_ERR_TIMEOUT, "a raster launch gave up a bounded wait (its output is incomplete)");
  }
  return MBR_OK;
}

// pp_out (optional) receives the front half of this render
int forward_impl(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam, int T, int H,
                 int W, int solver, float* image, int dbg_k, int32_t* dbg_ids, cudaStream_t st,
                 Prepared* pp_out = nullptr) {
  int rc = validate(c, mesh, motion, cam, T, H, W, solver);
  if (rc) return rc;
  if (!image && !dbg_ids) return fail(c, MBR_ERR_ARG, "null image");
  Prepared pp;
  if ((rc = prepare(c, mesh, motion, cam, T, H, W, solver, st, true, pp))) return rc;
  RasterParams P = raster_params(c, ctx_bufs(c), mesh, cam, T, H, W, pp);
  const size_t npix = (size_t)H * W;
  if (dbg_ids) {
    P.dbg_k = dbg_k;
    P.dbg_ids = dbg_ids;
  }
  if (!image) {  // winner ids only: the colours go to scratch
    if ((rc = ensure(c, c->partial, sizeof(float4) * npix, st))) return rc;
    P.out = (float4*)c->partial.p;
  } else {
    P.out = (float4*)image;
    // per-sample state for a following adjoint, within the budget: winner or log soft product
    // (4 B) + status (1 B); above it the adjoint recomputes them
    pp.stored = keeps_state(c, T, H, W);
    if (pp.stored) {
      const size_t ns = (size_t)T * npix;
      if ((rc = ensure(c, c->bstate, ns * 5 + 256, st))) return rc;
      P.s_val = (float*)c->bstate.p;
      P.s_stat = (uint8_t*)c->bstate.p + ns * 4;
    }
    P.unit_cost = pp.d_cost;  // and its cost per unit (cleared by the unit order), for the adjoint's order
    P.fwd_cost = pp.d_fcost;  // and its own, for the next forward's order
  }
  if (pp.n_split > 1) CUDA_TRY(c, cudaMemsetAsync(P.out, 0, sizeof(float4) * npix, st));  // splits accumulate
  WorkQueue Q;
  if ((rc = upload_queue(c, &P, 1, st, Q))) return rc;
  const int kind = raster_kind(pp, mesh, cam);
  const int grid = std::max(1, std::min(persistent_grid_fwd(c->num_sms, c->tile, pp.spt, kind), Q.n_work));
  if ((rc = time_begin(c, 0, st))) return rc;
  launch_raster_fwd(Q, c->tile, pp.spt, kind, grid, st);
  CUDA_TRY(c, cudaGetLastError());
  if ((rc = time_end(c, 0, st))) return rc;
  c->stats.launches += 1;
  c->stats.n_split = pp.n_split;
  if ((rc = check_waits_now(c, Q.status, st))) return rc;
  if (pp_out) *pp_out = pp;
  if (P.fwd_cost) c->fcost = FwdCostKey{true, pp.n_units, pp.G, pp.n_tiles, pp.n_split, c->tile, c->order.p};
  if (image && !dbg_ids) {
    if (!c->last_pp) c->last_pp = new (std::nothrow) Prepared();
    if (c->last_pp) {
      *c->last_pp = pp;
      LastForward& L = c->last;
      L.mesh = *mesh;
      L.motion = *motion;
      L.cam = *cam;
      L.T = T; L.H = H; L.W = W; L.solver = solver;
      L.tile = c->tile; L.spt = c->spt; L.splits = c->splits;
      L.state_budget = c->state_budget;
      L.valid = true;
    }
  }
  return MBR_OK;
}

// field-by-field equality (padding bytes of the caller's structs are not compared)
bool same_motion(const mbr_motion& a, const mbr_motion& b) {
  for (int i = 0; i < 3; ++i)
    if (a.offset[i] != b.offset[i] || a.dir[i] != b.dir[i] || a.axis[i] != b.axis[i]) return false;
  for (int i = 0; i < 3; ++i)
    if (a.acc[i] != b.acc[i]) return false;
  return a.kind == b.kind && a.segments == b.segments && a.omega == b.omega;
}

bool same_camera(const mbr_camera& a, const mbr_camera& b) {
  for (int i = 0; i < 12; ++i)
    if (a.view[i] != b.view[i]) return false;
  for (int i = 0; i < 3; ++i)
    if (a.light_dir[i] != b.light_dir[i]) return false;
  return a.tan_half_fov == b.tan_half_fov && a.znear == b.znear && a.k_ambient == b.k_ambient &&
         a.k_diffuse == b.k_diffuse && a.delta == b.delta && a.time_rule == b.time_rule && a.prob == b.prob &&
         a.interp == b.interp;
}

bool matches_last_forward(const mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam,
                          int T, int H, int W, int solver) {
  const LastForward& L = c->last;
  return L.valid && c->last_pp && L.mesh.V == mesh->V && L.mesh.F == mesh->F && L.mesh.verts == mesh->verts &&
         L.mesh.faces == mesh->faces && L.mesh.albedo == mesh->albedo && L.mesh.uv == mesh->uv &&
         L.mesh.texture == mesh->texture && L.mesh.tex_h == mesh->tex_h && L.mesh.tex_w == mesh->tex_w &&
         same_motion(L.motion, *motion) &&
         same_camera(L.cam, *cam) && L.T == T && L.H == H && L.W == W && L.solver == solver && L.tile == c->tile &&
         L.spt == c->spt && L.splits == c->splits && L.state_budget == c->state_budget;
}

// the adjoint (a9): front half and forward raster state (the last forward's when reuse is allowed
// and it matches, else recomputed: the forward raster runs again into scratch), adjoint raster,
// slot -> vertex chain, normals adjoint
int backward_impl(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam, int T, int H,
                  int W, int solver, const float* dl_dimage, float* dl_dverts, float* dl_dalbedo, cudaStream_t st,
                  bool reuse) {
  int rc = validate(c, mesh, motion, cam, T, H, W, solver);
  if (rc) return rc;
  if (!dl_dimage || !dl_dverts) return fail(c, MBR_ERR_ARG, "null gradient buffer");
  Prepared pp;
  if (reuse && matches_last_forward(c, mesh, motion, cam, T, H, W, solver)) {
    pp = *c->last_pp;
    c->stats.reused += 1;
  } else {
    // the forward raster writes the per-sample state (its image goes to scratch)
    if ((rc = ensure(c, c->partial, sizeof(float4) * (size_t)H * W, st))) return rc;
    if ((rc = forward_impl(c, mesh, motion, cam, T, H, W, solver, (float*)c->partial.p, -1, nullptr, st, &pp)))
      return rc;
    c->last.valid = false;  // the scratch image is not the caller's
  }
  RasterParams P = raster_params(c, ctx_bufs(c), mesh, cam, T, H, W, pp);
  const int V = mesh->V;
  const size_t gbytes = sizeof(float4) * 2 * (size_t)V * pp.n_slots;
  if ((rc = ensure(c, c->gslot, gbytes, st))) return rc;
  if ((rc = ensure(c, c->gm, sizeof(float) * 3 * V, st))) return rc;
  if ((rc = ensure(c, c->galb, sizeof(float4) * V, st))) return rc;
  // one launch clears the slot gradients and the albedo and texture gradients the raster adds to
  ZeroList zl{};
  zl.p[0] = (int32_t*)c->gslot.p;
  zl.n[0] = gbytes / 4;
  if (dl_dalbedo) {
    zl.p[1] = (int32_t*)c->galb.p;
    zl.n[1] = (size_t)4 * V;
  }
  P.dl_dimage = (const float4*)dl_dimage;
  P.g_slot = (float4*)c->gslot.p;
  P.g_albedo = dl_dalbedo ? (float4*)c->galb.p : nullptr;
  if (mesh->texture && mesh->dl_dtexture) {
    zl.p[2] = (int32_t*)mesh->dl_dtexture;
    zl.n[2] = (size_t)3 * mesh->tex_h * mesh->tex_w;
    P.g_tex = mesh->dl_dtexture;
  }
  launch_zero(zl, st);
  // the forward raster's per-sample state (if it kept it; else the adjoint recomputes it), and the
  // units in the order of its measured cost
  if (pp.stored) {
    const size_t ns = (size_t)T * H * W;
    P.s_val = (float*)c->bstate.p;
    P.s_stat = (uint8_t*)c->bstate.p + ns * 4;
  }
  launch_unit_order_measured(pp.d_cost, pp.n_units, pp.d_order_bwd, pp.d_order_tmp, nullptr, nullptr, st);
  P.order = pp.d_order_bwd;
  WorkQueue Q;
  if ((rc = upload_queue(c, &P, 1, st, Q))) return rc;
  const int kind = raster_kind(pp, mesh, cam);
  const int grid = std::max(1, std::min(persistent_grid_bwd(c->num_sms, c->tile, pp.spt, kind), Q.n_work));
  if ((rc = time_begin(c, 1, st))) return rc;
  launch_raster_bwd(Q, c->tile, pp.spt, kind, grid, st);
  CUDA_TRY(c, cudaGetLastError());
  if ((rc = time_end(c, 1, st))) return rc;
  if ((rc = check_waits_now(c, Q.status, st))) return rc;
  c->stats.launches += 1 + 3 + 1 + 1 + (mesh->F > 0 ? 1 : 0);  // clear, order, raster, slot chain, normals
  c->stats.n_split = pp.n_split;
  launch_slot_chain(mesh->verts, (const float*)c->nacc.p, V, pp.d_xf, pp.n_slots, cam->tan_half_fov,
                    (const float4*)c->gslot.p, (const float4*)c->galb.p, dl_dverts, (float*)c->gm.p, dl_dalbedo, st);
  launch_normals_bwd(mesh->verts, mesh->faces, mesh->F, V, (const float*)c->gm.p, dl_dverts, st);
  CUDA_TRY(c, cudaGetLastError());
  return MBR_OK;
}

void destroy_batch(mbr_ctx* c);
int batch_run(mbr_ctx* c, int n, const mbr_item* items, int with_backward, cudaStream_t st);

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
  if (cudaMallocHost(&c->host_total, sizeof(int32_t) * 16) != cudaSuccess) {
    delete c;
    return MBR_ERR_OOM;
  }
  if (cudaMalloc(&c->status.p, 256) != cudaSuccess || cudaMemset(c->status.p, 0, 256) != cudaSuccess) {
    if (c->status.p) cudaFree(c->status.p);
    cudaFreeHost(c->host_total);
    delete c;
    return MBR_ERR_OOM;
  }
  c->status.cap = 256;
  *out = c;
  return MBR_OK;
}

void mbr_destroy(mbr_ctx* c) {
  if (!c) return;
  DevBuf* bufs[] = {&c->nacc, &c->pos, &c->nrm, &c->recs, &c->tables, &c->partial, &c->gslot, &c->galb, &c->gm,
                    &c->cnt64, &c->order, &c->bstate, &c->sdf_cnt, &c->sdf_off, &c->sdf_tmp,
                    &c->status, &c->queue, &c->bin_counts, &c->core.offsets, &c->core.list,
                    &c->core.scan_tmp, &c->soft.offsets, &c->soft.list,
                    &c->soft.scan_tmp};
  cudaDeviceSynchronize();
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (c->host_stage) cudaFreeHost(c->host_stage);
  if (c->host_total) cudaFreeHost(c->host_total);
  if (c->host_queue) cudaFreeHost(c->host_queue);
  for (int k = 0; k < 2; ++k)
    for (int q = 0; q < 2; ++q)
      if (c->ev[k][q]) cudaEventDestroy(c->ev[k][q]);
  destroy_batch(c);
  delete c->last_pp;
  if (c->queue_copied) cudaEventDestroy(c->queue_copied);
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

int mbr_sdf_extract(mbr_ctx* c, int32_t n, const float* sdf, const float lo[3], float h, int32_t max_verts,
                    int32_t max_faces, float* verts, int32_t* faces, int32_t* vert_edges, int32_t* counts,
                    void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  if (n < 1 || n > 512 || !sdf || !lo || !(h > 0.f) || !counts || max_verts < 0 || max_faces < 0 ||
      (max_verts > 0 && !verts) || (max_faces > 0 && !faces))
    return fail(c, MBR_ERR_ARG, "bad SDF extraction arguments (n in [1, 512], h > 0, output buffers)");
  cudaStream_t st = (cudaStream_t)stream;
  const long long m = (long long)n + 1, n_edges = m * m * m * 7;  // >= the tetrahedron count n^3 6
  int rc;
  // [0] edge flags -> vertex ids, [1] triangles per tetrahedron -> face offsets (zero-padded)
  if ((rc = ensure(c, c->sdf_cnt, sizeof(int32_t) * 2 * (size_t)n_edges, st))) return rc;
  if ((rc = ensure(c, c->sdf_off, sizeof(int32_t) * 2 * (size_t)(n_edges + 1), st))) return rc;
  if ((rc = ensure(c, c->sdf_tmp, sizeof(int32_t) * 2 * scan_temp_ints((int)n_edges), st))) return rc;
  int32_t* cnt = (int32_t*)c->sdf_cnt.p;
  int32_t* off = (int32_t*)c->sdf_off.p;
  int32_t* d_tot = (int32_t*)c->status.p + 8;  // [8], [9]: vertex and face totals
  CUDA_TRY(c, cudaMemsetAsync(cnt + n_edges, 0, sizeof(int32_t) * (size_t)n_edges, st));
  launch_sdf_count(n, sdf, cnt, cnt + n_edges, st);
  ScanPair sp{};
  for (int q = 0; q < 2; ++q) {
    sp.in[q] = cnt + q * (size_t)n_edges;
    sp.out[q] = off + q * (size_t)(n_edges + 1);
    sp.sums[q] = (int32_t*)c->sdf_tmp.p + q * scan_temp_ints((int)n_edges);
  }
  sp.total = d_tot;
  sp.n = (int)n_edges;
  const int scan_launches = launch_scan_pair(sp, st);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(c->host_total, d_tot, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  counts[0] = c->host_total[0];
  counts[1] = c->host_total[1];
  if (counts[0] > max_verts || counts[1] > max_faces)
    return fail(c, MBR_ERR_ARG, "the mesh has %d vertices and %d faces; the outputs hold %d and %d", counts[0],
                counts[1], max_verts, max_faces);
  launch_sdf_write(n, sdf, lo, h, off, off + n_edges + 1, verts, vert_edges, faces, st);
  CUDA_TRY(c, cudaGetLastError());
  c->stats.launches += 3 + scan_launches;
  return MBR_OK;
}

int mbr_sdf_extract_backward(mbr_ctx* c, int32_t n, const float* sdf, float h, int32_t n_verts,
                             const int32_t* vert_edges, const float* dl_dverts, float* dl_dsdf, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  if (n < 1 || n > 512 || !sdf || !(h > 0.f) || n_verts < 0 || (n_verts > 0 && (!vert_edges || !dl_dverts)) ||
      !dl_dsdf)
    return fail(c, MBR_ERR_ARG, "bad SDF adjoint arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t m = (size_t)n + 1;
  CUDA_TRY(c, cudaMemsetAsync(dl_dsdf, 0, sizeof(float) * m * m * m, st));
  launch_sdf_grad(n, sdf, h, n_verts, vert_edges, dl_dverts, dl_dsdf, st);
  CUDA_TRY(c, cudaGetLastError());
  c->stats.launches += 1;
  return MBR_OK;
}

int mbr_measure_fp32_peak(mbr_ctx* c, int32_t iters, int32_t launches, double* flops, float* ms, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  if (iters < 1 || launches < 1 || !flops || !ms) return fail(c, MBR_ERR_ARG, "bad peak measurement arguments");
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if ((rc = ensure(c, c->cnt64, sizeof(float) * 8 * (size_t)c->num_sms * 32, st))) return rc;
  cudaEvent_t e0, e1;
  CUDA_TRY(c, cudaEventCreate(&e0));
  CUDA_TRY(c, cudaEventCreate(&e1));
  launch_fma_peak(c->num_sms, std::max(1, iters / 16), (float*)c->cnt64.p, st);  // warm-up
  double total = 0.0;
  cudaEventRecord(e0, st);
  for (int i = 0; i < launches; ++i) total += launch_fma_peak(c->num_sms, iters, (float*)c->cnt64.p, st);
  cudaEventRecord(e1, st);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(c, MBR_ERR_CUDA, "peak measurement: %s", cudaGetErrorString(e));
  *flops = total;
  *ms = t;
  return MBR_OK;
}

int mbr_debug_wait_limit(int32_t polls, int32_t stall, int32_t check_now) {
  if (polls < 0 || (stall && polls <= 0) || (stall && polls > (1 << 20))) return MBR_ERR_ARG;
  g_wait_polls.store(polls);
  g_wait_stall.store(stall ? 1 : 0);
  g_wait_check.store(check_now ? 1 : 0);
  return MBR_OK;
}

int mbr_set_state_budget(mbr_ctx* c, int64_t bytes) {
  if (!c) return MBR_ERR_ARG;
  if (bytes < 0) return fail(c, MBR_ERR_ARG, "the state budget must be >= 0 bytes");
  c->state_budget = bytes;
  c->last.valid = false;
  return MBR_OK;
}

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
  return backward_impl(c, mesh, motion, cam, T, H, W, solver, dl_dimage, dl_dverts, dl_dalbedo,
                       (cudaStream_t)stream, false);
}

int mbr_render_blur_backward_reuse(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion,
                                   const mbr_camera* cam, int32_t T, int32_t H, int32_t W, int32_t solver,
                                   const float* dl_dimage, float* dl_dverts, float* dl_dalbedo, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  return backward_impl(c, mesh, motion, cam, T, H, W, solver, dl_dimage, dl_dverts, dl_dalbedo,
                       (cudaStream_t)stream, true);
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

int mbr_count_work(mbr_ctx* c, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* cam, int32_t T,
                   int32_t H, int32_t W, int32_t solver, float* image, int64_t* out, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  cudaStream_t st = (cudaStream_t)stream;
  int rc = validate(c, mesh, motion, cam, T, H, W, solver);
  if (rc) return rc;
  if (!out) return fail(c, MBR_ERR_ARG, "null out");
  const int saved_tile = c->tile;
  c->tile = 16;  // the counting build exists for 16 x 16 tiles
  Prepared pp;
  rc = prepare(c, mesh, motion, cam, T, H, W, solver, st, true, pp);
  c->tile = saved_tile;
  if (rc) return rc;
  RasterParams P = raster_params(c, ctx_bufs(c), mesh, cam, T, H, W, pp);
  const size_t npix = (size_t)H * W;
  if (!image) {
    if ((rc = ensure(c, c->partial, sizeof(float4) * npix, st))) return rc;
    P.out = (float4*)c->partial.p;
  } else {
    P.out = (float4*)image;
  }
  if (pp.n_split > 1) CUDA_TRY(c, cudaMemsetAsync(P.out, 0, sizeof(float4) * npix, st));
  if ((rc = ensure(c, c->cnt64, sizeof(unsigned long long) * 8, st))) return rc;
  unsigned long long* d_cnt = (unsigned long long*)c->cnt64.p;
  CUDA_TRY(c, cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long) * 8, st));
  P.counts = d_cnt + 1;  // [1..6]
  const float r_count = (float)std::sqrt((double)cam->delta * std::log(1e12));
  launch_count((const TriRec*)c->recs.p, mesh->F, pp.d_groups, pp.G, W, H, r_count, d_cnt, st);
  launch_count((const TriRec*)c->recs.p, mesh->F, pp.d_groups, pp.G, W, H, 0.f, d_cnt + 7, st);  // N_box
  WorkQueue Q;
  if ((rc = upload_queue(c, &P, 1, st, Q))) return rc;
  const int kind = pp.moving ? 1 : 0;
  launch_raster_count(Q, pp.spt, kind,
                      std::max(1, std::min(persistent_grid_fwd(c->num_sms, 16, pp.spt, kind), Q.n_work)), st);
  CUDA_TRY(c, cudaGetLastError());
  c->stats.launches += 2;
  unsigned long long h[8];
  CUDA_TRY(c, cudaMemcpyAsync(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  for (int q = 0; q < 8; ++q) out[q] = (int64_t)h[q];
  return MBR_OK;
}

int mbr_autotune(mbr_ctx* c, int32_t n, const mbr_item* items, int32_t with_backward, int32_t* best_tile,
                 int32_t* best_spt, float* best_ms, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  if (n <= 0 || !items) return fail(c, MBR_ERR_ARG, "bad batch");
  cudaStream_t st = (cudaStream_t)stream;
  bool any_fast = false;
  for (int i = 0; i < n; ++i) any_fast |= items[i].solver == MBR_FAST;
  const int tiles[2] = {16, 8};
  const int spts_fast[3] = {1, 2, 4};
  const int n_spt = any_fast ? 3 : 1;
  const int saved_tile = c->tile, saved_spt = c->spt, saved_splits = c->splits;
  cudaEvent_t e0, e1;
  CUDA_TRY(c, cudaEventCreate(&e0));
  CUDA_TRY(c, cudaEventCreate(&e1));
  float best = INFINITY;
  int bt = saved_tile, bs = saved_spt, rc = MBR_OK;
  for (int ti = 0; ti < 2 && !rc; ++ti) {
    for (int si = 0; si < n_spt && !rc; ++si) {
      c->tile = tiles[ti];
      c->spt = any_fast ? spts_fast[si] : saved_spt;
      c->splits = saved_splits;
      // first call plans and captures; then time replays
      if ((rc = batch_run(c, n, items, with_backward, st))) break;
      float ms_min = INFINITY;
      for (int r = 0; r < 3 && !rc; ++r) {
        cudaEventRecord(e0, st);
        rc = batch_run(c, n, items, with_backward, st);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_min = std::min(ms_min, ms);
      }
      if (!rc && ms_min < best) {
        best = ms_min;
        bt = c->tile;
        bs = c->spt;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tile = rc ? saved_tile : bt;
  c->spt = rc ? saved_spt : bs;
  c->splits = saved_splits;
  if (rc) return rc;
  if (best_tile) *best_tile = bt;
  if (best_spt) *best_spt = bs;
  if (best_ms) *best_ms = best;
  return MBR_OK;
}

int mbr_render_blur_batch(mbr_ctx* c, int32_t n, const mbr_item* items, int32_t with_backward, void* stream) {
  if (!c) return MBR_ERR_ARG;
  c->err.clear();
  if (n < 0 || (n > 0 && !items)) return fail(c, MBR_ERR_ARG, "bad batch");
  if (n == 0) return MBR_OK;
  return batch_run(c, n, items, with_backward, (cudaStream_t)stream);
}

}  // extern "C"

namespace {

// ------------------------------------------------------------------ batched renders
// mbr_render_blur_batch: every item gets its own slice of one arena; the front halves of all items
// (normals, transform, setup, bin counts and scans) run first, one stream sync reads every bin
// total, the fills follow, then ONE persistent raster launch covers every item's work units
// (largest renders first), and the adjoint likewise.  The whole sequence is then captured in a
// CUDA graph: a later call with the same structure (sizes, solvers, buffers, tuning) only rewrites
// the pinned tables and replays the graph.  Replays bin into lists with 25% headroom; if a list
// would overflow (the geometry moved more), the call re-plans eagerly and recaptures.

struct BatchItem {
  Prepared pp;
  std::vector<SlotXform> xf;
  std::vector<int2> sets;
  std::vector<Group> groups;
  long long nb = 0;
  size_t o_status = 0, o_nacc = 0, o_pos = 0, o_nrm = 0, o_recs = 0, o_tab = 0, o_sets = 0, o_groups = 0;
  size_t tab_bytes = 0, o_order = 0, o_gslot = 0, o_galb = 0, o_gm = 0, o_bstate = 0;
  size_t o_counts = 0, o_offs[2] = {0, 0}, o_tmp[2] = {0, 0};
  size_t o_list[2] = {0, 0};
  int cap[2] = {0, 0};
  size_t stage_tab = 0;
};

struct BatchState {
  std::vector<long long> sig;
  std::vector<BatchItem> items;
  std::vector<int> order;  // item indices, largest render first
  DevBuf arena, lists, queue;
  void* stage = nullptr;
  size_t stage_cap = 0, stage_queue = 0, stage_off = 0, stage_status = 0, stage_bytes = 0;
  size_t arena_bytes = 0, list_bytes = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;  // private stream the graph is captured on (the caller's stream
                                   // may be the legacy default stream, which cannot be captured)
  int kind = 1;
  int grid_fwd = 1, grid_bwd = 1;  // persistent grids, fixed by the eager run (no queries in capture)
  bool with_backward = false;
};

void free_graph(BatchState* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  B->exec = nullptr;
}

void destroy_batch(mbr_ctx* c) {
  if (!c->batch) return;
  BatchState* B = c->batch;
  free_graph(B);
  if (B->capture) cudaStreamDestroy(B->capture);
  DevBuf* bufs[] = {&B->arena, &B->lists, &B->queue};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  if (B->stage) cudaFreeHost(B->stage);
  delete B;
  c->batch = nullptr;
}

long long fbits(float x) {
  int32_t i;
  std::memcpy(&i, &x, 4);
  return i;
}

std::vector<long long> batch_signature(mbr_ctx* c, int n, const mbr_item* items, int wb) {
  std::vector<long long> s = {n, wb, c->tile, c->spt, c->splits, c->state_budget};
  for (int i = 0; i < n; ++i) {
    const mbr_item& it = items[i];
    const long long vals[] = {it.mesh.V, it.mesh.F, it.T, it.H, it.W, it.solver,
                              it.solver == MBR_FAST ? num_segments(&it.motion) : 0, it.camera.time_rule,
                              fbits(it.camera.tan_half_fov), fbits(it.camera.znear), fbits(it.camera.delta),
                              (long long)(uintptr_t)it.mesh.verts, (long long)(uintptr_t)it.mesh.faces,
                              (long long)(uintptr_t)it.mesh.albedo, (long long)(uintptr_t)it.image,
                              (long long)(uintptr_t)it.dl_dimage, (long long)(uintptr_t)it.dl_dverts,
                              (long long)(uintptr_t)it.dl_dalbedo, (long long)(uintptr_t)it.mesh.dl_dtexture,
                              (long long)(uintptr_t)it.mesh.texture, it.mesh.tex_h, it.mesh.tex_w};
    s.insert(s.end(), std::begin(vals), std::end(vals));
  }
  return s;
}

size_t carve(size_t& at, size_t bytes) {
  const size_t o = (at + 255) & ~size_t(255);
  at = o + bytes;
  return o;
}

// host tables of every item into the pinned stage (called on every call: motion, camera change)
void batch_write_tables(mbr_ctx* c, const mbr_item* items, BatchState& B, bool rebuild_groups) {
  char* h = (char*)B.stage;
  for (size_t i = 0; i < B.items.size(); ++i) {
    BatchItem& I = B.items[i];
    const mbr_item& it = items[i];
    if (rebuild_groups) {
      Prepared pp = I.pp;
      build_tables(c, &it.motion, &it.camera, it.T, it.solver, I.xf, I.sets, I.groups, pp);
    }
    std::memcpy(h + I.stage_tab, I.xf.data(), sizeof(SlotXform) * I.xf.size());
    std::memcpy(h + I.stage_tab + (I.o_sets - I.o_tab), I.sets.data(), sizeof(int2) * I.sets.size());
    std::memcpy(h + I.stage_tab + (I.o_groups - I.o_tab), I.groups.data(), sizeof(Group) * I.groups.size());
  }
}

// Raster parameters of every item (queue order) into the pinned stage
void batch_write_params(mbr_ctx* c, const mbr_item* items, BatchState& B) {
  char* h = (char*)B.stage;
  char* A = (char*)B.arena.p;
  char* Lb = (char*)B.lists.p;
  RasterParams* par = (RasterParams*)(h + B.stage_queue);
  int32_t* off = (int32_t*)(h + B.stage_off);
  off[0] = 0;
  for (size_t k = 0; k < B.order.size(); ++k) {
    const int i = B.order[k];
    const BatchItem& I = B.items[i];
    const mbr_item& it = items[i];
    const RasterBufs bufs{A + I.o_recs, A + I.o_nrm, {A + I.o_offs[0], A + I.o_offs[1]},
                          {Lb + I.o_list[0], Lb + I.o_list[1]}};
    Prepared pp = I.pp;
    pp.d_groups = (Group*)(A + I.o_groups);
    carve_orders((int32_t*)(A + I.o_order), pp);
    pp.core_cap = I.cap[0];
    pp.soft_cap = I.cap[1];
    RasterParams P = raster_params(c, bufs, &it.mesh, &it.camera, it.T, it.H, it.W, pp);
    P.out = (float4*)it.image;
    P.fwd_cost = pp.d_fcost;  // the forward measures its per-unit work for the next replay's order
    if (B.with_backward) {  // the forward launch writes the per-sample state, the adjoint reads it
      P.dl_dimage = (const float4*)it.dl_dimage;
      P.g_slot = (float4*)(A + I.o_gslot);
      P.g_albedo = it.dl_dalbedo ? (float4*)(A + I.o_galb) : nullptr;
      if (it.mesh.texture) P.g_tex = it.mesh.dl_dtexture;
      if (pp.stored) {
        P.s_val = (float*)(A + I.o_bstate);
        P.s_stat = (uint8_t*)(A + I.o_bstate) + (size_t)it.T * it.H * it.W * 4;
      }
      P.unit_cost = pp.d_cost;
    }
    par[k] = P;
    off[k + 1] = off[k] + P.work;
  }
}

int batch_plan(mbr_ctx* c, int n, const mbr_item* items, int wb, cudaStream_t st, BatchState& B) {
  int rc;
  free_graph(&B);
  B.items.assign(n, BatchItem());
  B.with_backward = wb != 0;
  bool any_fast = false, any_plain = false, any_ext = false;
  size_t at = 0, stage_at = 0;
  for (int i = 0; i < n; ++i) {
    const mbr_item& it = items[i];
    if ((rc = validate(c, &it.mesh, &it.motion, &it.camera, it.T, it.H, it.W, it.solver))) return rc;
    if (!it.image) return fail(c, MBR_ERR_ARG, "item %d: null image", i);
    if (wb && (!it.dl_dimage || !it.dl_dverts)) return fail(c, MBR_ERR_ARG, "item %d: null gradient buffer", i);
    BatchItem& I = B.items[i];
    if ((rc = build_tables(c, &it.motion, &it.camera, it.T, it.solver, I.xf, I.sets, I.groups, I.pp))) return rc;
    Prepared& pp = I.pp;
    (it.solver == MBR_FAST ? any_fast : any_plain) = true;
    any_ext = any_ext || uses_variants(&it.mesh, &it.camera);
    const int V = it.mesh.V, F = it.mesh.F;
    pp.tiles_x = (it.W + c->tile - 1) / c->tile;
    pp.tiles_y = (it.H + c->tile - 1) / c->tile;
    pp.n_tiles = pp.tiles_x * pp.tiles_y;
    pp.r = (float)std::sqrt((double)it.camera.delta * (double)kSoftCutoff);
    pp.n_split = choose_splits(c, pp.G, patches_of(c->tile, pp.n_tiles));
    pp.n_units = patches_of(c->tile, pp.n_tiles) * pp.n_split;
    I.nb = (long long)pp.G * pp.n_tiles;
    if (I.nb > (1LL << 30)) return fail(c, MBR_ERR_ARG, "item %d: too many bins", i);
    I.o_status = carve(at, sizeof(int32_t) * 4);  // [0] status, [2], [3] list totals
    I.o_nacc = carve(at, sizeof(float) * 3 * V);
    I.o_pos = carve(at, sizeof(float4) * (size_t)pp.n_slots * V);
    I.o_nrm = carve(at, sizeof(float4) * (size_t)pp.n_slots * V);
    I.o_recs = carve(at, sizeof(TriRec) * (size_t)pp.n_sets * std::max(F, 1));
    I.o_tab = carve(at, sizeof(SlotXform) * I.xf.size());
    I.o_sets = carve(at, sizeof(int2) * I.sets.size());
    I.o_groups = carve(at, sizeof(Group) * I.groups.size());
    I.tab_bytes = I.o_groups + sizeof(Group) * I.groups.size() - I.o_tab;
    I.o_counts = carve(at, sizeof(int32_t) * 2 * (size_t)I.nb);  // core, soft counts (then cursors)
    for (int q = 0; q < 2; ++q) {
      I.o_offs[q] = carve(at, sizeof(int32_t) * (size_t)(I.nb + 1));
      I.o_tmp[q] = carve(at, sizeof(int32_t) * scan_temp_ints((int)I.nb));
    }
    I.o_order = carve(at, sizeof(int32_t) * order_buffer_ints(pp.n_units));
    if (wb) {
      I.o_gslot = carve(at, sizeof(float4) * 2 * (size_t)V * pp.n_slots);
      I.o_galb = carve(at, sizeof(float4) * V);
      I.o_gm = carve(at, sizeof(float) * 3 * V);
      pp.stored = keeps_state(c, it.T, it.H, it.W);
      if (pp.stored) I.o_bstate = carve(at, (size_t)it.T * it.H * it.W * 5);
    }
    I.stage_tab = carve(stage_at, I.tab_bytes);
  }
  B.kind = (any_fast && any_plain ? 2 : (any_fast ? 1 : 0)) | (any_ext ? kKindExt : 0);
  B.order.resize(n);
  for (int i = 0; i < n; ++i) B.order[i] = i;
  std::stable_sort(B.order.begin(), B.order.end(), [&](int a, int b) {
    const double ca = (double)items[a].H * items[a].W * items[a].T, cb = (double)items[b].H * items[b].W * items[b].T;
    return ca > cb;
  });
  B.stage_queue = carve(stage_at, sizeof(RasterParams) * n);
  B.stage_off = carve(stage_at, sizeof(int32_t) * (n + 1));
  B.stage_status = carve(stage_at, sizeof(int32_t) * 4 * n);
  B.stage_bytes = stage_at;
  B.arena_bytes = at;
  if ((rc = ensure(c, B.arena, at, st))) return rc;
  if ((rc = ensure(c, B.queue, B.stage_off - B.stage_queue + sizeof(int32_t) * (n + 1) + 512, st))) return rc;
  if (stage_at > B.stage_cap) {
    CUDA_TRY(c, cudaStreamSynchronize(st));
    if (B.stage) cudaFreeHost(B.stage);
    B.stage = nullptr;
    B.stage_cap = 0;
    if (cudaMallocHost(&B.stage, stage_at + stage_at / 4) != cudaSuccess)
      return fail(c, MBR_ERR_OOM, "cudaMallocHost(%zu) failed", stage_at);
    B.stage_cap = stage_at + stage_at / 4;
  }
  return MBR_OK;
}

// Issue the batch on st.  sizing: count bins, sync and size the lists (eager, not capturable);
// otherwise the lists keep the plan's capacities and the fills are bound-checked.
int batch_enqueue(mbr_ctx* c, const mbr_item* items, BatchState& B, cudaStream_t st, bool sizing) {
  int rc;
  char* A = (char*)B.arena.p;
  const int n = (int)B.items.size();
  for (int i = 0; i < n; ++i) {
    const BatchItem& I = B.items[i];
    CUDA_TRY(c, cudaMemcpyAsync(A + I.o_tab, (char*)B.stage + I.stage_tab, I.tab_bytes, cudaMemcpyHostToDevice, st));
  }
  for (int i = 0; i < n; ++i) {
    const BatchItem& I = B.items[i];
    const mbr_item& it = items[i];
    const Prepared& pp = I.pp;
    const int V = it.mesh.V, F = it.mesh.F;
    int* d_status = (int*)(A + I.o_status);
    CUDA_TRY(c, cudaMemsetAsync(d_status, 0, sizeof(int32_t), st));
    CUDA_TRY(c, cudaMemsetAsync(A + I.o_nacc, 0, sizeof(float) * 3 * V, st));
    launch_face_normals(it.mesh.verts, it.mesh.faces, F, V, (float*)(A + I.o_nacc), d_status, st);
    launch_xform(it.mesh.verts, (const float*)(A + I.o_nacc), V, (const SlotXform*)(A + I.o_tab), pp.n_slots,
                 it.camera.tan_half_fov, (float4*)(A + I.o_pos), (float4*)(A + I.o_nrm), st);
    launch_setup((const float4*)(A + I.o_pos), it.mesh.faces, F, V, (const int2*)(A + I.o_sets), pp.n_sets,
                 it.camera.znear, (TriRec*)(A + I.o_recs), st);
    BinTargets bt{};
    ScanPair sp{};
    CUDA_TRY(c, cudaMemsetAsync(A + I.o_counts, 0, sizeof(int32_t) * 2 * (size_t)I.nb, st));
    for (int q = 0; q < 2; ++q) {
      bt.counts_or_cursor[q] = (int32_t*)(A + I.o_counts) + q * (size_t)I.nb;
      sp.in[q] = bt.counts_or_cursor[q];
      sp.out[q] = (int32_t*)(A + I.o_offs[q]);
      sp.sums[q] = (int32_t*)(A + I.o_tmp[q]);
    }
    sp.total = d_status + 2;
    sp.n = (int)I.nb;
    launch_bin(false, (const TriRec*)(A + I.o_recs), F, (const Group*)(A + I.o_groups), pp.G, it.W, it.H, c->tile,
               c->tile, pp.tiles_x, pp.n_tiles, kCoreMargin, pp.r + kCoreMargin, bt, d_status, st);
    launch_scan_pair(sp, st);
    CUDA_TRY(c, cudaGetLastError());
  }
  int32_t* hs = (int32_t*)((char*)B.stage + B.stage_status);
  if (sizing) {
    // per item [0] status, [2], [3] list totals
    for (int i = 0; i < n; ++i)
      CUDA_TRY(c, cudaMemcpyAsync(hs + 4 * i, A + B.items[i].o_status, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost,
                                  st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    size_t lat = 0;
    for (int i = 0; i < n; ++i) {
      BatchItem& I = B.items[i];
      if (hs[4 * i] & kStatusBadFace) return fail(c, MBR_ERR_ARG, "item %d: face index outside [0, V)", i);
      for (int q = 0; q < 2; ++q) {
        const long long t = hs[4 * i + 2 + q];
        if (t < 0) return fail(c, MBR_ERR_DEVICE, "item %d: bin total overflow", i);
        I.cap[q] = (int)std::min<long long>(t + t / 4 + 4096, 0x7fffffffLL);  // headroom for replays
        I.o_list[q] = carve(lat, sizeof(int32_t) * (size_t)I.cap[q]);
      }
    }
    B.list_bytes = lat;
    if ((rc = ensure(c, B.lists, lat, st))) return rc;
    batch_write_params(c, items, B);  // now with the list slices and capacities
  }
  char* Lb = (char*)B.lists.p;
  for (int i = 0; i < n; ++i) {
    const BatchItem& I = B.items[i];
    const mbr_item& it = items[i];
    const Prepared& pp = I.pp;
    BinTargets bt{};
    for (int q = 0; q < 2; ++q) {
      bt.counts_or_cursor[q] = (int32_t*)(A + I.o_counts) + q * (size_t)I.nb;  // zeroed by the scan
      bt.list[q] = (int32_t*)(Lb + I.o_list[q]);
      bt.off[q] = (const int32_t*)(A + I.o_offs[q]);
      bt.cap[q] = I.cap[q];
    }
    launch_bin(true, (const TriRec*)(A + I.o_recs), it.mesh.F, (const Group*)(A + I.o_groups), pp.G, it.W, it.H,
               c->tile, c->tile, pp.tiles_x, pp.n_tiles, kCoreMargin, pp.r + kCoreMargin, bt, (int*)(A + I.o_status),
               st);
    Prepared po = pp;
    carve_orders((int32_t*)(A + I.o_order), po);
    // the sizing run orders the units by the bin estimate; the captured replays by the previous
    // run's measured forward cost (same plan, so the same unit layout)
    if (sizing)
      launch_unit_order((const int32_t*)(A + I.o_offs[0]), (const int32_t*)(A + I.o_offs[1]), pp.G, pp.n_tiles,
                        c->tile, pp.n_split, pp.n_units, po.d_order, po.d_order_tmp, po.d_cost, po.d_fcost, st);
    else
      launch_unit_order_measured(po.d_fcost, pp.n_units, po.d_order, po.d_order_tmp, po.d_fcost, po.d_cost, st);
    if (pp.n_split > 1) CUDA_TRY(c, cudaMemsetAsync(it.image, 0, sizeof(float4) * (size_t)it.H * it.W, st));
    if (B.with_backward) {
      CUDA_TRY(c, cudaMemsetAsync(A + I.o_gslot, 0, sizeof(float4) * 2 * (size_t)it.mesh.V * pp.n_slots, st));
      if (it.dl_dalbedo) CUDA_TRY(c, cudaMemsetAsync(A + I.o_galb, 0, sizeof(float4) * it.mesh.V, st));
      if (it.mesh.texture && it.mesh.dl_dtexture)
        CUDA_TRY(c, cudaMemsetAsync(it.mesh.dl_dtexture, 0, sizeof(float) * 3 * (size_t)it.mesh.tex_h * it.mesh.tex_w,
                                    st));
    }
  }
  CUDA_TRY(c, cudaGetLastError());
  // work queue: parameters (written to the stage by the caller) -> device, counter zeroed
  char* dq = (char*)B.queue.p;
  const size_t qbytes = B.stage_off - B.stage_queue + sizeof(int32_t) * (n + 1);
  const size_t cnt_at = (qbytes + 255) & ~size_t(255);
  CUDA_TRY(c, cudaMemcpyAsync(dq, (char*)B.stage + B.stage_queue, qbytes, cudaMemcpyHostToDevice, st));
  WorkQueue Q;
  Q.items = (const RasterParams*)dq;
  Q.item_off = (const int32_t*)(dq + (B.stage_off - B.stage_queue));
  Q.n_items = n;
  Q.n_work = ((int32_t*)((char*)B.stage + B.stage_off))[n];
  Q.counter = (int32_t*)(dq + cnt_at);
  Q.status = (int32_t*)(A + B.items[0].o_status);
  set_wait_fields(Q);
  const int spt = std::max(1, std::min(kMaxSpt, c->spt));
  if (sizing) {
    B.grid_fwd = std::max(1, std::min(persistent_grid_fwd(c->num_sms, c->tile, spt, B.kind), Q.n_work));
    B.grid_bwd = std::max(1, std::min(persistent_grid_bwd(c->num_sms, c->tile, spt, B.kind), Q.n_work));
  }
  CUDA_TRY(c, cudaMemsetAsync(Q.counter, 0, sizeof(int32_t), st));
  launch_raster_fwd(Q, c->tile, spt, B.kind, B.grid_fwd, st);
  CUDA_TRY(c, cudaGetLastError());
  c->stats.launches += 1;
  if (B.with_backward) {
    // the adjoint visits each item's units in the order of the forward's measured cost: the
    // order array the launches share is rewritten in place
    for (int i = 0; i < n; ++i) {
      Prepared po = B.items[i].pp;
      carve_orders((int32_t*)(A + B.items[i].o_order), po);
      launch_unit_order_measured(po.d_cost, po.n_units, po.d_order, po.d_order_tmp, nullptr, nullptr, st);
    }
    CUDA_TRY(c, cudaMemsetAsync(Q.counter, 0, sizeof(int32_t), st));
    launch_raster_bwd(Q, c->tile, spt, B.kind, B.grid_bwd, st);
    CUDA_TRY(c, cudaGetLastError());
    c->stats.launches += 3 * n + 1;
    for (int i = 0; i < n; ++i) {
      const BatchItem& I = B.items[i];
      const mbr_item& it = items[i];
      launch_slot_chain(it.mesh.verts, (const float*)(A + I.o_nacc), it.mesh.V, (const SlotXform*)(A + I.o_tab),
                        I.pp.n_slots, it.camera.tan_half_fov, (const float4*)(A + I.o_gslot),
                        (const float4*)(A + I.o_galb), it.dl_dverts, (float*)(A + I.o_gm), it.dl_dalbedo, st);
      launch_normals_bwd(it.mesh.verts, it.mesh.faces, it.mesh.F, it.mesh.V, (const float*)(A + I.o_gm),
                         it.dl_dverts, st);
    }
    CUDA_TRY(c, cudaGetLastError());
  }
  // statuses back to the stage (overflow detection after a replay)
  for (int i = 0; i < n; ++i)
    CUDA_TRY(c, cudaMemcpyAsync(hs + 4 * i + 1, A + B.items[i].o_status, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                st));
  return MBR_OK;
}

int batch_check(mbr_ctx* c, const BatchState& B) {
  const int32_t* hs = (const int32_t*)((char*)B.stage + B.stage_status);
  for (size_t i = 0; i < B.items.size(); ++i) {
    if (hs[4 * i + 1] & kStatusBadFace) return fail(c, MBR_ERR_ARG, "item %zu: face index outside [0, V)", i);
    if (hs[4 * i + 1] & kStatusSpin) return fail(c, MBR_ERR_TIMEOUT, "a raster launch gave up a bounded wait");
    if (hs[4 * i + 1] & kStatusBinOverflow) return -1;  // lists too small: re-plan
  }
  return MBR_OK;
}

int batch_run(mbr_ctx* c, int n, const mbr_item* items, int wb, cudaStream_t st) {
  int rc;
  if (!c->batch) c->batch = new (std::nothrow) BatchState();
  if (!c->batch) return fail(c, MBR_ERR_OOM, "batch state");
  BatchState& B = *c->batch;
  std::vector<long long> sig = batch_signature(c, n, items, wb);
  if (B.exec && sig == B.sig) {
    // replay: refresh the pinned tables and parameters, launch the graph, check for overflow
    batch_write_tables(c, items, B, true);
    batch_write_params(c, items, B);
    CUDA_TRY(c, cudaGraphLaunch(B.exec, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    rc = batch_check(c, B);
    if (rc == MBR_OK) return MBR_OK;
    if (rc != -1) return rc;
  }
  // plan, run eagerly (sizes the bin lists), then capture the same sequence for later calls
  if ((rc = batch_plan(c, n, items, wb, st, B))) return rc;
  batch_write_tables(c, items, B, false);
  if ((rc = batch_enqueue(c, items, B, st, true))) return rc;
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if ((rc = batch_check(c, B))) return rc == -1 ? fail(c, MBR_ERR_DEVICE, "bin lists overflowed") : rc;
  B.sig = sig;
  // capture for replays (same sequence, lists at their planned capacities) on the private stream
  if (!B.capture) CUDA_TRY(c, cudaStreamCreateWithFlags(&B.capture, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  CUDA_TRY(c, cudaStreamBeginCapture(B.capture, cudaStreamCaptureModeThreadLocal));
  rc = batch_enqueue(c, items, B, B.capture, false);
  cudaError_t ce = cudaStreamEndCapture(B.capture, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (ce != cudaSuccess) return fail(c, MBR_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
  ce = cudaGraphInstantiate(&B.exec, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) {
    B.exec = nullptr;
    return fail(c, MBR_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ce));
  }
  return MBR_OK;
}

}  // namespace

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
  const long long nb = (long long)pp.G * pp.n_tiles;
  if (nb > (1LL << 30)) return fail(c, MBR_ERR_ARG, "too many (group, tile) bins: %lld", nb);
  CUDA_TRY(c, cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev));
  pp.n_split = choose_splits(c, pp.G, patches_of(tw, pp.n_tiles));
  pp.n_units = patches_of(tw, pp.n_tiles) * pp.n_split;
  pp.r = (float)std::sqrt((double)cam->delta * (double)kSoftCutoff);

  // fixed part of the arena; the tables travel in one copy
  const size_t xf_b = sizeof(SlotXform) * xf.size(), sets_b = sizeof(int2) * sets.size(),
               g_b = sizeof(Group) * groups.size();
  const size_t off_sets = (xf_b + 255) & ~size_t(255), off_g = (off_sets + sets_b + 255) & ~size_t(255);
  const size_t tab_b = off_g + g_b;
  Arena A{(char*)base, kStaticScratchBytes, 0};
  // [0] this call's status, [1] raster waits (sticky until reported), [2], [3] list totals
  int* d_status = (int*)A.take(sizeof(int32_t) * 4);
  float* nacc = (float*)A.take(sizeof(float) * 3 * (size_t)V);
  float4* pos = (float4*)A.take(sizeof(float4) * (size_t)pp.n_slots * V);
  float4* nrm = (float4*)A.take(sizeof(float4) * (size_t)pp.n_slots * V);
  TriRec* recs = (TriRec*)A.take(sizeof(TriRec) * (size_t)pp.n_sets * std::max(F, 1));
  char* d_tab = (char*)A.take(tab_b);
  int32_t *offs[2] = {nullptr, nullptr}, *tmp[2] = {nullptr, nullptr}, *list[2];
  int32_t* counts = (int32_t*)A.take(sizeof(int32_t) * 2 * (size_t)nb);  // core, soft counts (then cursors)
  for (int q = 0; q < 2; ++q) {
    offs[q] = (int32_t*)A.take(sizeof(int32_t) * (size_t)(nb + 1));
    tmp[q] = (int32_t*)A.take(sizeof(int32_t) * scan_temp_ints((int)nb));
  }
  if (!d_status || !nacc || !pos || !nrm || !recs || !d_tab || !counts || !offs[1] || !tmp[1])
    return fail(c, MBR_ERR_ARG,
                "render needs more than the %zu MiB static scratch (V=%d F=%d T=%d %dx%d); use mbr_render_blur",
                kStaticScratchBytes >> 20, V, F, T, W, H);
  pp.d_xf = (SlotXform*)d_tab;
  const int2* d_sets = (const int2*)(d_tab + off_sets);
  pp.d_groups = (Group*)(d_tab + off_g);
  {
    std::vector<char> h(tab_b, 0);
    std::memcpy(h.data(), xf.data(), xf_b);
    std::memcpy(h.data() + off_sets, sets.data(), sets_b);
    std::memcpy(h.data() + off_g, groups.data(), g_b);
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    CUDA_TRY(c, cudaMemcpyAsync(d_tab, h.data(), tab_b, cudaMemcpyHostToDevice, st));
  }

  // the array keeps the previous call's contents: clear everything that accumulates (not [1])
  CUDA_TRY(c, cudaMemsetAsync(d_status, 0, sizeof(int32_t), st));
  CUDA_TRY(c, cudaMemsetAsync(nacc, 0, sizeof(float) * 3 * V, st));
  launch_face_normals(mesh->verts, mesh->faces, F, V, nacc, d_status, st);
  launch_xform(mesh->verts, nacc, V, pp.d_xf, pp.n_slots, cam->tan_half_fov, pos, nrm, st);
  launch_setup(pos, mesh->faces, F, V, d_sets, pp.n_sets, cam->znear, recs, st);
  int32_t status4[4] = {0, 0, 0, 0};  // pageable: the copy below is synchronised before it is read
  BinTargets bt{};
  ScanPair sp{};
  CUDA_TRY(c, cudaMemsetAsync(counts, 0, sizeof(int32_t) * 2 * (size_t)nb, st));
  for (int q = 0; q < 2; ++q) {
    bt.counts_or_cursor[q] = counts + q * (size_t)nb;
    sp.in[q] = bt.counts_or_cursor[q];
    sp.out[q] = offs[q];
    sp.sums[q] = tmp[q];
  }
  sp.total = d_status + 2;
  sp.n = (int)nb;
  launch_bin(false, recs, F, pp.d_groups, pp.G, W, H, tw, th, pp.tiles_x, pp.n_tiles, kCoreMargin, pp.r + kCoreMargin,
             bt, d_status, st);
  launch_scan_pair(sp, st);
  CUDA_TRY(c, cudaGetLastError());
  CUDA_TRY(c, cudaMemcpyAsync(status4, d_status, sizeof(status4), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(c, cudaStreamSynchronize(st));
  if (status4[0] & kStatusBadFace) return fail(c, MBR_ERR_ARG, "face index outside [0, V)");
  if (status4[1] & kStatusSpin) {
    CUDA_TRY(c, cudaMemsetAsync(d_status + 1, 0, sizeof(int32_t), st));
    return fail(c, MBR_ERR_TIMEOUT,
                "a raster launch of an earlier call gave up a bounded wait (its output is incomplete)");
  }
  const int32_t host[2] = {status4[2], status4[3]};
  for (int q = 0; q < 2; ++q) {
    list[q] = (int32_t*)A.take(sizeof(int32_t) * (size_t)std::max(host[q], 1));
    if (host[q] < 0 || !list[q])
      return fail(c, MBR_ERR_ARG, "tile lists (%d + %d entries) exceed the %zu MiB static scratch; use mbr_render_blur",
                  host[0], host[1], kStaticScratchBytes >> 20);
  }
  for (int q = 0; q < 2; ++q) {
    bt.list[q] = list[q];
    bt.off[q] = offs[q];
    bt.cap[q] = host[q];
  }
  launch_bin(true, recs, F, pp.d_groups, pp.G, W, H, tw, th, pp.tiles_x, pp.n_tiles, kCoreMargin, pp.r + kCoreMargin, bt,
             d_status, st);
  CUDA_TRY(c, cudaGetLastError());

  // unit order, then the raster into the caller's image (accumulated when the groups are split)
  pp.core_cap = host[0];
  pp.soft_cap = host[1];
  struct QueueHead {  // the raster's parameters, its work offsets and the queue counter, one copy
    RasterParams P;
    int32_t off[2];
    int32_t counter;
  };
  QueueHead* d_head = (QueueHead*)A.take(sizeof(QueueHead));
  pp.d_order = (int32_t*)A.take(sizeof(int32_t) * (pp.n_units + unit_order_ints(pp.n_units)));
  if (!d_head || !pp.d_order)
    return fail(c, MBR_ERR_ARG, "render needs more than the %zu MiB static scratch; use mbr_render_blur",
                kStaticScratchBytes >> 20);
  launch_unit_order(offs[0], offs[1], pp.G, pp.n_tiles, tw, pp.n_split, pp.n_units, pp.d_order,
                    pp.d_order + pp.n_units, nullptr, nullptr, st);
  const RasterBufs bufs{recs, nrm, {offs[0], offs[1]}, {list[0], list[1]}};
  QueueHead head;
  std::memset(&head, 0, sizeof(head));
  head.P = raster_params(c, bufs, mesh, cam, T, H, W, pp);
  head.P.out = (float4*)image;
  head.off[0] = 0;
  head.off[1] = head.P.work;
  head.counter = 0;
  if (pp.n_split > 1) CUDA_TRY(c, cudaMemsetAsync(image, 0, sizeof(float4) * (size_t)H * W, st));
  // the stream is idle after the binning sync, so this pageable copy does not wait
  CUDA_TRY(c, cudaMemcpyAsync(d_head, &head, sizeof(head), cudaMemcpyHostToDevice, st));
  WorkQueue Q;
  Q.items = &d_head->P;
  Q.item_off = d_head->off;
  Q.n_items = 1;
  Q.n_work = head.P.work;
  Q.counter = &d_head->counter;
  Q.status = d_status + 1;  // sticky: reported by the next call's binning sync
  set_wait_fields(Q);
  const int kind = raster_kind(pp, mesh, cam);
  const int grid = std::max(1, std::min(persistent_grid_fwd(c->num_sms, tw, pp.spt, kind), Q.n_work));
  launch_raster_fwd(Q, tw, pp.spt, kind, grid, st);
  CUDA_TRY(c, cudaGetLastError());
  return check_waits_now(c, Q.status, st);
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
