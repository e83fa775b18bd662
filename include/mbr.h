/*
 * mbr.h -- C ABI of the GB300 (sm_103a) motion-blurred differentiable mesh renderer.
 *
 * Operation (paper: "Recovering 3D Shapes from Ultra-Fast Motion-Blurred Images",
 * arXiv 2602.07860): a triangle mesh moves rigidly over one exposure (Sec. "Motion Parameters":
 * translation, or rotation about an axis through the origin).  At T sub-frame times
 * t_k = k/(T-1) (Sec. 3.2) every pixel centre p = [u, v, 1] gets barycentric coordinates
 * w = F(t)^-1 p for the triangles near it (Eq. barycentric), the nearest covering triangle wins
 * the z-test (Sec. 3.1), its interpolated colour and normal are shaded (Eq. fore, Lambert), and
 * uncovered samples get the soft coverage alpha 1 - prod_j (1 - exp(-d_j/delta))
 * (Eqs. probability-function, back).  The T sub-frames are averaged into one RGBA image
 * (Sec. 3.3).  Two solvers compute the sub-frame barycentrics:
 *   MBR_PLAIN -- per sub-frame: exact motion and projection at every t_k, F(t_k)^-1 p per sample;
 *   MBR_FAST  -- the paper's fast solver (Sec. 3.2, Eq. time-dependent2): motion split into S
 *                linear segments; per (pixel, triangle, segment) the quadratic-rational
 *                coefficients are formed once and w(tau) is evaluated per sample; background
 *                distances use keyframe F(X) (Eqs. euc-dist-approx-2/3).
 *
 * Conventions
 *   - NDC: pixel (i, j) has centre u = 2(i+0.5)/W - 1, v = 1 - 2(j+0.5)/H (row 0 at the top);
 *     projection x = x_c / (z_c tan_half_fov), y = y_c / (z_c tan_half_fov) (Sec. "Camera").
 *   - Images are [H, W, 4] float32 RGBA, row-major, device memory.
 *   - All pointers in mbr_mesh and all image / gradient buffers are DEVICE pointers owned by the
 *     caller; the library never frees them.  The context owns its scratch (vertex states,
 *     triangle records, tile bins, gradient slots), grows it on demand and frees it in
 *     mbr_destroy.
 *   - Every call is enqueued on the caller's CUDA stream (cudaStream_t passed as void*; NULL =
 *     legacy default stream).  mbr_render_blur and mbr_render_blur_backward synchronise that
 *     stream once, after binning, to size the tile lists.
 *   - Errors: every call returns MBR_OK (0) or an MBR_ERR_* code and never aborts; the message
 *     of the last failure is returned by mbr_last_error.  A context is used by one host thread
 *     at a time.
 */
#ifndef MBR_H
#define MBR_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MBR_OK 0
#define MBR_ERR_ARG 1     /* invalid argument (null pointer, bad size, unsupported value)      */
#define MBR_ERR_CUDA 2    /* a CUDA runtime call failed                                        */
#define MBR_ERR_OOM 3     /* device allocation failed                                          */
#define MBR_ERR_TIMEOUT 4 /* a bounded device-side wait of the raster gave up (output incomplete) */
#define MBR_ERR_DEVICE 5  /* a kernel reported an error through the device status word        */

#define MBR_PLAIN 0
#define MBR_FAST 1

#define MBR_TRANSLATE 0
#define MBR_ROTATE 1
#define MBR_PARABOLIC 2

#define MBR_TIME_PAPER 0    /* t_k = k/(T-1), T = 1 -> 0.5 (Sec. 3.2)  */
#define MBR_TIME_MIDPOINT 1 /* t_k = (k + 0.5)/T                        */
/* soft-coverage probability of a background pixel at squared distance d from a triangle */
#define MBR_PROB_EXP 0      /* A = exp(-d/delta), the paper's choice (App. "Implementation Details") */
#define MBR_PROB_SIGMOID 1  /* A = sigmoid(-d/delta), the original SoftRas map the appendix replaces */
/* attribute (albedo, normal) interpolation of a covered sample */
#define MBR_INTERP_SCREEN 0       /* screen-space barycentrics w (Eq. fore)                          */
#define MBR_INTERP_PERSPECTIVE 1  /* perspective-correct (w_i / z_i) / sum_j (w_j / z_j), z camera depth */

typedef struct mbr_ctx mbr_ctx;

/* Triangle mesh (device pointers).  The vertex attribute c_i of Eq. fore is the per-vertex
 * colour, or, when texture is set, a texture coordinate: the colour of a covered sample is then
 * the texture sampled bilinearly (clamp to edge, texel centres at (k + 0.5) / size) at the
 * interpolated (u, v); u runs along the texture's width, v along its rows. */
typedef struct {
  int32_t V, F;
  const float* verts;    /* [V,3] base vertex positions, world units                    */
  const int32_t* faces;  /* [F,3] vertex indices in [0, V)                               */
  const float* albedo;   /* [V,3] per-vertex colour (unused when textured)              */
  const float* uv;       /* [V,2] texture coordinates (required when textured), or null */
  const float* texture;  /* [tex_h, tex_w, 3] RGB texels, or null (per-vertex colour)   */
  int32_t tex_h, tex_w;
  float* dl_dtexture;    /* adjoint only: [tex_h, tex_w, 3] texel gradients, overwritten; or null */
} mbr_mesh;

/* Rigid motion over the exposure, t in [0, 1] (Sec. "Motion Parameters"). */
typedef struct {
  int32_t kind;     /* MBR_TRANSLATE: P(t) = v + offset + t dir
                       MBR_ROTATE:    P(t) = R(omega t) v, right-handed about unit(axis)
                       MBR_PARABOLIC: P(t) = R(omega t) v + offset + t dir + t^2 acc, the
                                      combined rotation and parabolic translation of the
                                      appendix's parabolic recovery (there: omega = pi about
                                      +y, offset (0.5, -0.5, 0.5), dir (-1, 4, -1),
                                      acc (0, -4, 0))                                      */
  int32_t segments; /* fast solver's linear segments; 0 = 1 (translation) or
                       ceil(12 |omega| / 2 pi), at least 1 (rotation and parabolic; 12 per
                       turn, Sec. 3.3)                                                     */
  float offset[3], dir[3], axis[3], omega;
  float acc[3];     /* MBR_PARABOLIC only: quadratic term of the translation              */
} mbr_motion;

/* Camera, shading and soft-coverage parameters. */
typedef struct {
  float view[12];       /* 3x4 world->camera matrix, camera +z forward                        */
  float tan_half_fov;   /* tan of half the field of view                                      */
  float znear;          /* triangles with a vertex at camera z <= znear are skipped           */
  float light_dir[3];   /* direction towards the light, world space (normalised internally)  */
  float k_ambient, k_diffuse; /* I = c (k_ambient + k_diffuse max(0, n.l))                   */
  float delta;          /* soft-coverage temperature of Eq. probability-function (1e-4)      */
  int32_t time_rule;    /* MBR_TIME_PAPER or MBR_TIME_MIDPOINT                                */
  int32_t prob;         /* MBR_PROB_EXP or MBR_PROB_SIGMOID                                   */
  int32_t interp;       /* MBR_INTERP_SCREEN or MBR_INTERP_PERSPECTIVE                        */
} mbr_camera;

/* One render of a batch (device pointers; see mbr_render_blur_batch). */
typedef struct {
  mbr_mesh mesh;
  mbr_motion motion;
  mbr_camera camera;
  int32_t T, H, W, solver;
  float* image;            /* [H,W,4] out                                               */
  const float* dl_dimage;  /* [H,W,4] in, read when with_backward                       */
  float* dl_dverts;        /* [V,3] out (overwritten) when with_backward                */
  float* dl_dalbedo;       /* [V,3] out (overwritten) when with_backward, may be NULL   */
} mbr_item;

/* Create / destroy a context on the current CUDA device.  Returns MBR_OK or MBR_ERR_*. */
int mbr_create(mbr_ctx** out);
void mbr_destroy(mbr_ctx* ctx);

/* Forward render (Secs. 3.1-3.3).  T >= 1, H, W >= 1, V >= 1, F >= 0.  image [H,W,4] is
 * overwritten with the blurred RGBA.  MBR_ERR_ARG on invalid sizes / null pointers. */
int mbr_render_blur(mbr_ctx* ctx, const mbr_mesh* mesh, const mbr_motion* motion,
                    const mbr_camera* camera, int32_t T, int32_t H, int32_t W, int32_t solver,
                    float* image, void* cuda_stream);

/* Adjoint of mbr_render_blur ("Gradient Computation", Sec. 3.3): given dL/dimage [H,W,4],
 * writes dL/dverts [V,3] (overwritten) and, if non-NULL, dL/dalbedo [V,3] (and, for a textured
 * mesh with dl_dtexture set, the texel gradients).  It runs the forward raster first (into
 * context scratch), which leaves per sample the winner face, or the log soft product and the
 * count of vanishing factors; the adjoint kernel reads that and recomputes every sub-frame
 * quantity it differentiates (barycentrics, depths, distances, closest points, shading).
 * Discrete choices (coverage, z-test winner, closest-point region, Lambert clamp) carry no
 * gradient.  It is the derivative of the single-precision image the forward computes: soft
 * factors with exp(-d/delta) <= 2^-25, which leave that image unchanged, contribute nothing. */
int mbr_render_blur_backward(mbr_ctx* ctx, const mbr_mesh* mesh, const mbr_motion* motion,
                             const mbr_camera* camera, int32_t T, int32_t H, int32_t W,
                             int32_t solver, const float* dl_dimage, float* dl_dverts,
                             float* dl_dalbedo, void* cuda_stream);

/* The adjoint of the immediately preceding mbr_render_blur on the same context: like
 * mbr_render_blur_backward (same arguments, same results), but when no other call has used the
 * context since that forward and every argument equals the forward's (the same mesh pointers and
 * sizes, motion, camera, T, H, W, solver and tuning), the forward's front half -- vertex states,
 * triangle records, tile bins, unit costs -- and its per-sample raster state are reused, which
 * saves the front half, its stream synchronisation and the forward raster.  Otherwise it runs
 * them, exactly as mbr_render_blur_backward.  The CALLER guarantees that the contents of verts, faces and albedo
 * have not changed since the forward (the library compares pointers, not contents); PyTorch's
 * saved-tensor version check gives that guarantee to the autograd path. */
int mbr_render_blur_backward_reuse(mbr_ctx* ctx, const mbr_mesh* mesh, const mbr_motion* motion,
                                   const mbr_camera* camera, int32_t T, int32_t H, int32_t W, int32_t solver,
                                   const float* dl_dimage, float* dl_dverts, float* dl_dalbedo,
                                   void* cuda_stream);

/* Render n independent items (objects, motions, solvers, sub-frame counts and resolutions may
 * differ), forward and, if with_backward != 0, the adjoint too.  The front halves of all items run
 * first, one stream sync sizes every item's tile lists, then a single persistent raster launch
 * covers every item's work (largest renders first), and likewise for the adjoint.  The sequence
 * is captured in a CUDA graph owned by the context: a later call with the same structure (item
 * count, sizes, solvers, segment counts, device buffers, camera fov/znear/delta and tuning) only
 * refreshes the motion/camera tables and replays the graph.  Replays bin into lists with 25%
 * headroom; if geometry changed enough to overflow them, the call re-plans and recaptures by
 * itself.  The call synchronises its stream before returning.  Motivated by the paper's
 * optimisation loops that render many views per iteration (Sec. 5); the batching itself is a
 * design of this library. */
int mbr_render_blur_batch(mbr_ctx* ctx, int32_t n, const mbr_item* items, int32_t with_backward,
                          void* cuda_stream);

/* Autotuner: times mbr_render_blur_batch on these items for every candidate tile shape (16x16,
 * 8x8 pixels) and, when a fast-solver item is present, sub-frames per group (1, 2, 4), keeps
 * the fastest on the context (as mbr_set_tuning would) and reports it.  Any out pointer may be
 * NULL.  The items are rendered several times (their outputs are overwritten). */
int mbr_autotune(mbr_ctx* ctx, int32_t n, const mbr_item* items, int32_t with_backward,
                 int32_t* best_tile, int32_t* best_spt, float* best_ms, void* cuda_stream);

/* Test hook: the z-test winner (face id, -1 = background) of every pixel at sub-frame k,
 * written to ids [H,W] (device).  Same arguments as mbr_render_blur otherwise. */
int mbr_debug_winners(mbr_ctx* ctx, const mbr_mesh* mesh, const mbr_motion* motion,
                      const mbr_camera* camera, int32_t T, int32_t H, int32_t W, int32_t solver,
                      int32_t k, int32_t* ids, void* cuda_stream);

/* Measurement hook: count N_cand, the (pixel, sub-frame, triangle) triples whose triangle's
 * bounding box at that sub-frame, dilated by sqrt(delta ln 1e12), contains the pixel centre
 * (plain solver: exact positions; fast solver: keyframe-lerped positions).  *out is a HOST
 * int64; the call synchronises the stream. */
int mbr_count_candidates(mbr_ctx* ctx, const mbr_mesh* mesh, const mbr_motion* motion,
                         const mbr_camera* camera, int32_t T, int32_t H, int32_t W,
                         int32_t solver, int64_t* out, void* cuda_stream);

/* Measurement hook: the units of the raster's work model for one forward render, counted by the
 * GPU path's own (FP32) decisions.  out[0] = N_cand (as mbr_count_candidates); out[1] = N_soft,
 * the soft-coverage factors 1 - exp(-d/delta) of uncovered samples that enter the products of
 * Eqs. probability-function .. back (those with exp(-d/delta) > 2^-25; smaller ones leave the
 * single-precision product unchanged); out[2] = covered samples.  Efficiency of the raster's
 * passes: out[3] = soft distance evaluations (per pixel and sample), out[4] = warp steps over
 * live soft candidates, out[5] = coverage tests (per pixel and sample), out[6] = warp steps over
 * live coverage candidates; out[7] = N_box, the triples whose undilated bounding box contains
 * the pixel centre (the coverage tests a binned rasteriser cannot avoid).  It runs the forward raster in its counting build
 * (16 x 16 tiles, slower than mbr_render_blur) and, if image is not NULL, writes the image as
 * mbr_render_blur does.  out is a HOST int64[8]; the call synchronises the stream.  Errors as
 * mbr_render_blur. */
int mbr_count_work(mbr_ctx* ctx, const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* camera,
                   int32_t T, int32_t H, int32_t W, int32_t solver, float* image, int64_t* out,
                   void* cuda_stream);

/* Memory of the adjoint ("Gradient Computation", Sec. 3.3).  The forward raster can keep, per
 * pixel and sub-frame, its discrete outcome -- the winner face of a covered sample, else the log
 * soft product and the count of vanishing factors -- 5 bytes, so that the adjoint does not repeat
 * its coverage and soft-product passes.  It keeps them only while T x H x W x 5 bytes <= bytes
 * (default 2^30); above that, the adjoint recomputes them per sample group from the geometry and
 * no storage grows with T.  bytes = 0: always recompute.  Applies to every following render and
 * batch on ctx; MBR_ERR_ARG for a negative value. */
int mbr_set_state_budget(mbr_ctx* ctx, int64_t bytes);

/* Tuning knobs (autotuner): tile edge in pixels (8 or 16), sub-frames per thread for the fast
 * solver (1..4, default 2), and the number of sub-frame group splits of the raster work units
 * (0 = automatic: about 64 units per SM). */
int mbr_set_tuning(mbr_ctx* ctx, int32_t tile, int32_t spt, int32_t splits);

/* Measurement counters of a context. */
typedef struct {
  int64_t launches;          /* kernels this context has launched (cumulative)                 */
  int64_t bin_entries;       /* (group, tile, face) entries of the last binning                */
  double raster_fwd_ms;      /* summed duration of the timed forward raster launches          */
  double raster_bwd_ms;      /* summed duration of the timed adjoint raster launches          */
  int64_t raster_fwd_count;  /* forward raster launches timed since profiling was switched on  */
  int64_t raster_bwd_count;  /* adjoint raster launches timed                                  */
  int32_t n_split;           /* sub-frame group splits of the last raster launch                */
  int32_t groups;            /* sample groups of the last call                                   */
  int64_t reused;            /* adjoint calls that reused the forward's front half (cumulative)  */
} mbr_stats;

/* Switch CUDA-event timing of the raster kernels on (1, and reset the sums) or off (0).  Events
 * are recorded on the caller's stream around each raster launch without synchronising; their
 * durations are collected at the next call's existing binning sync or by mbr_get_stats (which
 * waits for the last recorded event). */
int mbr_set_profiling(mbr_ctx* ctx, int32_t on);
int mbr_get_stats(mbr_ctx* ctx, mbr_stats* out);

/* Forward render like mbr_render_blur, for callers that cannot allocate device memory: a process
 * that hands all of the GPU's memory to its own pool or to a fixed budget at start-up, or a
 * latency-sensitive loop that cannot take the device-wide synchronisation a cudaMalloc/cudaFree
 * may bring.  The paper has no counterpart; this is a deployment option of this library.
 *
 * It needs no context.  All scratch comes from one statically sized array of 32 MiB that every
 * GPU loading this library holds until the process exits; nothing is allocated or freed (no
 * cudaMalloc, cudaFree or allocating library call).  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before any stream capture.
 * Renders whose scratch would not fit (large meshes, many sub-frames or segments, large images)
 * return MBR_ERR_ARG with a message naming the limit; use mbr_render_blur for those.
 * All calls on a device share the array, which keeps the last call's contents (the call clears
 * what it accumulates): calls whose work overlaps on the GPU -- different streams or threads
 * without ordering between them -- race.  Host <-> device traffic: one copy of the motion and
 * camera tables from pageable host memory at the start (it may wait for work already queued on
 * the stream), one stream synchronisation after binning (it reads the tile-list sizes), then one
 * copy of the raster's parameters into the idle stream.  The raster itself is not waited for: if
 * one of its bounded device-side waits gave up (the image is then incomplete), the NEXT call on
 * this device returns MBR_ERR_TIMEOUT and clears the report.  Arguments are those of
 * mbr_render_blur; err (may be NULL) receives the error message of a failed call, truncated to
 * err_len bytes including the terminating zero. */
int mbr_render_blur_noalloc(const mbr_mesh* mesh, const mbr_motion* motion, const mbr_camera* camera,
                            int32_t T, int32_t H, int32_t W, int32_t solver, float* image,
                            void* cuda_stream, char* err, int32_t err_len);

/* SDF -> triangle mesh (the rotational recovery of Sec. 5 optimises a signed distance field and
 * extracts the mesh it renders from it differentiably; the paper uses FlexiCubes, this library
 * marching tetrahedra).  sdf [(n+1)^3] DEVICE float samples at lo + h (i, j, k) (lo HOST [3]),
 * index (k (n+1) + j) (n+1) + i, 1 <= n <= 512; a sample is inside when s < 0.  Every grid cube is
 * split into the six tetrahedra corner 0 -> +e_a -> +e_a +e_b -> corner 7 (one per order of the
 * axes); every tetrahedron edge whose ends differ in sign carries one vertex at the zero of the
 * linear interpolant, p = p_a + t (p_b - p_a), t = s_a / (s_a - s_b), shared by the tetrahedra of
 * that grid edge.  A tetrahedron with one corner alone on its side gives one triangle, two and two
 * the quad on the crossing edges (a,c), (a,d), (b,d), (b,c) (a < b inside, c < d outside in
 * tetrahedron order) cut along (a,c)-(b,d); every face is wound so that its normal points outside
 * (s >= 0).  Writes the vertices [V,3] and faces [F,3] (DEVICE, caller-owned, capacities max_verts
 * and max_faces; V <= 7 (n+1)^3 and F <= 12 n^3 always hold), and if vert_edges is not NULL the grid
 * indices (a, b), a < b, of each vertex's edge [V,2] (needed by the adjoint).  counts (HOST [2])
 * receives V and F; if they exceed the capacities nothing is written and MBR_ERR_ARG is returned
 * with counts set.  The call synchronises its stream once (to read V and F). */
int mbr_sdf_extract(mbr_ctx* ctx, int32_t n, const float* sdf, const float lo[3], float h, int32_t max_verts,
                    int32_t max_faces, float* verts, int32_t* faces, int32_t* vert_edges, int32_t* counts,
                    void* cuda_stream);

/* Adjoint of mbr_sdf_extract's vertex positions w.r.t. the samples, the crossing topology held
 * fixed: dL/ds_a += dL/dt (-s_b) / (s_a - s_b)^2, dL/ds_b += dL/dt s_a / (s_a - s_b)^2 with
 * dL/dt = dL/dp . (p_b - p_a).  dl_dverts [n_verts,3] and vert_edges [n_verts,2] as returned by the
 * extraction of the same sdf; dl_dsdf [(n+1)^3] DEVICE is overwritten.  Stream-ordered. */
int mbr_sdf_extract_backward(mbr_ctx* ctx, int32_t n, const float* sdf, float h, int32_t n_verts,
                             const int32_t* vert_edges, const float* dl_dverts, float* dl_dsdf, void* cuda_stream);

/* Measurement hook: the FP32 CUDA-core peak of this GPU, measured.  Runs `launches` back-to-back
 * launches of a kernel that fills every SM with independent FMA chains (`iters` x 128 FMAs per
 * thread each), timed by CUDA events on the stream; *flops receives the FP32 operations executed
 * (an FMA counts 2), *ms the elapsed time.  flops / ms is the roofline denominator of the
 * renderer's ALU-bound kernels (the paper has no counterpart).  Synchronises the stream. */
int mbr_measure_fp32_peak(mbr_ctx* ctx, int32_t iters, int32_t launches, double* flops, float* ms,
                          void* cuda_stream);

/* Test hook for the raster's bounded waits (process-wide; applies to raster launches issued after
 * it, not to CUDA graphs captured before it).  The persistent raster CTAs hand work units to their
 * warps through shared-memory flags; every wait on such a flag polls at most `polls` times
 * (about 64 ns each; polls = 0 restores the default of 2^22, about 0.27 s), then sets the
 * kernel's status word, stops taking work and returns -- the kernel never hangs.  stall = 1 makes
 * the CTAs never publish a claimed unit, so every wait for a publication runs out after `polls`
 * polls (the flag that nothing sets); it needs 0 < polls <= 2^20.  check_now = 1 makes
 * mbr_render_blur, mbr_render_blur_backward(_reuse) and mbr_render_blur_noalloc synchronise their
 * stream after the raster and return MBR_ERR_TIMEOUT from the same call; otherwise a give-up is
 * reported by the next call on the same context (or device, for the no-alloc entry) at its
 * binning synchronisation, and mbr_render_blur_batch reports it from the same call.  Returns
 * MBR_ERR_ARG for invalid values. */
int mbr_debug_wait_limit(int32_t polls, int32_t stall, int32_t check_now);

/* Message of the last failed call on ctx ("" if none).  Valid until the next call. */
const char* mbr_last_error(mbr_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
