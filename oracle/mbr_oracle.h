/*
 * mbr_oracle.h -- FP64, single-threaded CPU oracle of the motion-blurred differentiable mesh
 * renderer in "Recovering 3D Shapes from Ultra-Fast Motion-Blurred Images" (arXiv 2602.07860).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or helper with the
 * CUDA path and includes nothing from it.
 *
 * The oracle evaluates the plain definitions: per sub-frame it places every vertex (exact motion,
 * or the keyframe lerp of Sec. 3.2), solves F(t) w = p by Gaussian elimination (Eq. barycentric),
 * z-tests the covering triangles (Sec. 3.1), shades the winner (Eq. fore + Lambert), and for
 * uncovered samples aggregates exp(-d/delta) soft coverage (Eqs. probability-function and back)
 * with d the exact squared distance (plain modes) or the keyframe approximation of
 * Eqs. euc-dist-approx-2/3 (fast mode).  Sub-frame results are averaged (Sec. 3.3).
 *
 * Parity unpinned: the paper's own images, gradients and timings (figures stripped).
 */
#ifndef MBR_ORACLE_H
#define MBR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t V, F;
  const double* verts;    /* [V,3] base vertex positions (world)                         */
  const int32_t* faces;   /* [F,3] vertex indices                                          */
  const double* albedo;   /* [V,3] per-vertex colour (unused when textured)               */
  const double* uv;       /* [V,2] texture coordinates, or NULL                            */
  const double* texture;  /* [tex_h, tex_w, 3] RGB texels, or NULL: when set, the vertex
                             attribute c_i of Eq. fore is uv_i and the sample colour is the
                             texture sampled bilinearly (clamp to edge, texel centres at
                             (k + 0.5) / size, u along the width, v along the rows)         */
  int32_t tex_h, tex_w;
  double* dl_dtexture;    /* orc_render_backward: [tex_h, tex_w, 3] texel gradients
                             (accumulated; the caller zeroes it), or NULL                   */
  int32_t motion_kind;    /* 0: P(t) = v + offset + t*dir ; 1: P(t) = R(omega*t, axis) v ;
                             2: P(t) = R(omega*t, axis) v + offset + t*dir + t^2*acc (the
                             rotation plus parabolic translation of the appendix's parabolic
                             recovery)                                                        */
  int32_t segments;       /* linear segments of the fast solver; 0 = default rule          */
  double offset[3], dir[3], axis[3], omega;
  double acc[3];          /* kind 2: quadratic translation term                             */
  double view[12];        /* 3x4 world->camera, camera +z forward                          */
  double tan_half_fov, znear;
  double light_dir[3];    /* direction towards the light, world space (normalised here)    */
  double k_ambient, k_diffuse, delta;
  int32_t time_rule;      /* 0: t_k = k/(T-1) (T=1: 0.5) ; 1: t_k = (k+0.5)/T             */
  int32_t prob;           /* soft-coverage probability of Eq. probability-function: 0 exp(-d/delta)
                             (the paper's), 1 sigmoid(-d/delta) (SoftRas's, App. "Implementation
                             Details")                                                        */
  int32_t interp;         /* attribute weights of a covered sample: 0 screen-space w (Eq. fore),
                             1 perspective-correct (w_i / z_i) / sum_j (w_j / z_j)             */
  int32_t T, H, W;
} orc_scene;

enum { ORC_PLAIN_EXACT = 0, ORC_PLAIN_LINEAR = 1, ORC_FAST_REF = 2 };
/* flags: ORC_SOFT_ALL no soft-coverage truncation, every triangle at every pixel; ORC_SOFT32 the
 * single-precision truncation instead of d <= delta ln 1e12: keep a factor only while
 * exp(-d/delta) > 2^-25, i.e. d < delta 25 ln 2 (below it 1 - A rounds to 1 in single precision,
 * so an FP32 product cannot see the factor; the adjoint of that product has no term for it) */
enum { ORC_SOFT_ALL = 1, ORC_SOFT32 = 2 };

/* counters[] written by orc_render / orc_render_backward */
enum {
  ORC_CNT_CAND = 0,       /* (pixel, sample, triangle) triples inside the dilated bbox            */
  ORC_CNT_COVERED = 1,    /* covered samples                                                      */
  ORC_CNT_AMBIG = 2,      /* samples flagged ambiguous for FP32 comparison                        */
  ORC_CNT_HASH = 3,       /* 64-bit hash of every discrete decision                               */
  ORC_CNT_SOFT = 4,       /* soft-coverage terms that entered a product                          */
  ORC_CNT_SOFT32 = 5,     /* of those, terms of uncovered samples with exp(-d/delta) > 2^-25: the
                             ones that can change a single-precision product (work measure)      */
  ORC_CNT_N = 8
};

int32_t orc_num_segments(const orc_scene* s);
/* sub-frame k -> time t, segment index and local time tau inside the segment */
void orc_sample_time(const orc_scene* s, int32_t k, int32_t* seg, double* t, double* tau);
/* area-weighted vertex normals of the base mesh, [V,3] */
void orc_vertex_normals(const orc_scene* s, double* normals);
/* exact per-vertex state at time t: [V,6] = ndc x, ndc y, camera z, world normal xyz */
void orc_vertex_state(const orc_scene* s, const double* normals, double t, double* state);
/* w = F^-1 p by Gaussian elimination with partial pivoting; returns det F */
double orc_barycentric(const double tri[6], double u, double v, double w[3]);
/* closest point of triangle tri (x0,y0,x1,y1,x2,y2) to (px,py) by the three clamped edge
 * projections of the appendix; returns the squared distance, its barycentrics in w[3] and a
 * region code (0..2: interior of edge (0,1), (1,2), (2,0); 3 + i: vertex i) */
double orc_closest_point(const double tri[6], double px, double py, double w[3], int32_t* region);

/* Render the window [x0, x0+w) x [y0, y0+h) of the H x W image.
 *   rgba     [h*w*4]   blurred RGBA, row-major, pixel (0,0) at the window's top-left
 *   winners  [T*h*w]   per-sample z-test winner (face id) or -1; may be NULL
 *   ambig    [T*h*w]   per-sample flags (bitmask) where FP32 may take another discrete choice:
 *                      1 coverage (pixel within 2e-6 of a triangle boundary), 2 depth tie,
 *                      4 near-degenerate triangle, 8 fast-mode closest-edge tie (these four can
 *                      change a pixel); 16 fast-mode closest-feature switch (edge interior vs
 *                      vertex, or a near tie), 32 Lambert clamp, 64 single-precision
 *                      conditioning eps32 Lmax^2/|det F| max(1,|w|) > 1e-4 of a term through
 *                      w = F^-1 p, 128 a textured sample within 2e-4 texels of a texel-centre
 *                      line (where the bilinear slope jumps) (these four only change
 *                      gradients); may be NULL
 *   counters [ORC_CNT_N]
 * returns 0, or -1 on bad arguments / allocation failure. */
int32_t orc_render(const orc_scene* s, int32_t mode, int32_t flags, int32_t x0, int32_t y0,
                   int32_t w, int32_t h, double* rgba, int32_t* winners, uint8_t* ambig,
                   int64_t* counters);

/* Reverse mode of orc_render over the same window: given dL/drgba [h*w*4], writes
 * dL/dverts [V,3] and (if non-NULL) dL/dalbedo [V,3].  Discrete choices (coverage, winner,
 * closest-point region, Lambert clamp, truncation) are held fixed. */
int32_t orc_render_backward(const orc_scene* s, int32_t mode, int32_t flags, int32_t x0,
                            int32_t y0, int32_t w, int32_t h, const double* dl_drgba,
                            double* dl_dverts, double* dl_dalbedo, int64_t* counters);

/* SDF -> triangle mesh extraction (rotational recovery, Sec. 5), marching tetrahedra on a regular
 * grid of n cells per axis; s [(n+1)^3] samples at lo + h (i, j, k), index (k (n+1) + j) (n+1) + i.
 * Writes up to max_verts vertices [V,3] in ascending order of their grid edge (a, b) (a < b,
 * vert_edges [V,2], may be NULL) and up to max_faces faces [F,3] facing the outside (s >= 0);
 * counts[0] = V, counts[1] = F.  Returns 0, 1 if the outputs are too small (counts still set),
 * -1 on bad arguments.  See sdf_oracle.c for the rules. */
int32_t orc_sdf_extract(int32_t n, const double* s, const double lo[3], double h, int64_t max_verts,
                        int64_t max_faces, double* verts, int64_t* vert_edges, int32_t* faces, int64_t* counts);
/* adjoint of the vertex positions w.r.t. the samples (topology held fixed): dl_ds [(n+1)^3]
 * accumulates (the caller zeroes it) */
int32_t orc_sdf_extract_backward(int32_t n, const double* s, const double lo[3], double h, int64_t n_verts,
                                 const int64_t* vert_edges, const double* dl_dverts, double* dl_ds);

#ifdef __cplusplus
}
#endif
#endif
