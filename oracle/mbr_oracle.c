/*
 * mbr_oracle.c -- FP64, single-threaded CPU oracle (TEST INFRASTRUCTURE ONLY; see mbr_oracle.h).
 *
 * Paper: "Recovering 3D Shapes from Ultra-Fast Motion-Blurred Images" (arXiv 2602.07860).
 * Each function names the passage it follows.  Readings of silent or ambiguous points:
 *   - sample times t_k = k/(T-1) (Sec. 3.2), T = 1 -> t = 0.5; optional midpoint rule (k+0.5)/T;
 *   - global sub-frame times are mapped to segment s = min(floor(t S), S-1) and local
 *     tau = t S - s (Sec. 3.3); S = 1 for translation, ceil(12 |omega| / 2 pi) for rotation;
 *   - "linear motion" (Sec. 3.2) lerps the projected keyframe x, y (and camera z, normals);
 *   - coverage is inclusive (all w_i >= 0); z-test keeps the largest sum_i w_i / z_i
 *     (perspective-correct inverse depth), ties to the smaller face id;
 *   - a triangle is skipped at a sample when |det F| <= 1e-10 or any vertex has camera
 *     z <= znear (exact modes: at t; keyframe modes: at either keyframe of the segment);
 *   - foreground samples have alpha 1 and Lambertian colour; background samples are black with
 *     alpha 1 - prod_j (1 - A_j) over triangles with d_j <= delta ln 1e12, A_j = exp(-d_j / delta)
 *     (the paper's map) or sigmoid(-d_j / delta) (the SoftRas map it replaces, App.
 *     "Implementation Details"); the sigmoid is below the exponential, so the truncation bound
 *     holds for both;
 *   - the closest point lies on the triangle (sum of weights 1), found by the appendix's three
 *     clamped edge projections; the fast mode searches F(X) (X = 0 if tau <= 0.5 else 1) around
 *     F(X) w(tau) and measures d at F(tau) w* (Eqs. euc-dist-approx-2/3).
 */
#include "mbr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define PI_D 3.14159265358979323846
#define D_MIN 1e-10        /* |det F| at or below this: triangle skipped (NDC^2)               */
#define ETA_COV 2e-6       /* ambiguity: pixel within this NDC distance of a triangle boundary   */
#define ETA_DEPTH 2e-5     /* ambiguity: relative inverse-depth gap of the two nearest surfaces   */
#define ETA_DET 1e-5       /* ambiguity: |det F| <= D_MIN + ETA_DET * (longest edge)^2          */
#define ETA_REGION 1e-6    /* ambiguity: fast-mode closest-edge tie (relative)                   */

enum { AMB_COVER = 1, AMB_DEPTH = 2, AMB_DEGEN = 4, AMB_REGION = 8, AMB_CLAMP = 16, AMB_LAMBERT = 32, AMB_COND = 64,
       AMB_TEXCELL = 128 };
/* gradient-only flag: single-precision conditioning.  The FP32 relative error of a gradient term
 * that passes through w = F^-1 p grows like eps32 (Lmax^2 / |det F|) max(1, |w|); flag when that
 * estimate exceeds 1e-4 (a tenth of the gradient tolerance). */
#define EPS32 5.96e-8
#define COND_LIMIT 1e-4
#define SOFT32_MIN 2.98023223876953125e-8  /* 2^-25: 1 - A rounds to 1 in single precision below */
#define ETA_CLAMP 1e-5     /* gradient-only flag: closest-feature switch within this relative d^2 */
#define ETA_LAMBERT 1e-5   /* gradient-only flag: |n.l| below this (Lambert clamp switches)     */
#define ETA_TEXCELL 2e-4   /* gradient-only flag: texel-space coordinate this near a texel centre line */

/* ------------------------------------------------------------------ small helpers */

static uint64_t fnv(uint64_t h, int64_t x) {
  for (int i = 0; i < 8; ++i) {
    h ^= (uint64_t)((x >> (8 * i)) & 0xff);
    h *= 1099511628211ULL;
  }
  return h;
}

/* Rodrigues rotation of v by angle theta about the unit vector along axis (right-handed). */
static void rotate_vec(const double axis[3], double theta, const double v[3], double out[3]) {
  double n = sqrt(axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2]);
  double k[3] = {axis[0] / n, axis[1] / n, axis[2] / n};
  double c = cos(theta), s = sin(theta);
  double kv = k[0] * v[0] + k[1] * v[1] + k[2] * v[2];
  double kx[3] = {k[1] * v[2] - k[2] * v[1], k[2] * v[0] - k[0] * v[2], k[0] * v[1] - k[1] * v[0]};
  for (int i = 0; i < 3; ++i) out[i] = v[i] * c + kx[i] * s + k[i] * kv * (1.0 - c);
}

/* Transposed rotation (inverse) -- used by the adjoint. */
static void rotate_vec_T(const double axis[3], double theta, const double v[3], double out[3]) {
  rotate_vec(axis, -theta, v, out);
}

/* ------------------------------------------------------------------ time map (Secs. 3.2, 3.3) */

int32_t orc_num_segments(const orc_scene* s) {
  if (s->segments > 0) return s->segments;
  if (s->motion_kind == 0) return 1; /* translation: one linear segment (visualisation details) */
  /* rotation: 12 segments per full turn (Sec. 3.3, segmentation analysis) */
  double x = 12.0 * fabs(s->omega) / (2.0 * PI_D);
  int32_t n = (int32_t)ceil(x - 1e-4); /* tolerance: omega = 2 pi rounded to float is 12 segments */
  return n < 1 ? 1 : n;
}

/* t_k as an exact fraction num/den */
static void time_fraction(const orc_scene* s, int32_t k, int64_t* num, int64_t* den) {
  if (s->time_rule == 1) {
    *num = 2 * (int64_t)k + 1;
    *den = 2 * (int64_t)s->T;
  } else if (s->T == 1) {
    *num = 1;
    *den = 2;
  } else {
    *num = k;
    *den = (int64_t)s->T - 1;
  }
}

void orc_sample_time(const orc_scene* s, int32_t k, int32_t* seg, double* t, double* tau) {
  int64_t S = orc_num_segments(s), num, den;
  time_fraction(s, k, &num, &den);
  int64_t g = (num * S) / den;
  if (g > S - 1) g = S - 1;
  *seg = (int32_t)g;
  *t = (double)num / (double)den;
  *tau = (double)(num * S - g * den) / (double)den;
}

/* keyframe X of Eq. euc-dist-approx-2: 0 if tau <= 0.5 else 1, decided on the exact fraction */
/* Bilinear texture sample at (u, v) (clamp to edge; texel centres at (k + 0.5) / size; u along
 * the width, v along the rows): colour c[3], the four taps (texel index, weight), dc/du and
 * dc/dv (zero across a clamped border), and the cell (x0, y0) for the decision hash. */
typedef struct { int64_t idx[4]; double wt[4]; int64_t cell; double edge; } tex_taps;  /* edge: distance of
  the texel-space coordinates to the nearest texel-centre line, where the bilinear slope jumps */

static void tex_sample(const orc_scene* s, double u, double v, double c[3], double dcdu[3], double dcdv[3],
                       tex_taps* t) {
  const int32_t w = s->tex_w, h = s->tex_h;
  double X = u * w - 0.5, Y = v * h - 0.5;
  X = fmin(fmax(X, -1.0), (double)w);
  Y = fmin(fmax(Y, -1.0), (double)h);
  const double x0f = floor(X), y0f = floor(Y), fx = X - x0f, fy = Y - y0f;
  const int64_t x0 = (int64_t)x0f, y0 = (int64_t)y0f;
  const int64_t xa = x0 < 0 ? 0 : (x0 > w - 1 ? w - 1 : x0), xb = x0 + 1 < 0 ? 0 : (x0 + 1 > w - 1 ? w - 1 : x0 + 1);
  const int64_t ya = y0 < 0 ? 0 : (y0 > h - 1 ? h - 1 : y0), yb = y0 + 1 < 0 ? 0 : (y0 + 1 > h - 1 ? h - 1 : y0 + 1);
  t->idx[0] = ya * w + xa; t->idx[1] = ya * w + xb; t->idx[2] = yb * w + xa; t->idx[3] = yb * w + xb;
  t->wt[0] = (1 - fx) * (1 - fy); t->wt[1] = fx * (1 - fy); t->wt[2] = (1 - fx) * fy; t->wt[3] = fx * fy;
  t->cell = (x0 + 2) * 100003 + (y0 + 2);
  t->edge = fmin(fabs(X - nearbyint(X)), fabs(Y - nearbyint(Y)));
  for (int k = 0; k < 3; ++k) {
    const double t00 = s->texture[3 * t->idx[0] + k], t10 = s->texture[3 * t->idx[1] + k];
    const double t01 = s->texture[3 * t->idx[2] + k], t11 = s->texture[3 * t->idx[3] + k];
    c[k] = t->wt[0] * t00 + t->wt[1] * t10 + t->wt[2] * t01 + t->wt[3] * t11;
    dcdu[k] = w * ((1 - fy) * (t10 - t00) + fy * (t11 - t01));
    dcdv[k] = h * ((1 - fx) * (t01 - t00) + fx * (t11 - t10));
  }
}

/* soft-coverage probability A (Eq. probability-function) of squared distance d, its factor
 * 1 - A (computed without cancellation) and dA/dd */
static double soft_prob(const orc_scene* s, double d, double* one_minus, double* dA_dd) {
  const double x = d / s->delta, e = exp(-x);
  if (s->prob == 1) {
    const double A = e / (1.0 + e);
    *one_minus = 1.0 / (1.0 + e);
    *dA_dd = -A * *one_minus / s->delta;
    return A;
  }
  *one_minus = -expm1(-x);
  *dA_dd = -e / s->delta;
  return e;
}

static int32_t sample_key_x(const orc_scene* s, int32_t k) {
  int64_t S = orc_num_segments(s), num, den;
  time_fraction(s, k, &num, &den);
  int64_t g = (num * S) / den;
  if (g > S - 1) g = S - 1;
  return 2 * (num * S - g * den) <= den ? 0 : 1;
}

/* ------------------------------------------------------------------ motion + camera */

/* Motion parameters (scene settings): translation v + offset + t dir; rotation R(omega t) v;
 * the parabolic recovery's motion: the vertex rotated by R(omega t), then translated by a
 * quadratic in t, offset + t dir + t^2 acc (the appendix writes it in s = 0.5 - t). */
static void place(const orc_scene* s, double t, const double p[3], double out[3]) {
  if (s->motion_kind == 0) {
    for (int i = 0; i < 3; ++i) out[i] = p[i] + s->offset[i] + t * s->dir[i];
  } else if (s->motion_kind == 1) {
    rotate_vec(s->axis, s->omega * t, p, out);
  } else {
    double r[3];
    if (s->omega != 0.0) rotate_vec(s->axis, s->omega * t, p, r);
    else { r[0] = p[0]; r[1] = p[1]; r[2] = p[2]; }
    for (int i = 0; i < 3; ++i) out[i] = r[i] + s->offset[i] + t * s->dir[i] + t * t * s->acc[i];
  }
}

static void orient(const orc_scene* s, double t, const double n[3], double out[3]) {
  if (s->motion_kind == 0 || (s->motion_kind == 2 && s->omega == 0.0)) {
    out[0] = n[0]; out[1] = n[1]; out[2] = n[2];
  } else {
    rotate_vec(s->axis, s->omega * t, n, out);
  }
}

/* Camera (scene settings): world -> camera by the 3x4 view matrix, then x_p = x / (z tan a). */
static void project(const orc_scene* s, const double P[3], double* x, double* y, double* z,
                    double cam[3]) {
  const double* m = s->view;
  double xc = m[0] * P[0] + m[1] * P[1] + m[2] * P[2] + m[3];
  double yc = m[4] * P[0] + m[5] * P[1] + m[6] * P[2] + m[7];
  double zc = m[8] * P[0] + m[9] * P[1] + m[10] * P[2] + m[11];
  *x = xc / (zc * s->tan_half_fov);
  *y = yc / (zc * s->tan_half_fov);
  *z = zc;
  if (cam) { cam[0] = xc; cam[1] = yc; cam[2] = zc; }
}

void orc_vertex_normals(const orc_scene* s, double* n) {
  memset(n, 0, sizeof(double) * 3 * (size_t)s->V);
  for (int32_t f = 0; f < s->F; ++f) {
    const int32_t* id = s->faces + 3 * f;
    const double *a = s->verts + 3 * id[0], *b = s->verts + 3 * id[1], *c = s->verts + 3 * id[2];
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                    e1[0] * e2[1] - e1[1] * e2[0]};
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) n[3 * id[j] + i] += cr[i];
  }
  for (int32_t v = 0; v < s->V; ++v) {
    double* p = n + 3 * v;
    double l = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
    if (l > 0) { p[0] /= l; p[1] /= l; p[2] /= l; }
  }
}

void orc_vertex_state(const orc_scene* s, const double* normals, double t, double* st) {
  for (int32_t v = 0; v < s->V; ++v) {
    double P[3], N[3];
    place(s, t, s->verts + 3 * v, P);
    project(s, P, st + 6 * v, st + 6 * v + 1, st + 6 * v + 2, NULL);
    orient(s, t, normals + 3 * v, N);
    st[6 * v + 3] = N[0]; st[6 * v + 4] = N[1]; st[6 * v + 5] = N[2];
  }
}

/* ------------------------------------------------------------------ linear algebra (Eq. barycentric) */

/* Solve A x = b (3x3) by Gaussian elimination with partial pivoting.  Returns 0 if singular. */
static int solve3(const double Ain[9], const double bin[3], double x[3]) {
  double A[3][4];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) A[r][c] = Ain[3 * r + c];
    A[r][3] = bin[r];
  }
  for (int c = 0; c < 3; ++c) {
    int piv = c;
    for (int r = c + 1; r < 3; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (A[piv][c] == 0.0) return 0;
    if (piv != c)
      for (int k = 0; k < 4; ++k) { double tmp = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = tmp; }
    for (int r = c + 1; r < 3; ++r) {
      double m = A[r][c] / A[c][c];
      for (int k = c; k < 4; ++k) A[r][k] -= m * A[c][k];
    }
  }
  for (int r = 2; r >= 0; --r) {
    double acc = A[r][3];
    for (int k = r + 1; k < 3; ++k) acc -= A[r][k] * x[k];
    x[r] = acc / A[r][r];
  }
  return 1;
}

static double det_tri(const double t[6]) {
  return (t[2] - t[0]) * (t[5] - t[1]) - (t[4] - t[0]) * (t[3] - t[1]);
}

double orc_barycentric(const double tri[6], double u, double v, double w[3]) {
  double F[9] = {tri[0], tri[2], tri[4], tri[1], tri[3], tri[5], 1.0, 1.0, 1.0};
  double p[3] = {u, v, 1.0};
  if (!solve3(F, p, w)) w[0] = w[1] = w[2] = NAN;
  return det_tri(tri);
}

/* y = F^-T g (used by the adjoint of w = F^-1 p) */
static void solve_transposed(const double tri[6], const double g[3], double y[3]) {
  double Ft[9] = {tri[0], tri[1], 1.0, tri[2], tri[3], 1.0, tri[4], tri[5], 1.0};
  if (!solve3(Ft, g, y)) y[0] = y[1] = y[2] = 0.0;
}

/* ------------------------------------------------------------------ closest point (appendix) */

typedef struct {
  double d2;      /* squared distance */
  double w[3];    /* barycentrics of the closest point */
  int32_t region; /* 0..2: interior of edge (0,1), (1,2), (2,0); 3 + i: vertex i */
  int32_t ei, ej; /* edge vertex slots */
  double t;       /* clamped edge parameter */
  double d2_second; /* second-best edge distance (for tie detection) */
  double w_second[3];
  double traw[3], d2e[3], L2e[3]; /* per edge: unclamped parameter, squared distance, length^2 */
} closest_t;

/* For each edge v_i v_j: t = ((p - v_i).(v_j - v_i)) / |v_j - v_i|^2 clamped to [0, 1]
 * (t < 0 -> v_i, t > 1 -> v_j); keep the edge point with the smallest distance. */
static void closest_point(const double tri[6], double px, double py, closest_t* out) {
  static const int E[3][2] = {{0, 1}, {1, 2}, {2, 0}};
  out->d2 = INFINITY;
  out->d2_second = INFINITY;
  for (int e = 0; e < 3; ++e) {
    int i = E[e][0], j = E[e][1];
    double xi = tri[2 * i], yi = tri[2 * i + 1], xj = tri[2 * j], yj = tri[2 * j + 1];
    double ex = xj - xi, ey = yj - yi, L2 = ex * ex + ey * ey;
    double t = L2 > 0 ? ((px - xi) * ex + (py - yi) * ey) / L2 : 0.0;
    out->traw[e] = t;
    out->L2e[e] = L2;
    int32_t reg = e;
    double qx, qy;
    if (t <= 0.0) { t = 0.0; qx = xi; qy = yi; reg = 3 + i; }
    else if (t >= 1.0) { t = 1.0; qx = xj; qy = yj; reg = 3 + j; }
    else { qx = xi + t * ex; qy = yi + t * ey; }
    double d2 = (px - qx) * (px - qx) + (py - qy) * (py - qy);
    out->d2e[e] = d2;
    double w[3] = {0, 0, 0};
    w[i] = 1.0 - t;
    w[j] = t;
    if (d2 < out->d2) {
      out->d2_second = out->d2;
      memcpy(out->w_second, out->w, sizeof(out->w));
      out->d2 = d2;
      memcpy(out->w, w, sizeof(w));
      out->region = reg;
      out->ei = i; out->ej = j; out->t = t;
    } else if (d2 < out->d2_second) {
      out->d2_second = d2;
      memcpy(out->w_second, w, sizeof(w));
    }
  }
}

double orc_closest_point(const double tri[6], double px, double py, double w[3], int32_t* region) {
  closest_t c;
  closest_point(tri, px, py, &c);
  if (w) { w[0] = c.w[0]; w[1] = c.w[1]; w[2] = c.w[2]; }
  if (region) *region = c.region;
  return c.d2;
}

/* ------------------------------------------------------------------ renderer */

typedef struct { int32_t p, f; double fval, dA, d; } soft_entry;  /* dA = dA/dd */

typedef struct {
  soft_entry* e;
  size_t n, cap;
} entry_list;

static int push_entry(entry_list* L, soft_entry x) {
  if (L->n == L->cap) {
    size_t nc = L->cap ? 2 * L->cap : 4096;
    soft_entry* ne = (soft_entry*)realloc(L->e, nc * sizeof(soft_entry));
    if (!ne) return 0;
    L->e = ne;
    L->cap = nc;
  }
  L->e[L->n++] = x;
  return 1;
}

/* state-gradient -> base vertex / base normal gradient at time t (projection, camera, motion) */
static void chain_state(const orc_scene* s, double t, const double* gst, double* gv, double* gn) {
  double th = s->tan_half_fov;
  const double* m = s->view;
  for (int32_t v = 0; v < s->V; ++v) {
    const double* g = gst + 6 * v;  /* x, y, nx, ny, nz, camera z */
    if (g[0] == 0 && g[1] == 0 && g[2] == 0 && g[3] == 0 && g[4] == 0 && g[5] == 0) continue;
    double P[3], cam[3], x, y, z;
    place(s, t, s->verts + 3 * v, P);
    project(s, P, &x, &y, &z, cam);
    double dxc = g[0] / (z * th), dyc = g[1] / (z * th);
    double dzc = g[5] - (g[0] * x + g[1] * y) / z;
    double dP[3];
    for (int i = 0; i < 3; ++i) dP[i] = m[i] * dxc + m[4 + i] * dyc + m[8 + i] * dzc;
    double dv[3], dn[3];
    if (s->motion_kind == 0 || (s->motion_kind == 2 && s->omega == 0.0)) {
      memcpy(dv, dP, sizeof(dP)); /* translations do not depend on v: d P / d v = identity */
      dn[0] = g[2]; dn[1] = g[3]; dn[2] = g[4];
    } else {
      rotate_vec_T(s->axis, s->omega * t, dP, dv);
      rotate_vec_T(s->axis, s->omega * t, g + 2, dn);
    }
    for (int i = 0; i < 3; ++i) { gv[3 * v + i] += dv[i]; gn[3 * v + i] += dn[i]; }
  }
}

/* adjoint of orc_vertex_normals: base-normal gradient -> vertex gradient */
static void normals_backward(const orc_scene* s, const double* gn, double* gv) {
  double* m = (double*)calloc(3 * (size_t)s->V, sizeof(double));
  double* gm = (double*)calloc(3 * (size_t)s->V, sizeof(double));
  if (!m || !gm) { free(m); free(gm); return; }
  for (int32_t f = 0; f < s->F; ++f) {
    const int32_t* id = s->faces + 3 * f;
    const double *a = s->verts + 3 * id[0], *b = s->verts + 3 * id[1], *c = s->verts + 3 * id[2];
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                    e1[0] * e2[1] - e1[1] * e2[0]};
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) m[3 * id[j] + i] += cr[i];
  }
  /* n = m / |m|  ->  dL/dm = (g - n (n.g)) / |m| */
  for (int32_t v = 0; v < s->V; ++v) {
    double* mv = m + 3 * v;
    double l = sqrt(mv[0] * mv[0] + mv[1] * mv[1] + mv[2] * mv[2]);
    if (l <= 0) continue;
    double n[3] = {mv[0] / l, mv[1] / l, mv[2] / l};
    const double* g = gn + 3 * v;
    double ng = n[0] * g[0] + n[1] * g[1] + n[2] * g[2];
    for (int i = 0; i < 3; ++i) gm[3 * v + i] = (g[i] - n[i] * ng) / l;
  }
  /* m_v += (b - a) x (c - a) for each face: dL/db = (c-a) x G, dL/dc = G x (b-a) */
  for (int32_t f = 0; f < s->F; ++f) {
    const int32_t* id = s->faces + 3 * f;
    const double *a = s->verts + 3 * id[0], *b = s->verts + 3 * id[1], *c = s->verts + 3 * id[2];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double w[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double G[3] = {0, 0, 0};
    for (int j = 0; j < 3; ++j)
      for (int i = 0; i < 3; ++i) G[i] += gm[3 * id[j] + i];
    double gb[3] = {w[1] * G[2] - w[2] * G[1], w[2] * G[0] - w[0] * G[2], w[0] * G[1] - w[1] * G[0]};
    double gc[3] = {G[1] * u[2] - G[2] * u[1], G[2] * u[0] - G[0] * u[2], G[0] * u[1] - G[1] * u[0]};
    for (int i = 0; i < 3; ++i) {
      gv[3 * id[1] + i] += gb[i];
      gv[3 * id[2] + i] += gc[i];
      gv[3 * id[0] + i] -= gb[i] + gc[i];
    }
  }
  free(m);
  free(gm);
}

static void lerp_state(const double* a, const double* b, double tau, double* out, size_t n) {
  for (size_t i = 0; i < n; ++i) out[i] = (1.0 - tau) * a[i] + tau * b[i];
}

static int render_impl(const orc_scene* s, int32_t mode, int32_t flags, int32_t x0, int32_t y0,
                       int32_t w, int32_t h, double* rgba, int32_t* winners, uint8_t* ambig,
                       int64_t* cnt, const double* dl, double* gverts, double* galb) {
  if (!s || s->V <= 0 || s->F < 0 || s->T <= 0 || s->H <= 0 || s->W <= 0 || w < 0 || h < 0 ||
      x0 < 0 || y0 < 0 || x0 + w > s->W || y0 + h > s->H || mode < 0 || mode > 2 ||
      (s->texture && (!s->uv || s->tex_h < 1 || s->tex_w < 1)))
    return -1;
  const int32_t V = s->V, F = s->F, T = s->T, S = orc_num_segments(s);
  const size_t npix = (size_t)w * (size_t)h;
  const double r2 = (flags & ORC_SOFT32) ? s->delta * 25.0 * log(2.0) : s->delta * log(1e12), r = sqrt(r2);
  const int soft_all = (flags & ORC_SOFT_ALL) != 0;
  const int backward = dl != NULL;
  double Ld[3] = {s->light_dir[0], s->light_dir[1], s->light_dir[2]};
  {
    double l = sqrt(Ld[0] * Ld[0] + Ld[1] * Ld[1] + Ld[2] * Ld[2]);
    for (int i = 0; i < 3; ++i) Ld[i] /= l;
  }
  int64_t n_cand = 0, n_cov = 0, n_amb = 0, n_soft = 0, n_soft32 = 0;
  uint64_t hash = 1469598103934665603ULL;

  double* nrm = (double*)malloc(sizeof(double) * 3 * V);
  double* cur = (double*)malloc(sizeof(double) * 6 * V);
  double* key0 = (double*)malloc(sizeof(double) * 6 * V);
  double* key1 = (double*)malloc(sizeof(double) * 6 * V);
  double* bestk = (double*)malloc(sizeof(double) * (npix + 1));
  double* secondk = (double*)malloc(sizeof(double) * (npix + 1));
  double* bestw = (double*)malloc(sizeof(double) * 3 * (npix + 1));
  double* prod = (double*)malloc(sizeof(double) * (npix + 1));
  int32_t* bestf = (int32_t*)malloc(sizeof(int32_t) * (npix + 1));
  uint8_t* amb = (uint8_t*)malloc(npix + 1);
  uint8_t* samb = (uint8_t*)malloc(npix + 1); /* flags of soft terms: count only if uncovered */
  int32_t* nsoft32 = (int32_t*)malloc(sizeof(int32_t) * (npix + 1)); /* terms above 2^-25, per sample */
  double* gcur = backward ? (double*)calloc(6 * (size_t)V, sizeof(double)) : NULL;
  double* gslot = backward ? (double*)calloc(6 * (size_t)V * (S + 1), sizeof(double)) : NULL;
  double* gnb = backward ? (double*)calloc(3 * (size_t)V, sizeof(double)) : NULL;
  size_t* pstart = backward ? (size_t*)malloc(sizeof(size_t) * (npix + 2)) : NULL;
  soft_entry* sorted = NULL;
  entry_list L = {NULL, 0, 0};
  int ok = nrm && cur && key0 && key1 && bestk && secondk && bestw && prod && bestf && amb && samb &&
           (!backward || (gcur && gslot && gnb && pstart));
  if (!ok) goto fail;

  orc_vertex_normals(s, nrm);
  if (rgba) memset(rgba, 0, sizeof(double) * 4 * npix);
  if (backward) {
    memset(gverts, 0, sizeof(double) * 3 * V);
    if (galb) memset(galb, 0, sizeof(double) * 3 * V);
  }
  int32_t loaded_seg = -1;

  for (int32_t k = 0; k < T; ++k) {
    int32_t seg;
    double t, tau;
    orc_sample_time(s, k, &seg, &t, &tau);
    const int32_t X = sample_key_x(s, k);
    if (mode == ORC_PLAIN_EXACT) {
      orc_vertex_state(s, nrm, t, cur);
    } else {
      if (seg != loaded_seg) {
        orc_vertex_state(s, nrm, (double)seg / S, key0);
        orc_vertex_state(s, nrm, (double)(seg + 1) / S, key1);
        loaded_seg = seg;
      }
      lerp_state(key0, key1, tau, cur, 6 * (size_t)V);
    }
    const double* keyX = X == 0 ? key0 : key1;

    for (size_t p = 0; p < npix; ++p) {
      bestk[p] = -INFINITY;
      secondk[p] = -INFINITY;
      bestf[p] = -1;
      prod[p] = 1.0;
      amb[p] = 0;
      samb[p] = 0;
      nsoft32[p] = 0;
    }
    L.n = 0;

    /* ---- pass over triangles: coverage, z-test, soft terms */
    for (int32_t f = 0; f < F; ++f) {
      const int32_t* id = s->faces + 3 * f;
      double tri[6], z[3];
      int culled = 0;
      for (int i = 0; i < 3; ++i) {
        tri[2 * i] = cur[6 * id[i]];
        tri[2 * i + 1] = cur[6 * id[i] + 1];
        z[i] = cur[6 * id[i] + 2];
        if (mode == ORC_PLAIN_EXACT) {
          if (z[i] <= s->znear) culled = 1;
        } else if (key0[6 * id[i] + 2] <= s->znear || key1[6 * id[i] + 2] <= s->znear) {
          culled = 1;
        }
      }
      if (culled) continue;
      double D = det_tri(tri);
      double lmax2 = 0;
      for (int e = 0; e < 3; ++e) {
        int i = e, j = (e + 1) % 3;
        double dx = tri[2 * j] - tri[2 * i], dy = tri[2 * j + 1] - tri[2 * i + 1];
        if (dx * dx + dy * dy > lmax2) lmax2 = dx * dx + dy * dy;
      }
      const int degenerate = fabs(D) <= D_MIN;
      const int degen_band = fabs(D) <= D_MIN + ETA_DET * lmax2;
      double xmin = fmin(tri[0], fmin(tri[2], tri[4])) - r, xmax = fmax(tri[0], fmax(tri[2], tri[4])) + r;
      double ymin = fmin(tri[1], fmin(tri[3], tri[5])) - r, ymax = fmax(tri[1], fmax(tri[3], tri[5])) + r;
      int32_t ilo = x0, ihi = x0 + w - 1, jlo = y0, jhi = y0 + h - 1;
      if (!soft_all) {
        int32_t a = (int32_t)floor((xmin + 1.0) * s->W / 2.0 - 0.5) - 1;
        int32_t b = (int32_t)ceil((xmax + 1.0) * s->W / 2.0 - 0.5) + 1;
        int32_t c = (int32_t)floor((1.0 - ymax) * s->H / 2.0 - 0.5) - 1;
        int32_t d = (int32_t)ceil((1.0 - ymin) * s->H / 2.0 - 0.5) + 1;
        if (a > ilo) ilo = a;
        if (b < ihi) ihi = b;
        if (c > jlo) jlo = c;
        if (d < jhi) jhi = d;
      }
      /* edge lengths opposite each vertex, for signed edge distances */
      double elen[3];
      for (int i = 0; i < 3; ++i) {
        int a = (i + 1) % 3, b = (i + 2) % 3;
        elen[i] = hypot(tri[2 * b] - tri[2 * a], tri[2 * b + 1] - tri[2 * a + 1]);
      }
      for (int32_t j = jlo; j <= jhi; ++j) {
        double v = 1.0 - 2.0 * (j + 0.5) / s->H;
        int inside_y = v >= ymin && v <= ymax;
        if (!soft_all && !inside_y) continue;
        for (int32_t i = ilo; i <= ihi; ++i) {
          double u = 2.0 * (i + 0.5) / s->W - 1.0;
          int inside = inside_y && u >= xmin && u <= xmax;
          if (!soft_all && !inside) continue;
          size_t p = (size_t)(j - y0) * w + (i - x0);
          if (inside) {
            ++n_cand;
            if (degen_band) amb[p] |= AMB_DEGEN;
          }
          if (degenerate) continue;
          double wb[3];
          orc_barycentric(tri, u, v, wb);
          /* signed distances to the three edge lines, positive inside */
          double sd[3], sgn = D > 0 ? 1.0 : -1.0, mn = INFINITY;
          for (int q = 0; q < 3; ++q) {
            sd[q] = wb[q] * fabs(D) / (elen[q] > 0 ? elen[q] : 1.0);
            (void)sgn;
            if (sd[q] < mn) mn = sd[q];
          }
          if (mn >= -ETA_COV && mn <= ETA_COV) amb[p] |= AMB_COVER;
          const int covered = wb[0] >= 0.0 && wb[1] >= 0.0 && wb[2] >= 0.0;
          const double wmax = fmax(1.0, fmax(fabs(wb[0]), fmax(fabs(wb[1]), fabs(wb[2]))));
          const double cond = EPS32 * lmax2 / fabs(D) * wmax;
          if (covered && cond > COND_LIMIT) amb[p] |= AMB_COND;
          if (covered) {
            /* z-test on perspective-correct inverse depth: larger is nearer */
            double key = wb[0] / z[0] + wb[1] / z[1] + wb[2] / z[2];
            if (key > bestk[p] || (key == bestk[p] && f < bestf[p])) {
              secondk[p] = bestk[p];
              bestk[p] = key;
              bestf[p] = f;
              bestw[3 * p] = wb[0]; bestw[3 * p + 1] = wb[1]; bestw[3 * p + 2] = wb[2];
            } else if (key > secondk[p]) {
              secondk[p] = key;
            }
          } else {
            /* soft coverage of a background candidate (Eqs. probability-function .. back) */
            closest_t c;
            double d;
            if (mode == ORC_FAST_REF) {
              double trX[6];
              for (int q = 0; q < 3; ++q) {
                trX[2 * q] = keyX[6 * id[q]];
                trX[2 * q + 1] = keyX[6 * id[q] + 1];
              }
              double pxp = wb[0] * trX[0] + wb[1] * trX[2] + wb[2] * trX[4];
              double pyp = wb[0] * trX[1] + wb[1] * trX[3] + wb[2] * trX[5];
              closest_point(trX, pxp, pyp, &c);
              double qx = c.w[0] * tri[0] + c.w[1] * tri[2] + c.w[2] * tri[4];
              double qy = c.w[0] * tri[1] + c.w[1] * tri[3] + c.w[2] * tri[5];
              d = (u - qx) * (u - qx) + (v - qy) * (v - qy);
              if (c.d2_second <= c.d2 * (1.0 + ETA_REGION) + 1e-30) {
                /* a near tie between two edge candidates in F(X): it matters only if the two
                 * closest points give different soft terms at F(tau) */
                double ax = c.w_second[0] * tri[0] + c.w_second[1] * tri[2] + c.w_second[2] * tri[4];
                double ay = c.w_second[0] * tri[1] + c.w_second[1] * tri[3] + c.w_second[2] * tri[5];
                double d_alt = (u - ax) * (u - ax) + (v - ay) * (v - ay);
                double om, dA;
                if (fmin(d, d_alt) <= r2 && fabs(soft_prob(s, d, &om, &dA) - soft_prob(s, d_alt, &om, &dA)) > 1e-6)
                  samb[p] |= AMB_REGION;
              }
            } else {
              closest_point(tri, u, v, &c);
              d = c.d2;
            }
            const int include = soft_all || d <= r2;
            if (include && mode == ORC_FAST_REF && cond > COND_LIMIT) samb[p] |= AMB_COND;
            if (include && mode == ORC_FAST_REF) {
              /* The fast-mode gradient flows through w* only inside an edge region, so it jumps
               * where the search in F(X) switches feature.  Flag when the switch is within FP32
               * reach: an attaining edge whose projection lies near an end (the vertex
               * alternative is (m L)^2 farther), or a near tie between different features. (The
               * exact distance of the plain modes has a continuous gradient there.) */
              for (int q = 0; q < 3; ++q) {
                if (c.d2e[q] > c.d2 * (1.0 + 1e-9) + 1e-300) continue;
                double m = fmin(fabs(c.traw[q]), fabs(1.0 - c.traw[q]));
                if (m * m * c.L2e[q] <= ETA_CLAMP * c.d2) samb[p] |= AMB_CLAMP;
              }
              if (c.d2_second <= c.d2 * (1.0 + ETA_CLAMP) + 1e-30 &&
                  fabs(c.w[0] - c.w_second[0]) + fabs(c.w[1] - c.w_second[1]) + fabs(c.w[2] - c.w_second[2]) > 1e-9)
                samb[p] |= AMB_CLAMP;
            }
            hash = fnv(fnv(fnv(hash, k * 7919 + 1), (int64_t)p * 104729 + f), c.region * 2 + include);
            if (include) {
              double fv, dA;
              soft_prob(s, d, &fv, &dA);
              prod[p] *= fv;
              ++n_soft;
              if (exp(-d / s->delta) > SOFT32_MIN) ++nsoft32[p];  /* inside the single-precision radius */
              if (backward) {
                soft_entry se = {(int32_t)p, f, fv, dA, d};
                if (!push_entry(&L, se)) goto fail;
              }
            }
          }
        }
      }
    }

    /* ---- per pixel: shade the winner or take the soft alpha (Sec. 3.3 split, Eq. fore) */
    for (size_t p = 0; p < npix; ++p) {
      int32_t f = bestf[p];
      if (f >= 0 && secondk[p] > -INFINITY && bestk[p] - secondk[p] <= ETA_DEPTH * fabs(bestk[p]))
        amb[p] |= AMB_DEPTH;
      if (f < 0) amb[p] |= samb[p];
      if (amb[p]) ++n_amb;
      if (winners) winners[(size_t)k * npix + p] = f;
      hash = fnv(hash, (int64_t)k * 1000003 + (int64_t)p * 31 + f);
      if (f < 0) n_soft32 += nsoft32[p];
      if (f >= 0) {
        ++n_cov;
        const int32_t* id = s->faces + 3 * f;
        const double* wb = bestw + 3 * p;
        /* attribute weights: the screen-space barycentrics (Eq. fore) or the perspective-correct
         * aw_i = (w_i / z_i) / S, S = sum_j w_j / z_j, z the vertices' camera depths */
        double aw[3], zc[3], S_w = 0.0;
        for (int q = 0; q < 3; ++q) {
          zc[q] = cur[6 * id[q] + 2];
          aw[q] = wb[q];
          S_w += wb[q] / zc[q];
        }
        if (s->interp == 1)
          for (int q = 0; q < 3; ++q) aw[q] = wb[q] / zc[q] / S_w;
        double col[3] = {0, 0, 0}, nn[3] = {0, 0, 0};
        for (int q = 0; q < 3; ++q)
          for (int c = 0; c < 3; ++c) {
            if (!s->texture) col[c] += aw[q] * s->albedo[3 * id[q] + c];
            nn[c] += aw[q] * cur[6 * id[q] + 3 + c];
          }
        /* textured: the vertex attribute is uv_i (Eq. fore) and the colour its texture sample */
        double tuv[2] = {0, 0}, dcdu[3] = {0, 0, 0}, dcdv[3] = {0, 0, 0};
        tex_taps taps;
        if (s->texture) {
          for (int q = 0; q < 3; ++q) {
            tuv[0] += aw[q] * s->uv[2 * id[q]];
            tuv[1] += aw[q] * s->uv[2 * id[q] + 1];
          }
          tex_sample(s, tuv[0], tuv[1], col, dcdu, dcdv, &taps);
          hash = fnv(hash, taps.cell);
          if (taps.edge < ETA_TEXCELL * fmax(1.0, fmax(s->tex_w, s->tex_h) / 64.0)) amb[p] |= AMB_TEXCELL;
        }
        double len = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
        double dot = len > 0 ? (nn[0] * Ld[0] + nn[1] * Ld[1] + nn[2] * Ld[2]) / len : 0.0;
        double shade = s->k_ambient + s->k_diffuse * (dot > 0 ? dot : 0.0);
        hash = fnv(hash, dot > 0);
        if (fabs(dot) < ETA_LAMBERT) amb[p] |= AMB_LAMBERT;
        if (rgba) {
          for (int c = 0; c < 3; ++c) rgba[4 * p + c] += col[c] * shade;
          rgba[4 * p + 3] += 1.0;
        }
        if (backward) {
          const double* G = dl + 4 * p;
          double gcol[3], gshade = 0, gw[3] = {0, 0, 0};
          for (int c = 0; c < 3; ++c) {
            gcol[c] = G[c] / T * shade;
            gshade += G[c] / T * col[c];
          }
          if (s->texture) {
            /* c = texture(sum_q aw_q uv_q): dL/daw_q = uv_q . (dL/du, dL/dv); texels by the taps */
            double gu = 0, gv = 0;
            for (int c = 0; c < 3; ++c) {
              gu += dcdu[c] * gcol[c];
              gv += dcdv[c] * gcol[c];
            }
            for (int q = 0; q < 3; ++q) gw[q] += s->uv[2 * id[q]] * gu + s->uv[2 * id[q] + 1] * gv;
            if (s->dl_dtexture)
              for (int k = 0; k < 4; ++k)
                for (int c = 0; c < 3; ++c) s->dl_dtexture[3 * taps.idx[k] + c] += taps.wt[k] * gcol[c];
          } else {
            for (int q = 0; q < 3; ++q)
              for (int c = 0; c < 3; ++c) {
                if (galb) galb[3 * id[q] + c] += aw[q] * gcol[c];
                gw[q] += s->albedo[3 * id[q] + c] * gcol[c];
              }
          }
          if (len > 0 && dot > 0) {
            double nh[3] = {nn[0] / len, nn[1] / len, nn[2] / len};
            double gnh[3] = {s->k_diffuse * gshade * Ld[0], s->k_diffuse * gshade * Ld[1],
                             s->k_diffuse * gshade * Ld[2]};
            double ng = nh[0] * gnh[0] + nh[1] * gnh[1] + nh[2] * gnh[2];
            double gnn[3];
            for (int c = 0; c < 3; ++c) gnn[c] = (gnh[c] - nh[c] * ng) / len;
            for (int q = 0; q < 3; ++q)
              for (int c = 0; c < 3; ++c) {
                gcur[6 * id[q] + 2 + c] += aw[q] * gnn[c];
                gw[q] += cur[6 * id[q] + 3 + c] * gnn[c];
              }
          }
          if (s->interp == 1) {
            /* gw holds dL/daw: dL/dw_k = (gw_k - sum_i gw_i aw_i) / (z_k S), dL/dz_k = -(w_k / z_k) dL/dw_k */
            double sa = aw[0] * gw[0] + aw[1] * gw[1] + aw[2] * gw[2];
            for (int q = 0; q < 3; ++q) {
              gw[q] = (gw[q] - sa) / (zc[q] * S_w);
              gcur[6 * id[q] + 5] += -(wb[q] / zc[q]) * gw[q];
            }
          }
          double tri[6], y[3];
          for (int q = 0; q < 3; ++q) {
            tri[2 * q] = cur[6 * id[q]];
            tri[2 * q + 1] = cur[6 * id[q] + 1];
          }
          solve_transposed(tri, gw, y);
          for (int q = 0; q < 3; ++q) {
            gcur[6 * id[q]] += -y[0] * wb[q];
            gcur[6 * id[q] + 1] += -y[1] * wb[q];
          }
        }
      } else if (rgba) {
        rgba[4 * p + 3] += 1.0 - prod[p];
      }
      if (ambig) ambig[(size_t)k * npix + p] = amb[p];  /* after shading: Lambert, texel-cell flags */
    }

    /* ---- soft-coverage adjoint for uncovered samples: exclusive products per pixel */
    if (backward && L.n > 0) {
      for (size_t p = 0; p <= npix + 1; ++p) pstart[p] = 0;
      for (size_t q = 0; q < L.n; ++q) pstart[L.e[q].p + 2]++;
      for (size_t p = 2; p <= npix + 1; ++p) pstart[p] += pstart[p - 1];
      soft_entry* ns = (soft_entry*)realloc(sorted, L.n * sizeof(soft_entry));
      if (!ns) goto fail;
      sorted = ns;
      for (size_t q = 0; q < L.n; ++q) sorted[pstart[L.e[q].p + 1]++] = L.e[q];
      /* now entries of pixel p are sorted[pstart[p] .. pstart[p+1]) in face order */
      for (size_t p = 0; p < npix; ++p) {
        if (bestf[p] >= 0) continue;
        size_t b = pstart[p], e = pstart[p + 1];
        if (b == e) continue;
        double ga = dl[4 * p + 3] / T;
        if (ga == 0.0) continue;
        /* prefix products, then a reverse sweep with the suffix product */
        double suffix = 1.0;
        double* pre = (double*)malloc(sizeof(double) * (e - b + 1));
        if (!pre) goto fail;
        pre[0] = 1.0;
        for (size_t q = b; q < e; ++q) pre[q - b + 1] = pre[q - b] * sorted[q].fval;
        for (size_t qq = e; qq-- > b;) {
          const soft_entry* se = sorted + qq;
          double excl = pre[qq - b] * suffix;
          suffix *= se->fval;
          /* alpha = 1 - prod(1 - A_j): dalpha/dA_j = prod_{l != j}(1 - A_l) */
          double gd = ga * excl * se->dA;
          const int32_t* id = s->faces + 3 * se->f;
          int32_t i = (int32_t)(p % w) + x0, j = (int32_t)(p / w) + y0;
          double u = 2.0 * (i + 0.5) / s->W - 1.0, v = 1.0 - 2.0 * (j + 0.5) / s->H;
          double tri[6];
          for (int q = 0; q < 3; ++q) {
            tri[2 * q] = cur[6 * id[q]];
            tri[2 * q + 1] = cur[6 * id[q] + 1];
          }
          if (mode != ORC_FAST_REF) {
            /* exact squared distance: Danskin, dd/dv_i = -2 (p - q) w*_i */
            closest_t c;
            closest_point(tri, u, v, &c);
            double qx = c.w[0] * tri[0] + c.w[1] * tri[2] + c.w[2] * tri[4];
            double qy = c.w[0] * tri[1] + c.w[1] * tri[3] + c.w[2] * tri[5];
            for (int q = 0; q < 3; ++q) {
              gcur[6 * id[q]] += gd * -2.0 * (u - qx) * c.w[q];
              gcur[6 * id[q] + 1] += gd * -2.0 * (v - qy) * c.w[q];
            }
          } else {
            double wb[3], trX[6];
            orc_barycentric(tri, u, v, wb);
            for (int q = 0; q < 3; ++q) {
              trX[2 * q] = keyX[6 * id[q]];
              trX[2 * q + 1] = keyX[6 * id[q] + 1];
            }
            double pxp = wb[0] * trX[0] + wb[1] * trX[2] + wb[2] * trX[4];
            double pyp = wb[0] * trX[1] + wb[1] * trX[3] + wb[2] * trX[5];
            closest_t c;
            closest_point(trX, pxp, pyp, &c);
            double qx = c.w[0] * tri[0] + c.w[1] * tri[2] + c.w[2] * tri[4];
            double qy = c.w[0] * tri[1] + c.w[1] * tri[3] + c.w[2] * tri[5];
            /* d = |p - F(tau) w*|^2 */
            double gqx = -2.0 * (u - qx) * gd, gqy = -2.0 * (v - qy) * gd;
            double gws[3];
            for (int q = 0; q < 3; ++q) {
              gcur[6 * id[q]] += c.w[q] * gqx;
              gcur[6 * id[q] + 1] += c.w[q] * gqy;
              gws[q] = tri[2 * q] * gqx + tri[2 * q + 1] * gqy;
            }
            /* w* = (1-t) e_i + t e_j with t = ((p' - v_i).e)/|e|^2 when t is interior */
            double gpx = 0, gpy = 0;
            double* gX = gslot + 6 * (size_t)V * (seg + X);
            if (c.region < 3) {
              int ii = c.ei, jj = c.ej;
              double ex = trX[2 * jj] - trX[2 * ii], ey = trX[2 * jj + 1] - trX[2 * ii + 1];
              double L2 = ex * ex + ey * ey;
              double rx = pxp - trX[2 * ii], ry = pyp - trX[2 * ii + 1];
              double gt = gws[jj] - gws[ii], tt = c.t;
              gpx = gt * ex / L2;
              gpy = gt * ey / L2;
              gX[6 * id[ii]] += gt * (-ex - rx + 2.0 * tt * ex) / L2;
              gX[6 * id[ii] + 1] += gt * (-ey - ry + 2.0 * tt * ey) / L2;
              gX[6 * id[jj]] += gt * (rx - 2.0 * tt * ex) / L2;
              gX[6 * id[jj] + 1] += gt * (ry - 2.0 * tt * ey) / L2;
            }
            /* p' = F(X) w */
            double gw[3];
            for (int q = 0; q < 3; ++q) {
              gX[6 * id[q]] += wb[q] * gpx;
              gX[6 * id[q] + 1] += wb[q] * gpy;
              gw[q] = trX[2 * q] * gpx + trX[2 * q + 1] * gpy;
            }
            /* w = F(tau)^-1 p */
            double y[3];
            solve_transposed(tri, gw, y);
            for (int q = 0; q < 3; ++q) {
              gcur[6 * id[q]] += -y[0] * wb[q];
              gcur[6 * id[q] + 1] += -y[1] * wb[q];
            }
          }
        }
        free(pre);
      }
    }

    /* ---- state gradients of this sub-frame -> base vertices (exact) or keyframe slots */
    if (backward) {
      if (mode == ORC_PLAIN_EXACT) {
        chain_state(s, t, gcur, gverts, gnb);
      } else {
        double* g0 = gslot + 6 * (size_t)V * seg;
        double* g1 = gslot + 6 * (size_t)V * (seg + 1);
        for (size_t q = 0; q < 6 * (size_t)V; ++q) {
          g0[q] += (1.0 - tau) * gcur[q];
          g1[q] += tau * gcur[q];
        }
      }
      memset(gcur, 0, sizeof(double) * 6 * V);
    }
  }

  if (rgba)
    for (size_t q = 0; q < 4 * npix; ++q) rgba[q] /= T;
  if (backward) {
    if (mode != ORC_PLAIN_EXACT)
      for (int32_t sg = 0; sg <= S; ++sg)
        chain_state(s, (double)sg / S, gslot + 6 * (size_t)V * sg, gverts, gnb);
    normals_backward(s, gnb, gverts);
  }
  if (cnt) {
    for (int i = 0; i < ORC_CNT_N; ++i) cnt[i] = 0;
    cnt[ORC_CNT_CAND] = n_cand;
    cnt[ORC_CNT_COVERED] = n_cov;
    cnt[ORC_CNT_AMBIG] = n_amb;
    cnt[ORC_CNT_HASH] = (int64_t)hash;
    cnt[ORC_CNT_SOFT] = n_soft;
    cnt[ORC_CNT_SOFT32] = n_soft32;
  }
  free(nrm); free(cur); free(key0); free(key1); free(bestk); free(secondk); free(bestw);
  free(prod); free(bestf); free(amb); free(samb); free(nsoft32); free(gcur); free(gslot); free(gnb); free(pstart);
  free(sorted); free(L.e);
  return 0;
fail:
  free(nrm); free(cur); free(key0); free(key1); free(bestk); free(secondk); free(bestw);
  free(prod); free(bestf); free(amb); free(samb); free(nsoft32); free(gcur); free(gslot); free(gnb); free(pstart);
  free(sorted); free(L.e);
  return -1;
}

int32_t orc_render(const orc_scene* s, int32_t mode, int32_t flags, int32_t x0, int32_t y0,
                   int32_t w, int32_t h, double* rgba, int32_t* winners, uint8_t* ambig,
                   int64_t* counters) {
  return render_impl(s, mode, flags, x0, y0, w, h, rgba, winners, ambig, counters, NULL, NULL, NULL);
}

int32_t orc_render_backward(const orc_scene* s, int32_t mode, int32_t flags, int32_t x0,
                            int32_t y0, int32_t w, int32_t h, const double* dl_drgba,
                            double* dl_dverts, double* dl_dalbedo, int64_t* counters) {
  if (!dl_drgba || !dl_dverts) return -1;
  return render_impl(s, mode, flags, x0, y0, w, h, NULL, NULL, NULL, counters, dl_drgba, dl_dverts,
                     dl_dalbedo);
}
