/*
 * sdf_oracle.c -- FP64, single-threaded CPU oracle of the SDF -> triangle mesh extraction used by
 * the rotational recovery (Sec. 5, rotation task: an SDF field is optimised and a mesh is
 * extracted from it differentiably, then rendered).  TEST INFRASTRUCTURE ONLY (see
 * mbr_oracle.h); it shares nothing with the CUDA path.
 *
 * The paper extracts with FlexiCubes; this library's extractor is marching tetrahedra on the
 * regular grid, which the oracle states directly:
 *   - grid: n cells per axis, (n+1)^3 samples s at points lo + h (i, j, k), index
 *     (k (n+1) + j) (n+1) + i; a sample is inside when s < 0 (s = 0 counts as outside);
 *   - every cube splits into six tetrahedra that share the cube's main diagonal, one per order
 *     of the axes: corner 0 -> +e_first -> +e_second -> corner 7.  Each square face of the grid is
 *     then cut along the diagonal through its lowest corner on both sides, so neighbouring cubes
 *     agree and the surface closes;
 *   - a tetrahedron edge (a, b) whose ends lie on different sides carries the surface vertex
 *     p = p_a + t (p_b - p_a), t = s_a / (s_a - s_b) (the zero of the linear interpolant); vertices
 *     are shared by grid edge, identified by its end indices (a < b);
 *   - one vertex on its own side: one triangle on its three edges; two and two: the quad on the
 *     four crossing edges (in, out) = (a, c), (a, d), (b, d), (b, c) with a < b and c < d in the
 *     tetrahedron's vertex order, cut along (a, c) - (b, d);
 *   - every triangle faces the outside (s >= 0): oriented so that its normal, computed with the
 *     crossings at the edge midpoints (never degenerate), points from the mean of the
 *     tetrahedron's inside corners towards the mean of its outside corners.
 * The adjoint holds the crossing topology fixed: dp/ds_a = (p_b - p_a) (-s_b) / (s_a - s_b)^2,
 * dp/ds_b = (p_b - p_a) s_a / (s_a - s_b)^2.
 */
#include "mbr_oracle.h"

#include <stdlib.h>
#include <string.h>

static int64_t grid_index(int32_t n, int32_t i, int32_t j, int32_t k) {
  return ((int64_t)k * (n + 1) + j) * (n + 1) + i;
}

static void grid_point(int32_t n, const double lo[3], double h, int64_t idx, double p[3]) {
  const int64_t m = n + 1;
  p[0] = lo[0] + h * (double)(idx % m);
  p[1] = lo[1] + h * (double)((idx / m) % m);
  p[2] = lo[2] + h * (double)(idx / (m * m));
}

typedef struct {
  int64_t a, b;  /* grid indices of the crossing edge, a < b */
} edge_key;

/* a growable list of vertices keyed by grid edge, kept sorted for lookup */
typedef struct {
  edge_key* keys;
  int64_t n, cap;
} key_list;

static int key_cmp(const edge_key* x, const edge_key* y) {
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  return 0;
}

static int key_cmp_void(const void* x, const void* y) { return key_cmp((const edge_key*)x, (const edge_key*)y); }

static int push_key(key_list* L, edge_key k) {
  if (L->n == L->cap) {
    int64_t c = L->cap ? 2 * L->cap : 1024;
    edge_key* p = (edge_key*)realloc(L->keys, sizeof(edge_key) * (size_t)c);
    if (!p) return -1;
    L->keys = p;
    L->cap = c;
  }
  L->keys[L->n++] = k;
  return 0;
}

static int64_t find_key(const key_list* L, edge_key k) {
  int64_t lo = 0, hi = L->n - 1;
  while (lo <= hi) {
    const int64_t mid = (lo + hi) / 2;
    const int c = key_cmp(&L->keys[mid], &k);
    if (c == 0) return mid;
    if (c < 0) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

/* The six tetrahedra of a cube as corner numbers (bit 0 = +x, bit 1 = +y, bit 2 = +z). */
static void cube_tets(int tets[6][4]) {
  const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (int q = 0; q < 6; ++q) {
    const int c1 = 1 << perm[q][0];
    const int c2 = c1 | (1 << perm[q][1]);
    tets[q][0] = 0;
    tets[q][1] = c1;
    tets[q][2] = c2;
    tets[q][3] = 7;
  }
}

static edge_key make_key(int64_t x, int64_t y) {
  edge_key k;
  k.a = x < y ? x : y;
  k.b = x < y ? y : x;
  return k;
}

/* Emit the triangles of one tetrahedron (grid indices g[4], values sv[4], corner positions P[4])
 * as edge-key triples; count only when out == NULL. */
static int tet_triangles(const int64_t g[4], const double sv[4], const double P[4][3], edge_key out[2][3]) {
  int in[4], nin = 0, ou[4], nout = 0;
  for (int q = 0; q < 4; ++q) {
    if (sv[q] < 0.0) in[nin++] = q;
    else ou[nout++] = q;
  }
  if (nin == 0 || nin == 4) return 0;
  int tri[2][3][2];  /* per triangle corner: the tetrahedron edge (vertex q, vertex r) */
  int nt = 0;
  if (nin == 1 || nin == 3) {
    const int lone = nin == 1 ? in[0] : ou[0];
    const int* rest = nin == 1 ? ou : in;
    for (int c = 0; c < 3; ++c) {
      tri[0][c][0] = lone;
      tri[0][c][1] = rest[c];
    }
    nt = 1;
  } else {
    const int a = in[0], b = in[1], c = ou[0], d = ou[1];  /* in tetrahedron order: a < b, c < d */
    const int quad[4][2] = {{a, c}, {a, d}, {b, d}, {b, c}};
    const int cut[2][3] = {{0, 1, 2}, {0, 2, 3}};
    for (int t = 0; t < 2; ++t)
      for (int e = 0; e < 3; ++e) {
        tri[t][e][0] = quad[cut[t][e]][0];
        tri[t][e][1] = quad[cut[t][e]][1];
      }
    nt = 2;
  }
  /* outward direction: mean of the outside corners minus mean of the inside corners */
  double gdir[3] = {0, 0, 0};
  for (int q = 0; q < 4; ++q)
    for (int x = 0; x < 3; ++x) gdir[x] += (sv[q] < 0.0 ? -1.0 / nin : 1.0 / nout) * P[q][x];
  for (int t = 0; t < nt; ++t) {
    double m[3][3];
    for (int e = 0; e < 3; ++e)
      for (int x = 0; x < 3; ++x) m[e][x] = 0.5 * (P[tri[t][e][0]][x] + P[tri[t][e][1]][x]);
    const double u[3] = {m[1][0] - m[0][0], m[1][1] - m[0][1], m[1][2] - m[0][2]};
    const double w[3] = {m[2][0] - m[0][0], m[2][1] - m[0][1], m[2][2] - m[0][2]};
    const double nrm[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
    const int flip = nrm[0] * gdir[0] + nrm[1] * gdir[1] + nrm[2] * gdir[2] < 0.0;
    if (out) {
      for (int e = 0; e < 3; ++e) {
        const int ee = flip ? (e == 0 ? 0 : 3 - e) : e;
        out[t][e] = make_key(g[tri[t][ee][0]], g[tri[t][ee][1]]);
      }
    }
  }
  return nt;
}

/* Visit every tetrahedron of every cube; fn receives its triangles. */
static int for_each_tet(int32_t n, const double* s, const double lo[3], double h,
                        int (*fn)(void*, edge_key[2][3], int), void* user) {
  int tets[6][4];
  cube_tets(tets);
  for (int32_t k = 0; k < n; ++k)
    for (int32_t j = 0; j < n; ++j)
      for (int32_t i = 0; i < n; ++i) {
        int64_t corner[8];
        for (int c = 0; c < 8; ++c) corner[c] = grid_index(n, i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1));
        for (int q = 0; q < 6; ++q) {
          int64_t g[4];
          double sv[4], P[4][3];
          for (int r = 0; r < 4; ++r) {
            g[r] = corner[tets[q][r]];
            sv[r] = s[g[r]];
            grid_point(n, lo, h, g[r], P[r]);
          }
          edge_key tk[2][3];
          const int nt = tet_triangles(g, sv, P, tk);
          if (nt && fn(user, tk, nt)) return -1;
        }
      }
  return 0;
}

typedef struct {
  key_list keys;
  edge_key* tris;  /* [3 * F] */
  int64_t F, cap;
} collect_state;

static int collect(void* user, edge_key tk[2][3], int nt) {
  collect_state* C = (collect_state*)user;
  for (int t = 0; t < nt; ++t) {
    if (C->F == C->cap) {
      int64_t c = C->cap ? 2 * C->cap : 1024;
      edge_key* p = (edge_key*)realloc(C->tris, sizeof(edge_key) * 3 * (size_t)c);
      if (!p) return -1;
      C->tris = p;
      C->cap = c;
    }
    for (int e = 0; e < 3; ++e) {
      C->tris[3 * C->F + e] = tk[t][e];
      if (push_key(&C->keys, tk[t][e])) return -1;
    }
    ++C->F;
  }
  return 0;
}

int32_t orc_sdf_extract(int32_t n, const double* s, const double lo[3], double h, int64_t max_verts,
                        int64_t max_faces, double* verts, int64_t* vert_edges, int32_t* faces, int64_t* counts) {
  if (n < 1 || !s || !lo || !counts) return -1;
  collect_state C;
  memset(&C, 0, sizeof(C));
  int rc = for_each_tet(n, s, lo, h, collect, &C);
  if (rc == 0) {
    /* unique vertices in ascending (a, b) order */
    qsort(C.keys.keys, (size_t)C.keys.n, sizeof(edge_key), key_cmp_void);
    int64_t u = 0;
    for (int64_t q = 0; q < C.keys.n; ++q)
      if (u == 0 || key_cmp(&C.keys.keys[u - 1], &C.keys.keys[q]) != 0) C.keys.keys[u++] = C.keys.keys[q];
    C.keys.n = u;
    counts[0] = u;
    counts[1] = C.F;
    if (u <= max_verts && C.F <= max_faces) {
      for (int64_t q = 0; q < u; ++q) {
        const edge_key k = C.keys.keys[q];
        double pa[3], pb[3];
        grid_point(n, lo, h, k.a, pa);
        grid_point(n, lo, h, k.b, pb);
        const double t = s[k.a] / (s[k.a] - s[k.b]);
        for (int x = 0; x < 3; ++x) verts[3 * q + x] = pa[x] + t * (pb[x] - pa[x]);
        if (vert_edges) {
          vert_edges[2 * q] = k.a;
          vert_edges[2 * q + 1] = k.b;
        }
      }
      for (int64_t f = 0; f < C.F; ++f)
        for (int e = 0; e < 3; ++e) faces[3 * f + e] = (int32_t)find_key(&C.keys, C.tris[3 * f + e]);
    } else {
      rc = 1;  /* outputs too small; counts tell the sizes */
    }
  }
  free(C.keys.keys);
  free(C.tris);
  return rc;
}

int32_t orc_sdf_extract_backward(int32_t n, const double* s, const double lo[3], double h, int64_t n_verts,
                                 const int64_t* vert_edges, const double* dl_dverts, double* dl_ds) {
  if (n < 1 || !s || !vert_edges || !dl_dverts || !dl_ds) return -1;
  for (int64_t q = 0; q < n_verts; ++q) {
    const int64_t a = vert_edges[2 * q], b = vert_edges[2 * q + 1];
    double pa[3], pb[3];
    grid_point(n, lo, h, a, pa);
    grid_point(n, lo, h, b, pb);
    const double den = s[a] - s[b];
    double g = 0.0;  /* dL/dt */
    for (int x = 0; x < 3; ++x) g += dl_dverts[3 * q + x] * (pb[x] - pa[x]);
    dl_ds[a] += g * (-s[b]) / (den * den);
    dl_ds[b] += g * s[a] / (den * den);
  }
  (void)lo;
  (void)h;
  return 0;
}
