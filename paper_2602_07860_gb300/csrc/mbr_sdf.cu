// mbr_sdf.cu -- differentiable SDF -> triangle mesh extraction for the rotational recovery
// (Sec. 5: the rotating object's shape is an SDF field; a mesh is extracted from it in a
// differentiable way and rendered by the motion-blur renderer).
//
// Marching tetrahedra on a regular grid: n cells per axis, (n+1)^3 samples s at lo + h (i, j, k),
// index (k (n+1) + j) (n+1) + i; a sample is inside when s < 0.  Every cube is split into the six
// tetrahedra corner 0 -> +e_a -> +e_a +e_b -> corner 7 (one per order (a, b, c) of the axes), so
// a tetrahedron edge always joins a grid point g to g + o with o in {0,1}^3 \ {0}: the edge's id is
// 7 g + dir(o).  A sign-changing edge carries one mesh vertex at the zero of the linear interpolant,
// p = p_g + t (p_g+o - p_g), t = s_g / (s_g - s_g+o).  Per tetrahedron: one corner alone on its side
// -> one triangle on its three edges; two and two -> the quad (a,c), (a,d), (b,d), (b,c) (a < b
// inside, c < d outside, tetrahedron order) cut along (a,c)-(b,d).  Triangles face the outside.
//
//   sdf_count_kernel   sign-changing edges (one flag per edge id) and triangles per tetrahedron
//   (scan)             vertex ids and face offsets (the library's paired exclusive scan)
//   sdf_vertex_kernel  vertex positions and their grid edges (the edges where the vertex ids step)
//   sdf_face_kernel    faces, oriented
//   sdf_grad_kernel    adjoint: dL/dp of each vertex -> dL/ds of its edge's two samples
#include <cstdint>

#include "mbr_internal.h"

namespace mbr {

namespace {

__host__ __device__ __forceinline__ int dir_of(int ox, int oy, int oz) {  // o != 0 -> 0..6
  return (ox | (oy << 1) | (oz << 2)) - 1;
}

// the three axes of tetrahedron q in visiting order (0 x, 1 y, 2 z)
__device__ __forceinline__ void tet_axes(int q, int& a0, int& a1) {
  const int perm[6][2] = {{0, 1}, {0, 2}, {1, 0}, {1, 2}, {2, 0}, {2, 1}};
  a0 = perm[q][0];
  a1 = perm[q][1];
}

// corner bits (x = 1, y = 2, z = 4) of the four tetrahedron vertices
__device__ __forceinline__ void tet_corners(int q, int c[4]) {
  int a0, a1;
  tet_axes(q, a0, a1);
  c[0] = 0;
  c[1] = 1 << a0;
  c[2] = c[1] | (1 << a1);
  c[3] = 7;
}

__device__ __forceinline__ long long grid_idx(int n, int i, int j, int k) {
  return ((long long)k * (n + 1) + j) * (n + 1) + i;
}

__device__ __forceinline__ int tri_count(int nin) { return (nin == 1 || nin == 3) ? 1 : (nin == 2 ? 2 : 0); }

__global__ void sdf_count_kernel(int n, const float* __restrict__ s, int32_t* __restrict__ edge_flag,
                                 int32_t* __restrict__ tet_count) {
  const long long m = n + 1;
  const long long n_pts = m * m * m;
  const long long n_tets = (long long)n * n * n * 6;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < n_pts * 7) {
    const long long g = idx / 7;
    const int d = (int)(idx - g * 7) + 1;
    const int i = (int)(g % m), j = (int)((g / m) % m), k = (int)(g / (m * m));
    const int i2 = i + (d & 1), j2 = j + ((d >> 1) & 1), k2 = k + ((d >> 2) & 1);
    int flag = 0;
    if (i2 <= n && j2 <= n && k2 <= n) flag = (s[g] < 0.f) != (s[grid_idx(n, i2, j2, k2)] < 0.f);
    edge_flag[idx] = flag;
  }
  if (idx < n_tets) {
    const long long cube = idx / 6;
    const int q = (int)(idx - cube * 6);
    const int i = (int)(cube % n), j = (int)((cube / n) % n), k = (int)(cube / ((long long)n * n));
    int c[4], nin = 0;
    tet_corners(q, c);
#pragma unroll
    for (int r = 0; r < 4; ++r) nin += s[grid_idx(n, i + (c[r] & 1), j + ((c[r] >> 1) & 1), k + (c[r] >> 2))] < 0.f;
    tet_count[idx] = tri_count(nin);
  }
}

// a sign-changing edge is a step of the exclusive vertex offsets (n_edges + 1 entries)
__global__ void sdf_vertex_kernel(int n, const float* __restrict__ s, float lx, float ly, float lz, float h,
                                  const int32_t* __restrict__ vert_off, float* __restrict__ verts,
                                  int32_t* __restrict__ vert_edges) {
  const long long m = n + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * m * m * 7 || vert_off[idx + 1] == vert_off[idx]) return;
  const long long g = idx / 7;
  const int d = (int)(idx - g * 7) + 1;
  const int i = (int)(g % m), j = (int)((g / m) % m), k = (int)(g / (m * m));
  const int ox = d & 1, oy = (d >> 1) & 1, oz = (d >> 2) & 1;
  const long long g2 = grid_idx(n, i + ox, j + oy, k + oz);
  const float sa = s[g], sb = s[g2];
  const float t = sa / (sa - sb);
  const int v = vert_off[idx];
  verts[3 * (size_t)v] = fmaf(h, (float)i + t * (float)ox, lx);
  verts[3 * (size_t)v + 1] = fmaf(h, (float)j + t * (float)oy, ly);
  verts[3 * (size_t)v + 2] = fmaf(h, (float)k + t * (float)oz, lz);
  if (vert_edges) {
    vert_edges[2 * (size_t)v] = (int32_t)g;
    vert_edges[2 * (size_t)v + 1] = (int32_t)g2;
  }
}

__global__ void sdf_face_kernel(int n, const float* __restrict__ s, const int32_t* __restrict__ vert_off,
                                const int32_t* __restrict__ face_off, int32_t* __restrict__ faces) {
  const long long n_tets = (long long)n * n * n * 6;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_tets) return;
  const long long cube = idx / 6;
  const int q = (int)(idx - cube * 6);
  const int i = (int)(cube % n), j = (int)((cube / n) % n), k = (int)(cube / ((long long)n * n));
  int c[4];
  tet_corners(q, c);
  bool in[4];
  int nin = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    in[r] = s[grid_idx(n, i + (c[r] & 1), j + ((c[r] >> 1) & 1), k + (c[r] >> 2))] < 0.f;
    nin += in[r];
  }
  const int nt = tri_count(nin);
  if (!nt) return;
  int ins[4], outs[4], ni = 0, no = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if (in[r]) ins[ni++] = r;
    else outs[no++] = r;
  }
  int tri[2][3][2];
  if (nt == 1) {
    const int lone = ni == 1 ? ins[0] : outs[0];
    const int* rest = ni == 1 ? outs : ins;
    for (int e = 0; e < 3; ++e) {
      tri[0][e][0] = lone;
      tri[0][e][1] = rest[e];
    }
  } else {
    const int a = ins[0], b = ins[1], cc = outs[0], dd = outs[1];
    const int quad[4][2] = {{a, cc}, {a, dd}, {b, dd}, {b, cc}};
    const int cut[2][3] = {{0, 1, 2}, {0, 2, 3}};
    for (int t = 0; t < 2; ++t)
      for (int e = 0; e < 3; ++e) {
        tri[t][e][0] = quad[cut[t][e]][0];
        tri[t][e][1] = quad[cut[t][e]][1];
      }
  }
  // outward direction in exact integers: (mean of outside corners - mean of inside corners) x ni no
  int G[3] = {0, 0, 0};
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int w = in[r] ? -no : ni;
    G[0] += w * (c[r] & 1);
    G[1] += w * ((c[r] >> 1) & 1);
    G[2] += w * (c[r] >> 2);
  }
  const long long fbase = face_off[idx];
  for (int t = 0; t < nt; ++t) {
    // doubled edge midpoints of the canonical cube; the triangle they span is never degenerate
    int M[3][3];
    for (int e = 0; e < 3; ++e) {
      const int p = c[tri[t][e][0]], r = c[tri[t][e][1]];
      M[e][0] = (p & 1) + (r & 1);
      M[e][1] = ((p >> 1) & 1) + ((r >> 1) & 1);
      M[e][2] = (p >> 2) + (r >> 2);
    }
    const int ux = M[1][0] - M[0][0], uy = M[1][1] - M[0][1], uz = M[1][2] - M[0][2];
    const int wx = M[2][0] - M[0][0], wy = M[2][1] - M[0][1], wz = M[2][2] - M[0][2];
    const int nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
    const bool flip = nx * G[0] + ny * G[1] + nz * G[2] < 0;
    int32_t vid[3];
    for (int e = 0; e < 3; ++e) {
      const int p = c[tri[t][e][0]], r = c[tri[t][e][1]];
      const int lo_c = p < r ? p : r, hi_c = p < r ? r : p;  // corners are nested: lo_c's bits are in hi_c
      const long long g = grid_idx(n, i + (lo_c & 1), j + ((lo_c >> 1) & 1), k + (lo_c >> 2));
      const int o = hi_c & ~lo_c;
      vid[e] = vert_off[g * 7 + dir_of(o & 1, (o >> 1) & 1, o >> 2)];
    }
    int32_t* out = faces + 3 * (size_t)(fbase + t);
    out[0] = vid[0];
    out[1] = flip ? vid[2] : vid[1];
    out[2] = flip ? vid[1] : vid[2];
  }
}

__global__ void sdf_grad_kernel(int nv, const float* __restrict__ s, float h, const int32_t* __restrict__ vert_edges,
                                const float* __restrict__ dl_dverts, float* __restrict__ dl_ds, int n) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const long long a = vert_edges[2 * (size_t)v], b = vert_edges[2 * (size_t)v + 1];
  const long long m = n + 1;
  // p = p_a + t (p_b - p_a), p_b - p_a = h o;  t = s_a / (s_a - s_b)
  const int ox = (int)((b % m) - (a % m)), oy = (int)(((b / m) % m) - ((a / m) % m)),
            oz = (int)((b / (m * m)) - (a / (m * m)));
  const float gt = h * (dl_dverts[3 * (size_t)v] * ox + dl_dverts[3 * (size_t)v + 1] * oy +
                        dl_dverts[3 * (size_t)v + 2] * oz);
  const float sa = s[a], sb = s[b], den = sa - sb;
  const float q = gt / (den * den);
  atomicAdd(dl_ds + a, -sb * q);
  atomicAdd(dl_ds + b, sa * q);
}

}  // namespace

void launch_sdf_count(int n, const float* s, int32_t* edge_flag, int32_t* tet_count, cudaStream_t st) {
  const long long m = n + 1, work = m * m * m * 7;
  sdf_count_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(n, s, edge_flag, tet_count);
}

void launch_sdf_write(int n, const float* s, const float lo[3], float h, const int32_t* vert_off,
                      const int32_t* face_off, float* verts, int32_t* vert_edges, int32_t* faces, cudaStream_t st) {
  const long long m = n + 1, n_edges = m * m * m * 7, n_tets = (long long)n * n * n * 6;
  sdf_vertex_kernel<<<(unsigned)((n_edges + 255) / 256), 256, 0, st>>>(n, s, lo[0], lo[1], lo[2], h, vert_off,
                                                                      verts, vert_edges);
  sdf_face_kernel<<<(unsigned)((n_tets + 255) / 256), 256, 0, st>>>(n, s, vert_off, face_off, faces);
}

void launch_sdf_grad(int n, const float* s, float h, int nv, const int32_t* vert_edges, const float* dl_dverts,
                     float* dl_ds, cudaStream_t st) {
  if (nv > 0) sdf_grad_kernel<<<(nv + 255) / 256, 256, 0, st>>>(nv, s, h, vert_edges, dl_dverts, dl_ds, n);
}

}  // namespace mbr
