// mesh_cells.cuh -- surface of one marching cell: its topology as a function of which of its
// 8 corners are inside (D < 0), and its triangles. Host and device code: the mesh kernel
// builds a 256-entry topology table from it in shared memory and emits each cell's triangles
// with it; a host-compiled check runs the same code on single cells.
//
// Cube corners are numbered c = x + 2 y + 4 z. Edges 0-3 run along x, 4-7 along y, 8-11
// along z. Each face is walked counter-clockwise as seen from outside the cube; on it, the
// surface boundary runs from the edge where the walk leaves the inside corners to the edge
// where it next enters them, so the inside corners lie on the segment's left. A face whose
// four edges all cross cuts off each of its two inside corners on its own. Two cells sharing
// a face walk it in opposite directions, so their segments on it are the same ones reversed,
// and the surface of neighbouring cells closes up with one orientation. Following the
// segments from edge to edge gives closed loops of 3 to 12 edges, at most 4 per cell.
#pragma once

#include <cstdint>

namespace vbx {

// Corners at the two ends of edge e (4 bits per edge in a constant: 0,2,4,6 | 0,1,4,5 |
// 0,1,2,3); the upper one is one step along the edge's axis.
__host__ __device__ __forceinline__ int mc_edge_lo(int e) { return (int)((0x321054106420ull >> (4 * e)) & 15u); }
__host__ __device__ __forceinline__ int mc_edge_hi(int e) { return mc_edge_lo(e) + (1 << (e >> 2)); }
// Axis along which edge e runs.
__host__ __device__ __forceinline__ int mc_edge_axis(int e) { return e >> 2; }

// Face f (x = 0, x = 1, y = 0, y = 1, z = 0, z = 1): corner i and the edge from corner i to
// corner i + 1, counter-clockwise seen from outside. Packed 4 bits per entry.
__host__ __device__ __forceinline__ int mc_face_corner(int f, int i) {
  const uint32_t tab[6] = {0x2640u, 0x5731u, 0x4510u, 0x3762u, 0x1320u, 0x6754u};
  return (int)((tab[f] >> (4 * i)) & 15u);
}
__host__ __device__ __forceinline__ int mc_face_edge(int f, int i) {
  const uint32_t tab[6] = {0x4a68u, 0x97b5u, 0x8290u, 0x1b3au, 0x0514u, 0x6372u};
  return (int)((tab[f] >> (4 * i)) & 15u);
}

// Loops of one cell: `seq` holds the loops' edges one after the other, 4 bits each, first edge
// in the lowest bits; `meta` bits 0-3 the triangle count (a loop of 3 is one triangle, a loop
// of k > 3 is k triangles around its centroid), bits 4-6 the loop count, and 4 bits per loop
// length from bit 8.
struct McLoops {
  unsigned long long seq;
  uint32_t meta;
};

__host__ __device__ __forceinline__ int mc_triangles(uint32_t meta) { return (int)(meta & 15u); }
__host__ __device__ __forceinline__ int mc_loop_count(uint32_t meta) { return (int)((meta >> 4) & 7u); }
__host__ __device__ __forceinline__ int mc_loop_len(uint32_t meta, int j) { return (int)((meta >> (8 + 4 * j)) & 15u); }

__host__ __device__ inline McLoops mc_cell_loops(unsigned pattern) {
  unsigned cross = 0;  // edges whose two corners differ
  for (int e = 0; e < 12; ++e)
    if (((pattern >> mc_edge_lo(e)) ^ (pattern >> mc_edge_hi(e))) & 1u) cross |= 1u << e;
  int succ[12];
  for (int e = 0; e < 12; ++e) succ[e] = -1;
  for (int f = 0; f < 6; ++f) {
    int n = 0;
    for (int i = 0; i < 4; ++i) n += (cross >> mc_face_edge(f, i)) & 1u;
    for (int i = 0; i < 4; ++i) {
      if (!((pattern >> mc_face_corner(f, i)) & 1u)) continue;  // corner i outside
      const int leave = mc_face_edge(f, i);
      if (n == 4) {
        succ[leave] = mc_face_edge(f, (i + 3) & 3);  // the inside corner alone
      } else if (n == 2 && !((pattern >> mc_face_corner(f, (i + 1) & 3)) & 1u)) {
        int j = (i + 1) & 3;
        while (!((cross >> mc_face_edge(f, j)) & 1u)) j = (j + 1) & 3;
        succ[leave] = mc_face_edge(f, j);
      }
    }
  }
  McLoops out{0ull, 0u};
  unsigned used = 0;
  int pos = 0, loops = 0, tris = 0;
  for (int e0 = 0; e0 < 12; ++e0) {
    if (!((cross >> e0) & 1u) || ((used >> e0) & 1u)) continue;
    int k = 0;
    for (int e = e0; e >= 0 && !((used >> e) & 1u) && k < 12; e = succ[e], ++k) {
      used |= 1u << e;
      out.seq |= (unsigned long long)e << (4 * pos++);
    }
    if (loops < 4) out.meta |= (uint32_t)k << (8 + 4 * loops);
    ++loops;
    tris += k == 3 ? 1 : k;
  }
  out.meta |= (uint32_t)(tris & 15) | ((uint32_t)(loops & 7) << 4);
  return out;
}

// float32 operations rounded one at a time (no contraction into fused multiply-adds).
__host__ __device__ __forceinline__ float mc_add(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float mc_sub(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
__host__ __device__ __forceinline__ float mc_mul(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ float mc_div(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdiv_rn(a, b);
#else
  return a / b;
#endif
}

// Vertex on edge e: pa + t (pb - pa), t = Da / (Da - Db), with corner values D(c) and corner
// coordinates P(c, axis). The corners differ along the edge's axis only, and on the other two
// axes the formula returns pa exactly (t is finite in [0, 1], pb - pa = 0, pa != 0), so only
// that axis is computed.
#pragma nv_exec_check_disable
template <class DF, class PF>
__host__ __device__ __forceinline__ void mc_vertex(int e, const DF& D, const PF& P, float v[3]) {
  const int a = mc_edge_lo(e), b = mc_edge_hi(e), ax = mc_edge_axis(e);
  const float Da = D(a), Db = D(b);
  const float t = mc_div(Da, mc_sub(Da, Db));
#pragma unroll
  for (int q = 0; q < 3; ++q) v[q] = P(a, q);
  const float pa = P(a, ax), pb = P(b, ax);
  const float x = mc_add(pa, mc_mul(t, mc_sub(pb, pa)));
  v[0] = ax == 0 ? x : v[0];
  v[1] = ax == 1 ? x : v[1];
  v[2] = ax == 2 ? x : v[2];
}

// Triangles of one cell with loops L, each vertex evaluated once and handed to
// out(triangle index in cell, slot 0/1/2 = a/b/c, vertex). Each loop is emitted against its
// direction, so that (b - a) x (c - a) points to positive D: a loop of 3 edge vertices v0 v1 v2
// gives the triangle (v0, v2, v1); a loop of k > 3 gives the k triangles
// (centroid, v[i + 1], v[i]), so v[i] is slot c of triangle i and slot b of triangle i - 1, and
// the centroid -- the float32 sum of the loop's vertices in loop order, divided by k -- is
// slot a of all k.
#pragma nv_exec_check_disable
template <class DF, class PF, class Sink>
__host__ __device__ __forceinline__ void mc_emit(const McLoops& L, const DF& D, const PF& P, const Sink& out) {
  const int nl = mc_loop_count(L.meta);
  int pos = 0, idx = 0;
  for (int j = 0; j < nl; ++j) {
    const int k = mc_loop_len(L.meta, j);
    const unsigned long long s = L.seq >> (4 * pos);
    pos += k;
    if (k == 3) {
      float w[3];
      mc_vertex((int)(s & 15u), D, P, w);
      out(idx, 0, w);
      mc_vertex((int)((s >> 4) & 15u), D, P, w);
      out(idx, 2, w);
      mc_vertex((int)((s >> 8) & 15u), D, P, w);
      out(idx, 1, w);
      ++idx;
      continue;
    }
    float cen[3] = {0.0f, 0.0f, 0.0f};
    for (int i = 0; i < k; ++i) {
      float w[3];
      mc_vertex((int)((s >> (4 * i)) & 15u), D, P, w);
#pragma unroll
      for (int q = 0; q < 3; ++q) cen[q] = mc_add(cen[q], w[q]);
      out(idx + i, 2, w);
      out(idx + (i == 0 ? k - 1 : i - 1), 1, w);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) cen[q] = mc_div(cen[q], (float)k);
    for (int i = 0; i < k; ++i) out(idx + i, 0, cen);
    idx += k;
  }
}

}  // namespace vbx
