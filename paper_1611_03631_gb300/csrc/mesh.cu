// mesh.cu -- iso-surface (D = 0) of the TSDF as triangles: the mesh layer that the system
// overview (Sec. III) builds from updated TSDF voxels on demand, for display. The paper names
// marching cubes (Sec. II) but fixes no variant; the cell rule is in mesh_cells.cuh.
//
// A cell is the cube between 8 neighbouring voxel centres, meshed when all 8 voxels are
// observed (W > 0); it belongs to the block holding its minimum corner, so a block's cells
// reach into its 7 upper neighbours by one voxel. Extraction works on whole blocks:
//   k_mesh_select  lists every block, or only those with a cell that reaches into a block
//                  marked stale (the marks are set where a scan's rays enter a block and by
//                  TSDF import)
//   k_mesh_blocks  one CTA per listed block (persistent grid): the block's D plus its
//                  one-voxel upper halo go to shared memory (NaN where unobserved), each thread
//                  counts the triangles of its cells from a 256-entry topology table built per
//                  CTA, a CTA scan and one 64-bit atomic place the block's triangles in one
//                  contiguous range, and each thread writes its cells' triangles there
//   k_mesh_clear   drops the stale marks of the listed blocks (launched only once the caller's
//                  buffers were large enough)
// Algorithmic traffic per listed block: (B + 1)^3 voxels of 8 B read, 52 B per triangle
// written (cell key 16 B, vertices 36 B), 24 B per block record.
#include <cuda_runtime.h>

#include "launch.h"
#include "mesh_cells.cuh"
#include "vbx_internal.cuh"

namespace vbx {

namespace {

constexpr int kMeshThreads = 256;  // also the number of topology table entries
constexpr int kMeshWarps = kMeshThreads / 32;
constexpr int kMaxEdge = 17;  // B + 1 for the largest block (16^3)
static_assert(kMeshThreads == 256, "one thread per inside/outside pattern builds the table");

// Inside/outside pattern of the cell whose minimum corner is staged at sD[base] (corner
// c = x + 2 y + 4 z), or 256 if a corner is unobserved.
__device__ __forceinline__ unsigned cell_pattern(const float* sD, int base, int E) {
  unsigned pat = 0u;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float d = sD[base + (c & 1) + ((c >> 1) & 1) * E + (c >> 2) * E * E];
    if (isnan(d)) return 256u;
    pat |= (d < 0.0f ? 1u : 0u) << c;
  }
  return pat;
}

__global__ void __launch_bounds__(kMeshThreads) k_mesh_select(DevMap m, int all) {
  const unsigned nb = min(__ldcg(&m.ctr->blocks), m.cap_blocks);
  const unsigned lane = threadIdx.x & 31u;
  const unsigned stride = gridDim.x * blockDim.x;
  // warp-uniform loop: the whole warp takes part in each ballot
  for (unsigned p0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); p0 < nb; p0 += stride) {
    const unsigned p = p0 + lane;
    bool need = false;
    if (p < nb) {
      need = all || m.mdirty[p];
      // upper neighbours (dx, dy, dz) in {0, 1}^3 \ {0}: k = (dx+1)*9 + (dy+1)*3 + (dz+1)
      const int kUp[7] = {14, 16, 17, 22, 23, 25, 26};
#pragma unroll
      for (int j = 0; j < 7; ++j) {
        if (need) break;
        const uint32_t q = __ldg(&m.nbr[(size_t)p * 27 + kUp[j]]);
        need = q < m.cap_blocks && m.mdirty[q];
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    unsigned base = 0u;
    if (lane == 0 && mask) base = atomicAdd(&m.ctr->mesh_blocks, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (need) m.mlist[base + __popc(mask & ((1u << lane) - 1u))] = p;
  }
}

__global__ void __launch_bounds__(kMeshThreads) k_mesh_blocks(DevMap m, MeshOut o) {
  __shared__ float sD[kMaxEdge * kMaxEdge * kMaxEdge];
  __shared__ unsigned long long sSeq[256];
  __shared__ uint32_t sMeta[256];
  __shared__ uint32_t sSlot[8];
  __shared__ unsigned sWarp[kMeshWarps];
  __shared__ unsigned long long sBase;
  const unsigned nsel = __ldcg(&m.ctr->mesh_blocks);
  if (blockIdx.x >= nsel) return;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  {
    const McLoops L = mc_cell_loops((unsigned)t);
    sSeq[t] = L.seq;
    sMeta[t] = L.meta;
  }
  const int B = m.B, blog = m.blog, E = B + 1, EE = E * E, E3 = EE * E;
  const unsigned ncell = 1u << m.b3log;
  const float v = m.v;
  for (unsigned i = blockIdx.x; i < nsel; i += gridDim.x) {
    const uint32_t p = __ldcg(&m.mlist[i]);
    // slot of the block at offset o = ox + 2 oy + 4 oz (kInvalid if absent)
    if (t < 8) sSlot[t] = t == 0 ? p : __ldg(&m.nbr[(size_t)p * 27 + 13 + (t & 1) * 9 + ((t >> 1) & 1) * 3 + (t >> 2)]);
    __syncthreads();  // also: the previous block's writes have read sD, sWarp and sBase
    const int3 bc = m.bcoord[p];
    for (int e = t; e < E3; e += kMeshThreads) {
      const int z = e / EE, r = e - z * EE, y = r / E, x = r - y * E;
      const uint32_t q = sSlot[(x >> blog) | ((y >> blog) << 1) | ((z >> blog) << 2)];
      float D = __int_as_float(0x7fc00000);  // NaN: unobserved
      if (q < m.cap_blocks) {
        const uint32_t local = (uint32_t)((((z & (B - 1)) << blog | (y & (B - 1))) << blog) | (x & (B - 1)));
        const float2 dw = __ldg(&m.tsdf[((size_t)q << m.b3log) | local]);
        if (dw.y > 0.0f) D = dw.x;
      }
      sD[e] = D;
    }
    __syncthreads();
    unsigned cnt = 0u;
    for (unsigned l = t; l < ncell; l += kMeshThreads) {
      const int x = (int)(l & (B - 1)), y = (int)((l >> blog) & (B - 1)), z = (int)(l >> (2 * blog));
      const unsigned pat = cell_pattern(sD, (z * E + y) * E + x, E);
      if (pat < 256u) cnt += (unsigned)mc_triangles(sMeta[pat]);
    }
    // CTA exclusive scan of the per-thread counts; one atomic places the block
    unsigned incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += y;
    }
    if (lane == 31) sWarp[w] = incl;
    __syncthreads();
    if (w == 0) {
      unsigned s = lane < kMeshWarps ? sWarp[lane] : 0u;
#pragma unroll
      for (int d = 1; d < kMeshWarps; d <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, s, d);
        if (lane >= d) s += y;
      }
      if (lane < kMeshWarps) sWarp[lane] = s;
      if (lane == kMeshWarps - 1) {
        const unsigned long long first = atomicAdd(&m.ctr->mesh_tris, (unsigned long long)s);
        sBase = first;
        if (i < o.block_cap) {
          MeshBlockRec rec;
          rec.key[0] = bc.x;
          rec.key[1] = bc.y;
          rec.key[2] = bc.z;
          rec.ntri = s;
          rec.first = (long long)first;
          o.blocks[i] = rec;
        }
      }
    }
    __syncthreads();
    if (cnt == 0u) continue;
    unsigned long long pos = sBase + (w ? sWarp[w - 1] : 0u) + (incl - cnt);
    for (unsigned l = t; l < ncell; l += kMeshThreads) {
      const int x = (int)(l & (B - 1)), y = (int)((l >> blog) & (B - 1)), z = (int)(l >> (2 * blog));
      const int cb = (z * E + y) * E + x;
      const unsigned pat = cell_pattern(sD, cb, E);
      if (pat >= 256u) continue;
      const McLoops L{sSeq[pat], sMeta[pat]};
      if (mc_triangles(L.meta) == 0) continue;
      const int gx = bc.x * B + x, gy = bc.y * B + y, gz = bc.z * B + z;
      auto Dc = [&](int c) { return sD[cb + (c & 1) + ((c >> 1) & 1) * E + (c >> 2) * EE]; };
      auto Pc = [&](int c, int q) {  // voxel centre coordinate, ((float)index + 1/2) v
        const int gq = q == 0 ? gx : (q == 1 ? gy : gz);
        return mc_mul(mc_add((float)(gq + ((c >> q) & 1)), 0.5f), v);
      };
      auto out = [&](int idx, const float* a, const float* b, const float* c) {
        if (pos < o.tri_cap) {
          o.cells[pos] = make_int4(gx, gy, gz, idx);
          float* dst = o.verts + 9 * pos;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            dst[q] = a[q];
            dst[3 + q] = b[q];
            dst[6 + q] = c[q];
          }
        }
        ++pos;
      };
      mc_emit(L, Dc, Pc, out);
    }
  }
}

__global__ void __launch_bounds__(kMeshThreads) k_mesh_clear(DevMap m) {
  const unsigned n = __ldcg(&m.ctr->mesh_blocks);
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m.mdirty[m.mlist[i]] = 0u;
}

int capped_grid(long long items, int threads, long long cap) {
  long long g = (items + threads - 1) / threads;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_mesh(const DevMap& m, bool all, const MeshOut& o, const LaunchCfg& cfg, LaunchHook* hook) {
  const cudaStream_t s = cfg.stream;
  hook->begin(kKMeshSelect, s);
  k_mesh_select<<<capped_grid(m.cap_blocks, kMeshThreads, (long long)cfg.num_sms * 8), kMeshThreads, 0, s>>>(m, all ? 1 : 0);
  hook->end(kKMeshSelect, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mesh_blocks, kMeshThreads, 0);
  if (e != cudaSuccess) return e;
  const long long grid = (long long)cfg.num_sms * (occ > 0 ? occ : 1);
  hook->begin(kKMeshBlocks, s);
  k_mesh_blocks<<<(int)(grid < (long long)m.cap_blocks ? grid : (long long)m.cap_blocks), kMeshThreads, 0, s>>>(m, o);
  hook->end(kKMeshBlocks, s);
  return cudaGetLastError();
}

cudaError_t launch_mesh_clear(const DevMap& m, const LaunchCfg& cfg, LaunchHook* hook) {
  hook->begin(kKMeshClear, cfg.stream);
  k_mesh_clear<<<capped_grid(m.cap_blocks, kMeshThreads, (long long)cfg.num_sms * 4), kMeshThreads, 0, cfg.stream>>>(m);
  hook->end(kKMeshClear, cfg.stream);
  return cudaGetLastError();
}

}  // namespace vbx
