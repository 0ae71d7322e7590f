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
//   k_mesh_blocks  one CTA per listed block (persistent grid), templated on the block edge:
//                  the block's D (coalesced) plus its one-voxel upper halo go to shared memory
//                  (NaN where unobserved) and become per-row bitmasks (inside, observed), from
//                  which each thread classifies one row of cells with shifts; a 256-entry
//                  topology table (computed once on the host, passed by value) gives the
//                  triangle counts of the cells that cross the surface; a CTA scan of
//                  (surface cells, triangles) and one 64-bit atomic place the block's triangles
//                  in one contiguous range; the surface cells are listed in output order and
//                  spread evenly over the threads, which write their triangles
//   k_mesh_clear   drops the stale marks of the listed blocks (launched only once the caller's
//                  buffers were large enough)
// Algorithmic traffic per listed block: (B + 1)^3 voxels of 8 B read, 52 B per triangle
// written (cell key 16 B, vertices 36 B), 24 B per block record.
#include <cuda_runtime.h>

#include <atomic>

#include "launch.h"
#include "mesh_cells.cuh"
#include "vbx_internal.cuh"

namespace vbx {

namespace {

constexpr int kMeshThreads = 256;  // also the number of topology table entries
constexpr int kMeshWarps = kMeshThreads / 32;
constexpr int kMaxDevices = 64;
constexpr int kMeshChunk = 512;  // triangles staged in shared memory per coalesced copy-out
constexpr size_t kMeshChunkBytes = (size_t)kMeshChunk * (sizeof(int4) + 9 * sizeof(float));  // dynamic smem
static_assert(kMeshThreads == 256, "one thread per inside/outside pattern copies the topology table");

__global__ void __launch_bounds__(kMeshThreads) k_mesh_select(DevMap m, int all) {
  const unsigned nb = min(__ldcg(&m.ctr->blocks), m.cap_blocks);
  const unsigned lane = threadIdx.x & 31u;
  const unsigned stride = gridDim.x * blockDim.x;
  // warp-uniform loop: the whole warp takes part in each ballot
  for (unsigned p0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); p0 < nb; p0 += stride) {
    const unsigned p = p0 + lane;
    bool need = false;
    if (p < nb) {
      // upper neighbours (dx, dy, dz) in {0, 1}^3 \ {0}: k = (dx+1)*9 + (dy+1)*3 + (dz+1); all
      // slots are requested together, then all marks
      const int kUp[7] = {14, 16, 17, 22, 23, 25, 26};
      uint32_t q[7];
#pragma unroll
      for (int j = 0; j < 7; ++j) q[j] = __ldg(&m.nbr[(size_t)p * 27 + kUp[j]]);
      need = all || m.mdirty[p];
#pragma unroll
      for (int j = 0; j < 7; ++j) need |= q[j] < m.cap_blocks && m.mdirty[q[j]];
    }
    const unsigned mask = __ballot_sync(0xffffffffu, need);
    unsigned base = 0u;
    if (lane == 0 && mask) base = atomicAdd(&m.ctr->mesh_blocks, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (need) m.mlist[base + __popc(mask & ((1u << lane) - 1u))] = p;
  }
}

// Topology of every inside/outside pattern, computed once on the host and passed by value.
struct McTable {
  unsigned long long seq[256];
  uint32_t meta[256];
};

const McTable& mc_table() {
  static const McTable tab = [] {
    McTable t{};
    for (unsigned p = 0; p < 256; ++p) {
      const McLoops L = mc_cell_loops(p);
      t.seq[p] = L.seq;
      t.meta[p] = L.meta;
    }
    return t;
  }();
  return tab;
}

template <int B>
struct MeshGeo {
  static constexpr int LOG = B == 4 ? 2 : (B == 8 ? 3 : 4);
  static constexpr int E = B + 1, EE = E * E, E3 = EE * E;
  static constexpr int CELLS = B * B * B;
  static constexpr int CELLS_PER_THREAD = (CELLS + kMeshThreads - 1) / kMeshThreads;
  static constexpr int HALO = 3 * B * B + 3 * B + 1;  // the upper faces, edges and corner
  static constexpr int HALO_PER_THREAD = (HALO + kMeshThreads - 1) / kMeshThreads;
  static_assert((1 << LOG) == B, "block edge must be 4, 8 or 16");
};

// Halo voxel h of a block: local coordinates in the neighbour block (lx, ly, lz), that block's
// offset o = ox + 2 oy + 4 oz, and its staged index in the (B + 1)^3 box.
template <int B>
__device__ __forceinline__ void halo_voxel(int h, int* local, int* o, int* staged) {
  using G = MeshGeo<B>;
  int lx = 0, ly = 0, lz = 0, off;
  if (h < B * B) {
    ly = h & (B - 1), lz = h >> G::LOG, off = 1;
  } else if (h < 2 * B * B) {
    h -= B * B, lx = h & (B - 1), lz = h >> G::LOG, off = 2;
  } else if (h < 3 * B * B) {
    h -= 2 * B * B, lx = h & (B - 1), ly = h >> G::LOG, off = 4;
  } else if (h < 3 * B * B + B) {
    lz = h - 3 * B * B, off = 3;
  } else if (h < 3 * B * B + 2 * B) {
    ly = h - 3 * B * B - B, off = 5;
  } else if (h < 3 * B * B + 3 * B) {
    lx = h - 3 * B * B - 2 * B, off = 6;
  } else {
    off = 7;
  }
  *local = (lz * B + ly) * B + lx;
  *o = off;
  *staged = ((lz + (off >> 2) * B) * G::E + ly + ((off >> 1) & 1) * B) * G::E + lx + (off & 1) * B;
}

__device__ __forceinline__ float observed_d(float2 dw) { return dw.y > 0.0f ? dw.x : __int_as_float(0x7fc00000); }

template <int B>
__global__ void __launch_bounds__(kMeshThreads, 3) k_mesh_blocks(DevMap m, MeshOut o, McTable tab) {
  using G = MeshGeo<B>;
  constexpr int E = G::E, EE = G::EE;
  __shared__ float sD[G::E3];
  __shared__ uint32_t sIn[G::EE];   // per staged row (z, y): bit x set if voxel x is inside
  __shared__ uint32_t sObs[G::EE];  // per staged row (z, y): bit x set if voxel x is observed
  __shared__ uint32_t sList[G::CELLS];  // surface cells in output order: cell | first triangle << 12
  extern __shared__ int4 sChunk[];  // one chunk of the block's triangles (kMeshChunkBytes)
  int4* sTriCell = sChunk;
  float* sTriVert = reinterpret_cast<float*>(sChunk + kMeshChunk);
  __shared__ unsigned long long sSeq[256];
  __shared__ uint32_t sMeta[256];
  __shared__ uint32_t sSlot[8];
  __shared__ unsigned sWarp[kMeshWarps];
  __shared__ unsigned long long sBase;
  const unsigned nsel = __ldcg(&m.ctr->mesh_blocks);
  if (blockIdx.x >= nsel) return;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  sSeq[t] = tab.seq[t];
  sMeta[t] = tab.meta[t];
  const float v = m.v;
  for (unsigned i = blockIdx.x; i < nsel; i += gridDim.x) {
    const uint32_t p = __ldcg(&m.mlist[i]);
    const int3 bc = m.bcoord[p];
    // the block's own voxels (coalesced) are requested before the neighbour slots arrive
    const float2* blk = m.tsdf + ((size_t)p << (3 * G::LOG));
    float2 in[G::CELLS_PER_THREAD];
#pragma unroll
    for (int j = 0; j < G::CELLS_PER_THREAD; ++j) {
      const int l = t + j * kMeshThreads;
      if (l < G::CELLS) in[j] = __ldg(&blk[l]);
    }
    // slot of the block at offset o = ox + 2 oy + 4 oz (kInvalid if absent)
    if (t < 8) sSlot[t] = t == 0 ? p : __ldg(&m.nbr[(size_t)p * 27 + 13 + (t & 1) * 9 + ((t >> 1) & 1) * 3 + (t >> 2)]);
    __syncthreads();  // also: the previous block's copy-out has finished with the shared buffers
    // ---- stage D (NaN where unobserved): the block's voxels, then the halo
    {
      float2 hv[G::HALO_PER_THREAD];
      int hs[G::HALO_PER_THREAD];
#pragma unroll
      for (int j = 0; j < G::HALO_PER_THREAD; ++j) {
        const int h = t + j * kMeshThreads;
        hs[j] = -1;
        hv[j] = make_float2(0.0f, 0.0f);
        if (h < G::HALO) {
          int local, off;
          halo_voxel<B>(h, &local, &off, &hs[j]);
          const uint32_t q = sSlot[off];
          if (q < m.cap_blocks) hv[j] = __ldg(&m.tsdf[((size_t)q << (3 * G::LOG)) | (uint32_t)local]);
        }
      }
#pragma unroll
      for (int j = 0; j < G::CELLS_PER_THREAD; ++j) {
        const int l = t + j * kMeshThreads;
        if (l < G::CELLS) sD[((l >> (2 * G::LOG)) * E + ((l >> G::LOG) & (B - 1))) * E + (l & (B - 1))] = observed_d(in[j]);
      }
#pragma unroll
      for (int j = 0; j < G::HALO_PER_THREAD; ++j)
        if (hs[j] >= 0) sD[hs[j]] = observed_d(hv[j]);
    }
    __syncthreads();
    // ---- row masks of the staged box (bit x of row (z, y) is voxel (x, y, z))
    for (int r = t; r < EE; r += kMeshThreads) {
      uint32_t in = 0u, ob = 0u;
#pragma unroll
      for (int x = 0; x < E; ++x) {
        const float d = sD[r * E + x];
        in |= (d < 0.0f ? 1u : 0u) << x;
        ob |= (isnan(d) ? 0u : 1u) << x;
      }
      sIn[r] = in;
      sObs[r] = ob;
    }
    __syncthreads();
    // ---- thread t < B^2 owns the cells of row (y, z) = (t % B, t / B), x = 0 .. B-1; a cell's
    // pattern takes bits x, x + 1 of the four rows (y or y+1, z or z+1)
    uint32_t r00 = 0u, r10 = 0u, r01 = 0u, r11 = 0u, obs = 0u;
    if (t < B * B) {
      const int y = t & (B - 1), z = t >> G::LOG, r = z * E + y;
      r00 = sIn[r], r10 = sIn[r + 1], r01 = sIn[r + E], r11 = sIn[r + E + 1];
      obs = sObs[r] & sObs[r + 1] & sObs[r + E] & sObs[r + E + 1];
      obs &= obs >> 1;  // bit x: voxels x and x + 1 of all four rows observed
    }
    auto row_pattern = [&](int x) {
      return ((r00 >> x) & 3u) | (((r10 >> x) & 3u) << 2) | (((r01 >> x) & 3u) << 4) | (((r11 >> x) & 3u) << 6);
    };
    unsigned packed = 0u;  // (surface cells << 16) | triangles of this thread's cells
#pragma unroll
    for (int x = 0; x < B; ++x) {
      const unsigned pat = row_pattern(x);
      if (((obs >> x) & 1u) && pat != 0u && pat != 255u) {
        const unsigned nt = (unsigned)mc_triangles(sMeta[pat]);
        if (nt) packed += (1u << 16) | nt;
      }
    }
    // CTA exclusive scan (a block has at most 4096 surface cells and 49152 triangles, so the
    // two fields never carry into each other)
    unsigned incl = packed;
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
    }
    __syncthreads();
    const unsigned total = sWarp[kMeshWarps - 1];
    const unsigned ntri = total & 0xffffu, nsurf = total >> 16;
    // one atomic places the block; its result is needed only at the first copy-out
    unsigned long long first = 0ull;
    if (t == 0) first = atomicAdd(&m.ctr->mesh_tris, (unsigned long long)ntri);
    // ---- list the surface cells in output order
    if (packed) {
      const unsigned excl = (w ? sWarp[w - 1] : 0u) + incl - packed;
      unsigned sp = excl >> 16, tp = excl & 0xffffu;
#pragma unroll
      for (int x = 0; x < B; ++x) {
        const unsigned pat = row_pattern(x);
        if (!((obs >> x) & 1u) || pat == 0u || pat == 255u) continue;
        const unsigned nt = (unsigned)mc_triangles(sMeta[pat]);
        if (!nt) continue;
        sList[sp++] = (unsigned)((t << G::LOG) | x) | (tp << 12);
        tp += nt;
      }
    }
    __syncthreads();
    if (t == 0) {
      sBase = first;
      if (i < o.block_cap) {
        MeshBlockRec rec;
        rec.key[0] = bc.x;
        rec.key[1] = bc.y;
        rec.key[2] = bc.z;
        rec.ntri = ntri;
        rec.first = (long long)first;
        o.blocks[i] = rec;
      }
    }
    // ---- triangles, one chunk at a time: the surface cells spread evenly over the threads
    // write into shared memory at block-relative positions, then the CTA copies the chunk out
    // with coalesced stores (a cell whose triangles straddle two chunks is evaluated twice)
    for (unsigned c0 = 0; c0 < ntri; c0 += kMeshChunk) {
      for (unsigned k = (unsigned)t; k < nsurf; k += kMeshThreads) {
        const uint32_t ent = sList[k];
        const int l = (int)(ent & 4095u);
        const int x = l & (B - 1), y = (l >> G::LOG) & (B - 1), z = l >> (2 * G::LOG);
        const int cb = (z * E + y) * E + x, r = z * E + y;
        const unsigned pat = ((sIn[r] >> x) & 3u) | (((sIn[r + 1] >> x) & 3u) << 2) | (((sIn[r + E] >> x) & 3u) << 4) |
                             (((sIn[r + E + 1] >> x) & 3u) << 6);
        const McLoops L{sSeq[pat], sMeta[pat]};
        const unsigned q0 = ent >> 12;  // block-relative index of the cell's first triangle
        if (q0 >= c0 + kMeshChunk || q0 + (unsigned)mc_triangles(L.meta) <= c0) continue;
        const int gx = bc.x * B + x, gy = bc.y * B + y, gz = bc.z * B + z;
        // the cell's corner coordinates, voxel centres ((float)index + 1/2) v
        const float x0 = mc_mul(mc_add((float)gx, 0.5f), v), x1 = mc_mul(mc_add((float)(gx + 1), 0.5f), v);
        const float y0 = mc_mul(mc_add((float)gy, 0.5f), v), y1 = mc_mul(mc_add((float)(gy + 1), 0.5f), v);
        const float z0 = mc_mul(mc_add((float)gz, 0.5f), v), z1 = mc_mul(mc_add((float)(gz + 1), 0.5f), v);
        auto Dc = [&](int c) { return sD[cb + (c & 1) + ((c >> 1) & 1) * E + (c >> 2) * EE]; };
        auto Pc = [&](int c, int a) { return a == 0 ? ((c & 1) ? x1 : x0) : (a == 1 ? ((c & 2) ? y1 : y0) : ((c & 4) ? z1 : z0)); };
        auto out = [&](int idx, int slot, const float* wv) {
          const unsigned qq = q0 + (unsigned)idx;
          if (qq >= c0 && qq < c0 + kMeshChunk) {
            const unsigned sl = qq - c0;
            if (slot == 0) sTriCell[sl] = make_int4(gx, gy, gz, idx);
            float* dst = sTriVert + 9 * sl + 3 * slot;
            dst[0] = wv[0];
            dst[1] = wv[1];
            dst[2] = wv[2];
          }
        };
        mc_emit(L, Dc, Pc, out);
      }
      __syncthreads();
      const unsigned long long g0 = sBase + c0;
      // triangles past the caller's capacity are dropped (the call then reports the size needed)
      const unsigned long long room = g0 < o.tri_cap ? o.tri_cap - g0 : 0ull;
      const unsigned n = (unsigned)min((unsigned long long)min((unsigned)kMeshChunk, ntri - c0), room);
      int4* dc = o.cells + g0;
      float* dv = o.verts + 9ull * g0;
      for (unsigned j = (unsigned)t; j < n; j += kMeshThreads) dc[j] = sTriCell[j];
      for (unsigned j = (unsigned)t; j < 9u * n; j += kMeshThreads) dv[j] = sTriVert[j];
      __syncthreads();
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

template <int B>
cudaError_t launch_mesh_blocks(const DevMap& m, const MeshOut& o, const LaunchCfg& cfg) {
  // the shared-memory opt-in is per device; it and the occupancy do not depend on the map
  static std::atomic<int> occ_of_device[kMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  int occ = dev < kMaxDevices ? occ_of_device[dev].load() : 0;
  if (occ <= 0) {
    e = cudaFuncSetAttribute(k_mesh_blocks<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMeshChunkBytes);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mesh_blocks<B>, kMeshThreads, kMeshChunkBytes);
    if (e != cudaSuccess) return e;
    if (occ <= 0) occ = 1;
    if (dev < kMaxDevices) occ_of_device[dev].store(occ);
  }
  long long grid = (long long)cfg.num_sms * occ;
  if (grid > (long long)m.cap_blocks) grid = m.cap_blocks;
  k_mesh_blocks<B><<<(int)grid, kMeshThreads, kMeshChunkBytes, cfg.stream>>>(m, o, mc_table());
  return cudaGetLastError();
}

cudaError_t launch_mesh(const DevMap& m, bool all, const MeshOut& o, const LaunchCfg& cfg, LaunchHook* hook) {
  const cudaStream_t s = cfg.stream;
  hook->begin(kKMeshSelect, s);
  k_mesh_select<<<capped_grid(m.cap_blocks, kMeshThreads, (long long)cfg.num_sms * 8), kMeshThreads, 0, s>>>(m, all ? 1 : 0);
  hook->end(kKMeshSelect, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  hook->begin(kKMeshBlocks, s);
  e = m.B == 4 ? launch_mesh_blocks<4>(m, o, cfg) : m.B == 8 ? launch_mesh_blocks<8>(m, o, cfg) : launch_mesh_blocks<16>(m, o, cfg);
  hook->end(kKMeshBlocks, s);
  return e;
}

cudaError_t launch_mesh_clear(const DevMap& m, const LaunchCfg& cfg, LaunchHook* hook) {
  hook->begin(kKMeshClear, cfg.stream);
  k_mesh_clear<<<capped_grid(m.cap_blocks, kMeshThreads, (long long)cfg.num_sms * 4), kMeshThreads, 0, cfg.stream>>>(m);
  hook->end(kKMeshClear, cfg.stream);
  return cudaGetLastError();
}

}  // namespace vbx
