// integrate.cu -- TSDF integration of one posed scan (Sec. IV of Oleynikova et al. 2017):
//   k_bin_points     A1+A2  transform, filter, voxel key; grouped raycasting bins points into
//                           a per-scan hash table with exact integer sums (order-independent)
//   k_group_rays     A2+A3  group mean and weight -> one ray per group; block-level DDA over
//                           the ray and lock-free insertion of its blocks into the block hash,
//                           and a per-scan scratch block for every block the ray enters
//   k_link_blocks    A3     26-neighbour links of the new blocks (O(1) neighbour access later);
//                           pool slot <-> scratch block of the blocks entered this scan, whose
//                           meshes it marks stale
//   k_integrate_rays A4     voxel-level integer DDA; Eq. (1) distance, Eq. (2)/(4) weight;
//                           per-voxel sums of w and w*d as exact two-part fixed point numbers
//                           with integer atomics into the scratch blocks, pre-aggregated across
//                           the warp (order-independent, so the result does not depend on
//                           scheduling)
//   k_apply          A5     Eq. (3) merge of each voxel that received records (one thread per
//                           voxel of a scratch block); queues it for the ESDF
// All float32 arithmetic that decides a set (keys, endpoints, visited voxels, w > 0) uses
// explicitly rounded intrinsics, so the compiler cannot contract or reorder it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include <cooperative_groups.h>

#include "launch.h"
#include "vbx_internal.cuh"

namespace cg = cooperative_groups;

namespace vbx {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
static_assert(kThreads >= kMaxBatch, "one thread per map of a batch builds the per-map prefix");
constexpr unsigned kFull = 0xffffffffu;
// Long rays are traversed in segments spread over the lanes of a warp (DdaSeg): a voxel
// segment ends at every kVoxSeg-th crossing of the ray's dominant axis, a block segment at
// every kBlkSeg-th.
#ifndef VBX_VOX_SEG
#define VBX_VOX_SEG 16
#endif
#ifndef VBX_SEG_FILL
#define VBX_SEG_FILL 64
#endif
// The voxel walk keeps about 106 registers live. A single map's rays are cut into segments
// spread over the lanes: there 2 CTAs per SM without spills beat 4 CTAs per SM at 64 registers
// (about 150 B of spills per thread) by 12 % on the LiDAR sequence. A large batch's rays are
// walked whole, one per lane, and more warps in flight win: 4 CTAs per SM (3.1 against 3.9 ms
// on the 64-map mix).
#ifndef VBX_RAYS_MIN_CTAS
#define VBX_RAYS_MIN_CTAS 2
#endif
#ifndef VBX_RAYS_MIN_CTAS_BATCH
#define VBX_RAYS_MIN_CTAS_BATCH 4
#endif
constexpr int kVoxSeg = VBX_VOX_SEG;
constexpr int kBlkSeg = 4;
constexpr unsigned kSegFill = VBX_SEG_FILL;  // segments per 32 lanes aimed at by a warp task

// Segment bookkeeping of the 32 rays of a warp: lane `lane` holds nseg segments of its ray.
// Returns the warp's total and this lane's first segment index.
__device__ __forceinline__ int warp_segments(int nseg, int lane, int* first) {
  int incl = nseg;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int up = __shfl_up_sync(kFull, incl, off);
    if (lane >= off) incl += up;
  }
  *first = incl - nseg;
  return __shfl_sync(kFull, incl, 31);
}

// Whether the rays of a launch are cut into segments: only when 32-ray warp tasks would not
// keep every resident warp busy several times over (then the longest ray of a warp sets the
// kernel's duration); with plenty of rays each lane walks its whole ray.
#ifndef VBX_SPLIT_TASKS_PER_WARP
#define VBX_SPLIT_TASKS_PER_WARP 4
#endif
__device__ __forceinline__ bool split_rays(unsigned n, unsigned slots) {
  return (unsigned long long)n < 32ull * VBX_SPLIT_TASKS_PER_WARP * slots;
}

// Rays per warp task when rays are split (a power of two in [1, 32]): at most n / slots, so
// that n rays keep `slots` resident warps busy, and (when the segment total sg is known) about
// as many rays as give two segments per lane.
__device__ __forceinline__ unsigned rays_per_task(unsigned n, unsigned long long sg, unsigned slots) {
  unsigned R = 32;
  while (R > 1 && (unsigned long long)n < (unsigned long long)R * slots) R >>= 1;
  if (sg > 0)
    while (R > 1 && (unsigned long long)R * sg > (unsigned long long)kSegFill * n) R >>= 1;
  return R;
}

// Lane whose ray holds warp segment t: the last lane whose first segment index is <= t.
__device__ __forceinline__ int segment_owner(int first, int t) {
  int own = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    const int e = __shfl_sync(kFull, first, own + step);
    if (e <= t) own += step;
  }
  return own;
}

// A1 filter and per-point weight. Returns false for a dropped point.
__device__ __forceinline__ bool accept_point(const DevMap& m, float x, float y, float z, float* w) {
  if (!isfinite(x) || !isfinite(y) || !isfinite(z)) return false;
  const float r2 = __fadd_rn(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)), __fmul_rn(z, z));
  if (!(r2 > 0.0f)) return false;
  if (!(r2 < m.range_lim2)) return false;
  if (m.max_range2 > 0.0f && r2 > m.max_range2) return false;
  if (m.weighting == 1) {
    if (!(z > 0.0f)) return false;
    const float wi = __fdiv_rn(1.0f, __fmul_rn(z, z));  // Eq. (4): 1/z^2, z = depth in the sensor frame
    if (!(wi <= 1024.0f)) return false;
    *w = wi;
  } else {
    *w = 1.0f;
  }
  return true;
}

// floor((hi * 2^64 + lo) / d) for a quotient known to be below 2^17.
__device__ __forceinline__ unsigned div128_small(unsigned long long lo, unsigned long long hi, unsigned long long d) {
  if (hi == 0) return (unsigned)(lo / d);
  unsigned q = 0;
  for (int b = 16; b >= 0; --b) {
    const unsigned long long dl = d << b;
    const unsigned long long dh = b ? (d >> (64 - b)) : 0ull;
    if (hi > dh || (hi == dh && lo >= dl)) {
      const unsigned long long borrow = lo < dl ? 1ull : 0ull;
      lo -= dl;
      hi = hi - dh - borrow;
      q |= 1u << b;
    }
  }
  return q;
}

// ---- batch addressing: work items of all maps are concatenated; each CTA builds the exclusive
// prefix of the per-map counts in shared memory and finds an item's map by binary search.

__device__ __forceinline__ const DevMap& map_of(const Batch& b, unsigned mi) { return b.maps ? b.maps[mi] : b.one; }
__device__ __forceinline__ const ScanDesc& scan_of(const Batch& b, unsigned mi) { return b.scans ? b.scans[mi] : b.one_scan; }

template <typename F>
__device__ __forceinline__ unsigned cta_prefix(unsigned* pfx, const Batch& b, F count) {
  const int nm = b.maps ? b.nmaps : 1;
  const int t = threadIdx.x;
  if (nm == 1) {
    if (t == 0) {
      pfx[0] = 0u;
      pfx[1] = count(0u);
    }
    __syncthreads();
    return pfx[1];
  }
  // every thread reads one map's count; warp 0 scans them (kMaxBatch / 32 per lane)
  pfx[t + 1] = t < nm ? count((unsigned)t) : 0u;
  __syncthreads();
  if (t < 32) {
    constexpr int per = kMaxBatch / 32;
    unsigned v[per];
    unsigned sum = 0;
#pragma unroll
    for (int j = 0; j < per; ++j) {
      v[j] = pfx[t * per + j + 1];
      sum += v[j];
    }
    unsigned incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned up = __shfl_up_sync(kFull, incl, off);
      if (t >= off) incl += up;
    }
    unsigned run = incl - sum;
    if (t == 0) pfx[0] = 0u;
#pragma unroll
    for (int j = 0; j < per; ++j) {
      run += v[j];
      pfx[t * per + j + 1] = run;
    }
  }
  __syncthreads();
  return pfx[nm];
}

__device__ __forceinline__ unsigned map_index(const unsigned* pfx, int nm, unsigned i) {
  int lo = 0, hi = nm - 1;  // largest mi with pfx[mi] <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pfx[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  return (unsigned)lo;
}

__device__ __forceinline__ int nmaps_of(const Batch& b) { return b.maps ? b.nmaps : 1; }

__global__ void __launch_bounds__(kThreads) k_init_groups(GroupEntry* tab, uint32_t entries) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < entries; i += gridDim.x * blockDim.x) {
    GroupEntry e;
    e.key = kEmptyKey;
    e.sw = 0;
    e.swo_lo[0] = e.swo_lo[1] = e.swo_lo[2] = 0;
    e.swo_hi[0] = e.swo_hi[1] = e.swo_hi[2] = 0;
    e.n = 0;
    tab[i] = e;
  }
}

__global__ void __launch_bounds__(kThreads) k_reset_counters(Batch b) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nmaps_of(b); i += gridDim.x * blockDim.x) {
    Counters* c = map_of(b, i).ctr;
    c->ngroups = 0;
    c->nnew = 0;
    c->nupdated = 0;
    c->npoints_valid = 0;
    c->ntouched = 0;
    c->nvseg = 0;
    c->nrecords = 0;
    c->raise_rounds = 0;
    c->lower_rounds = 0;
    c->raise_pops = 0;
    c->lower_pops = 0;
    c->seeds = 0;
    c->esdf_in = 0;
    c->esdf_block_visits = 0;
    c->esdf_local_iters = 0;
    c->esdf_phase_ns[0] = c->esdf_phase_ns[1] = c->esdf_phase_ns[2] = 0;
  }
}

// ------------------------------------------------------------------------------- A1 + A2
__global__ void __launch_bounds__(kThreads) k_bin_points(Batch b) {
  __shared__ unsigned pfx[kMaxBatch + 1];
  __shared__ unsigned long long sh_w[kWarps][32];
  __shared__ unsigned long long sh_o[3][kWarps][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nm = nmaps_of(b);
  const unsigned total = cta_prefix(pfx, b, [&](unsigned mi) { return scan_of(b, mi).n; });
  const unsigned stride = gridDim.x * blockDim.x;
  for (unsigned base = blockIdx.x * blockDim.x; base < total; base += stride) {
    const unsigned i = base + threadIdx.x;
    bool valid = false;
    unsigned mi = 0;
    unsigned long long key = kEmptyKey;
    unsigned long long wq = 0, o[3] = {0, 0, 0};
    float pw[3] = {0.f, 0.f, 0.f};
    float w = 0.0f;
    if (i < total) {
      mi = map_index(pfx, nm, i);
      const DevMap& m = map_of(b, mi);
      const ScanDesc& sd = scan_of(b, mi);
      const unsigned j = i - pfx[mi];
      const float x = __ldg(&sd.pts[3 * (size_t)j + 0]);
      const float y = __ldg(&sd.pts[3 * (size_t)j + 1]);
      const float z = __ldg(&sd.pts[3 * (size_t)j + 2]);
      if (accept_point(m, x, y, z, &w)) {
        bool in_range = true;
        float q[3];
        for (int r = 0; r < 3; ++r) {
          pw[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(sd.T[4 * r], x), __fmul_rn(sd.T[4 * r + 1], y)),
                                      __fmul_rn(sd.T[4 * r + 2], z)),
                            sd.T[4 * r + 3]);
          q[r] = __fdiv_rn(pw[r], m.v);
          if (!(fabsf(q[r]) < 1048576.0f)) in_range = false;
        }
        if (in_range) {
          valid = true;
          int k[3];
          for (int r = 0; r < 3; ++r) {
            const float fq = floorf(q[r]);
            k[r] = (int)fq;
            long long oo = __float2ll_rn(__fmul_rn(__fsub_rn(q[r], fq), 65536.0f));
            o[r] = (unsigned long long)(oo > 65535 ? 65535 : oo);
          }
          key = pack_key(k[0], k[1], k[2]);
          wq = m.weighting == 0 ? 1ull : (unsigned long long)__float2ll_rn(__fmul_rn(w, 1048576.0f));
        }
      }
      if (valid && !m.grouped) {  // one ray per point
        const unsigned r = atomicAdd(&m.ctr->ngroups, 1u);
        m.rays[r] = make_float4(pw[0], pw[1], pw[2], w);
      }
    }
    // accepted points, counted once per warp and map
    const unsigned mpeers = __match_any_sync(kFull, mi);
    const unsigned vmask = __ballot_sync(kFull, valid);
    if (lane == __ffs(mpeers) - 1 && (vmask & mpeers)) atomicAdd(&map_of(b, mi).ctr->npoints_valid, (unsigned)__popc(vmask & mpeers));
    if (valid && !map_of(b, mi).grouped) {
      valid = false;
      key = kEmptyKey;
    }
    // warp pre-aggregation of points of one map that share a voxel (neighbouring pixels usually do)
    const unsigned peers = __match_any_sync(kFull, key) & mpeers;
    const int leader = __ffs(peers) - 1;
    sh_w[wid][lane] = wq;
    for (int r = 0; r < 3; ++r) sh_o[r][wid][lane] = wq * o[r];
    __syncwarp();
    if (valid && lane == leader) {
      const DevMap& m = map_of(b, mi);
      unsigned long long sw = 0, so[3] = {0, 0, 0};
      for (unsigned pm = peers; pm; pm &= pm - 1) {
        const int src = __ffs(pm) - 1;
        sw += sh_w[wid][src];
        for (int r = 0; r < 3; ++r) so[r] += sh_o[r][wid][src];
      }
      uint32_t h = hash64(key) & m.gmask;
      bool placed = false;
      for (uint32_t probe = 0; probe <= m.gmask; ++probe) {
        unsigned long long k = __ldcg(&m.gtab[h].key);
        if (k == kEmptyKey) {
          k = atomicCAS(&m.gtab[h].key, kEmptyKey, key);
          if (k == kEmptyKey) {
            const unsigned gi = atomicAdd(&m.ctr->ngroups, 1u);
            m.glist[gi] = h;
            placed = true;
            break;
          }
        }
        if (k == key) {
          placed = true;
          break;
        }
        h = (h + 1) & m.gmask;
      }
      if (placed) {
        GroupEntry* e = &m.gtab[h];
        atomicAdd(&e->n, (unsigned)__popc(peers));
        atomicAdd(&e->sw, sw);
        for (int r = 0; r < 3; ++r) {
          const unsigned long long old = atomicAdd(&e->swo_lo[r], so[r]);
          if (old + so[r] < old) atomicAdd(&e->swo_hi[r], 1u);
        }
      } else {
        atomicOr(&m.ctr->error, kErrGroupTable);
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------- A2 + A3
// The first ray of scan `ep` that enters the block of hash entry h gives the block a scratch
// block for the scan's sums (an entry's claim epoch only grows, so no reset pass is needed).
__device__ __forceinline__ void claim_scratch(const DevMap& m, uint32_t h, unsigned ep) {
  if (h == kInvalid || __ldcg(&m.hclaim[h]) == ep) return;
  if (atomicExch(&m.hclaim[h], ep) == ep) return;
  const unsigned i = atomicAdd(&m.ctr->ntouched, 1u);
  if (i < m.scr_cap)
    m.slist_h[i] = h;
  else
    atomicOr(&m.ctr->error, kErrScratchFull);
}

// Scratch blocks usable by this scan: none if the scan entered more blocks than the scratch
// holds (the scan is then rejected as a whole and the map keeps its previous state).
__device__ __forceinline__ unsigned scratch_blocks(const DevMap& m) {
  const unsigned n = __ldcg(&m.ctr->ntouched);
  return n <= m.scr_cap ? n : 0u;
}

__global__ void __launch_bounds__(kThreads) k_group_rays(Batch b, unsigned warp_slots) {
  __shared__ unsigned pfx[kMaxBatch + 1];
  __shared__ long long sh_se[kWarps][32][6];  // each lane's ray ends S, E (fixed point)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nm = nmaps_of(b);
  // warp tasks of R rays of one map; their block-traversal segments are spread over the lanes
  const unsigned nall = cta_prefix(pfx, b, [&](unsigned mi) { return __ldcg(&map_of(b, mi).ctr->ngroups); });
  const bool split = split_rays(nall, warp_slots);
  const unsigned R = split ? rays_per_task(nall, 0, warp_slots) : 32u;
  const int K = split ? kBlkSeg : (1 << 30);
  __syncthreads();
  const unsigned ntask = cta_prefix(pfx, b, [&](unsigned mi) { return (__ldcg(&map_of(b, mi).ctr->ngroups) + R - 1) / R; });
  for (unsigned task = blockIdx.x * kWarps + wid; task < ntask; task += gridDim.x * kWarps) {
    const unsigned mi = map_index(pfx, nm, task);
    const DevMap& m = map_of(b, mi);
    const ScanDesc& sd = scan_of(b, mi);
    const unsigned gi = (task - pfx[mi]) * R + lane;
    int nseg = 0, nvseg = 0;
    if (lane < (int)R && gi < __ldcg(&m.ctr->ngroups)) {
      const float s[3] = {sd.T[3], sd.T[7], sd.T[11]};
      float pbar[3];
      if (m.grouped) {
        const uint32_t h = m.glist[gi];
        GroupEntry e = m.gtab[h];
        GroupEntry z;  // reset the entry for the next scan
        z.key = kEmptyKey;
        z.sw = 0;
        z.swo_lo[0] = z.swo_lo[1] = z.swo_lo[2] = 0;
        z.swo_hi[0] = z.swo_hi[1] = z.swo_hi[2] = 0;
        z.n = 0;
        m.gtab[h] = z;
        const int3 k = unpack_key(e.key);
        const int kk[3] = {k.x, k.y, k.z};
        const unsigned long long half = e.sw >> 1;
        for (int a = 0; a < 3; ++a) {
          const unsigned long long lo = e.swo_lo[a] + half;
          const unsigned long long hi = (unsigned long long)e.swo_hi[a] + (lo < half ? 1ull : 0ull);
          const unsigned mo = div128_small(lo, hi, e.sw);
          pbar[a] = __fmul_rn(__fadd_rn((float)kk[a], __fmul_rn((float)mo, 1.0f / 65536.0f)), m.v);
        }
        const float Wg = m.weighting == 0 ? __uint2float_rn(e.n) : __fmul_rn(__ull2float_rn(e.sw), 1.0f / 1048576.0f);
        m.rays[gi] = make_float4(pbar[0], pbar[1], pbar[2], Wg);
      } else {
        const float4 r = m.rays[gi];
        pbar[0] = r.x;
        pbar[1] = r.y;
        pbar[2] = r.z;
      }
      RayGeom g;
      if (ray_setup(pbar, s, m.v, m.delta, &g)) {
        // block-level traversal: cells of 65536*B fixed-point units; same crossing order as
        // the voxel traversal, so it visits exactly the blocks of the traversed voxels
        DdaSeg sg;
        sg.init(g.S, g.E, 16 + m.blog);
        nseg = sg.segments(K);
        DdaSeg sv;  // segments of the voxel traversal (sizes the next kernel's warp tasks)
        sv.init(g.S, g.E, 16);
        nvseg = sv.segments(kVoxSeg);
        for (int a = 0; a < 3; ++a) {
          sh_se[wid][lane][a] = g.S[a];
          sh_se[wid][lane][3 + a] = g.E[a];
        }
      }
    }
    int vs = nvseg;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) vs += __shfl_xor_sync(kFull, vs, off);
    if (lane == 0 && vs) atomicAdd(&m.ctr->nvseg, (unsigned)vs);
    __syncwarp();
    int first = 0;
    const int tot = warp_segments(nseg, lane, &first);
    const unsigned ep = sd.epoch;
    for (int t0 = 0; t0 < tot; t0 += 32) {
      const int t = t0 + lane;
      const int own = segment_owner(first, t);
      const int seg = t - __shfl_sync(kFull, first, own);
      if (t >= tot) continue;
      DdaSeg sg;
      sg.init(&sh_se[wid][own][0], &sh_se[wid][own][3], 16 + m.blog);
      int left = 0;
      Dda dda = sg.seek(seg, K, &left);
      claim_scratch(m, block_insert(m, dda.cx, dda.cy, dda.cz), ep);
      for (int dk = 0; left > 0;) {
        const int ax = dda.step();
        --left;
        if (ax == sg.d && ++dk == K) break;
        claim_scratch(m, block_insert(m, dda.cx, dda.cy, dda.cz), ep);
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------ A3
__global__ void __launch_bounds__(kThreads) k_link_blocks(Batch b) {
  __shared__ unsigned pfx[kMaxBatch + 1];
  const int nm = nmaps_of(b);
  // one thread per (new block, direction), then one per scratch block of the scan
  const unsigned total = cta_prefix(pfx, b, [&](unsigned mi) {
    const DevMap& m = map_of(b, mi);
    return __ldcg(&m.ctr->nnew) * 27u + scratch_blocks(m);
  });
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const unsigned mi = map_index(pfx, nm, t);
    const DevMap& m = map_of(b, mi);
    const unsigned nl = __ldcg(&m.ctr->nnew) * 27u;
    const unsigned u = t - pfx[mi];
    if (u >= nl) {  // scratch block i <-> pool slot (the slots were published by k_group_rays)
      const unsigned i = u - nl;
      const uint32_t slot = __ldcg(&m.hvals[m.slist_h[i]]);
      m.slist[i] = slot;
      if (slot < m.cap_blocks) {
        m.sinfo[slot] = ((unsigned long long)scan_of(b, mi).epoch << 32) | i;
        m.mdirty[slot] = 1u;  // the scan may change the block's TSDF: its mesh is stale
      }
      continue;
    }
    const uint32_t p = m.newblk[u / 27u];
    if (p >= m.cap_blocks) continue;
    const int k = (int)(u % 27u);
    if (k == 13) {
      m.nbr[(size_t)p * 27 + 13] = p;
      continue;
    }
    const int3 bc = m.bcoord[p];
    const uint32_t q = block_lookup(m, bc.x + k / 9 - 1, bc.y + (k / 3) % 3 - 1, bc.z + k % 3 - 1);
    m.nbr[(size_t)p * 27 + k] = q;
    if (q != kInvalid) m.nbr[(size_t)q * 27 + (26 - k)] = p;
  }
}

// The scratch block of each neighbour of every scratch block of the scan, so that a ray stepping
// into the next block needs one load of a table its lane prefetched, not a chain of two (the
// neighbour's pool slot, then that slot's scratch block).
__global__ void __launch_bounds__(kThreads) k_scratch_links(Batch b) {
  __shared__ unsigned pfx[kMaxBatch + 1];
  const int nm = nmaps_of(b);
  const unsigned total = cta_prefix(pfx, b, [&](unsigned mi) { return scratch_blocks(map_of(b, mi)) * 27u; });
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const unsigned mi = map_index(pfx, nm, t);
    const DevMap& m = map_of(b, mi);
    const unsigned u = t - pfx[mi];
    const unsigned i = u / 27u, k = u % 27u;
    const uint32_t slot = __ldcg(&m.slist[i]);
    uint32_t sb = kInvalid;
    if (slot < m.cap_blocks) {
      const uint32_t q = k == 13 ? slot : __ldcg(&m.nbr[(size_t)slot * 27 + k]);
      if (q != kInvalid && q < m.cap_blocks) {
        const unsigned long long w = __ldcg(&m.sinfo[q]);
        if ((unsigned)(w >> 32) == scan_of(b, mi).epoch) sb = (uint32_t)w;
      }
    }
    m.snbr[(size_t)i * 27 + k] = sb;
  }
}

// ------------------------------------------------------------------------------------ A4
// Splits a float32 record into its exact two-part fixed-point representation.
__device__ __forceinline__ void fx_split(float x, long long* hi, long long* lo) {
  const float q = __fmul_rn(x, kAccScale);  // exact (power-of-two scaling)
  const float t = truncf(q);
  *hi = (long long)t;
  *lo = __float2ll_rn(__fmul_rn(__fsub_rn(q, t), kAccLoScale));
}

// The four parts are fire-and-forget reductions (no returned value), so the ray loop never
// waits on an atomic; the touch flag is a plain byte store (all writers store 1).
__device__ __forceinline__ void accumulate(const DevMap& m, uint32_t sv, const long long v[4]) {
  unsigned long long* a = &m.sacc[4 * (size_t)sv];
  for (int j = 0; j < 4; ++j)
    if (v[j] != 0) atomicAdd(&a[j], (unsigned long long)v[j]);
  m.stouch[sv] = 1u;
}

// Scratch block of pool slot `slot` in scan ep (kInvalid if the scan has none for it).
__device__ __forceinline__ uint32_t scratch_of(const DevMap& m, uint32_t slot, unsigned ep) {
  if (slot == kInvalid) return kInvalid;
  const unsigned long long w = __ldcg(&m.sinfo[slot]);
  return (unsigned)(w >> 32) == ep ? (uint32_t)w : kInvalid;
}

template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_integrate_rays(Batch b, unsigned warp_slots) {
  __shared__ unsigned pfx[kMaxBatch + 1];
  __shared__ long long sh_v[4][kWarps][32];
  __shared__ long long sh_se[kWarps][32][6];  // each lane's ray ends S, E (fixed point)
  __shared__ float sh_pg[kWarps][32][7];      // pbar, pbar - s, group weight
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nm = nmaps_of(b);
  // a map whose scan overflowed its scratch integrates nothing
  auto rays_of = [&](unsigned mi) {
    const DevMap& m = map_of(b, mi);
    return __ldcg(&m.ctr->ntouched) <= m.scr_cap ? __ldcg(&m.ctr->ngroups) : 0u;
  };
  // warp tasks of R rays of one map; their voxel-traversal segments are spread over the lanes
  const unsigned nall = cta_prefix(pfx, b, rays_of);
  __syncthreads();
  const unsigned sall = cta_prefix(pfx, b, [&](unsigned mi) { return rays_of(mi) ? __ldcg(&map_of(b, mi).ctr->nvseg) : 0u; });
  const bool split = split_rays(nall, warp_slots);
  const unsigned R = split ? rays_per_task(nall, sall, warp_slots) : 32u;
  const int K = split ? kVoxSeg : (1 << 30);
  __syncthreads();
  const unsigned ntask = cta_prefix(pfx, b, [&](unsigned mi) { return (rays_of(mi) + R - 1) / R; });
  unsigned long long nrec = 0;
  unsigned rec_map = 0;
  for (unsigned task = blockIdx.x * kWarps + wid; task < ntask; task += gridDim.x * kWarps) {
    const unsigned mi = map_index(pfx, nm, task);
    const DevMap& m = map_of(b, mi);
    const ScanDesc& sd = scan_of(b, mi);
    if (nrec && mi != rec_map) {
      atomicAdd(&map_of(b, rec_map).ctr->nrecords, nrec);
      nrec = 0;
    }
    rec_map = mi;
    const float s[3] = {sd.T[3], sd.T[7], sd.T[11]};
    const unsigned ep = sd.epoch;
    const int B = m.B, blog = m.blog;
    const unsigned gi = (task - pfx[mi]) * R + lane;
    int nseg = 0;
    if (lane < (int)R && gi < rays_of(mi)) {
      const float4 r = m.rays[gi];
      const float pbar[3] = {r.x, r.y, r.z};
      RayGeom g;
      if (ray_setup(pbar, s, m.v, m.delta, &g)) {
        DdaSeg sg;
        sg.init(g.S, g.E, 16);
        nseg = sg.segments(K);
        for (int a = 0; a < 3; ++a) {
          sh_se[wid][lane][a] = g.S[a];
          sh_se[wid][lane][3 + a] = g.E[a];
          sh_pg[wid][lane][a] = g.p[a];
          sh_pg[wid][lane][3 + a] = g.g[a];
        }
        sh_pg[wid][lane][6] = r.w;
      }
    }
    __syncwarp();
    int first = 0;
    const int tot = warp_segments(nseg, lane, &first);
    for (int t0 = 0; t0 < tot; t0 += 32) {
      const int t = t0 + lane;
      const int own = segment_owner(first, t);
      const int seg = t - __shfl_sync(kFull, first, own);
      bool active = t < tot;
      float gp[3] = {0.f, 0.f, 0.f}, gg[3] = {0.f, 0.f, 0.f}, Wg = 0.0f;
      Dda dda;
      int dsel = 0, left = 0, dk = 0;
      int bcx = 0, bcy = 0, bcz = 0;
      uint32_t sb = kInvalid;
      uint32_t nx = kInvalid, ny = kInvalid, nz = kInvalid;  // scratch blocks behind the three exit faces
      if (active) {
        for (int a = 0; a < 3; ++a) {
          gp[a] = sh_pg[wid][own][a];
          gg[a] = sh_pg[wid][own][3 + a];
        }
        Wg = sh_pg[wid][own][6];
        DdaSeg sg;
        sg.init(&sh_se[wid][own][0], &sh_se[wid][own][3], 16);
        dsel = sg.d;
        dda = sg.seek(seg, K, &left);
        bcx = dda.cx >> blog;
        bcy = dda.cy >> blog;
        bcz = dda.cz >> blog;
        sb = scratch_of(m, block_lookup(m, bcx, bcy, bcz), ep);
        if (sb != kInvalid) {
          const uint32_t* row = &m.snbr[(size_t)sb * 27];
          nx = __ldcg(&row[(dda.sx + 1) * 9 + 4]);
          ny = __ldcg(&row[9 + (dda.sy + 1) * 3 + 1]);
          nz = __ldcg(&row[13 + dda.sz]);
        }
      }
      while (__any_sync(kFull, active)) {
        uint32_t vid = kInvalid;
        long long qv[4] = {0, 0, 0, 0};  // w hi, w*d hi, w lo, w*d lo
        if (active) {
          // Eq. (1) at the voxel centre, truncated to [-delta, delta]
          float dx[3];
          const int cc[3] = {dda.cx, dda.cy, dda.cz};
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const float xc = __fmul_rn(__fadd_rn((float)cc[a], 0.5f), m.v);
            dx[a] = __fsub_rn(gp[a], xc);
          }
          const float dist = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(dx[0], dx[0]), __fmul_rn(dx[1], dx[1])), __fmul_rn(dx[2], dx[2])));
          const float dot = __fadd_rn(__fadd_rn(__fmul_rn(dx[0], gg[0]), __fmul_rn(dx[1], gg[1])), __fmul_rn(dx[2], gg[2]));
          float d = dot >= 0.0f ? dist : -dist;
          if (d > m.delta) d = m.delta;
          if (d < -m.delta) d = -m.delta;
          // Eq. (2) / Eq. (4); the 1/z^2 factor is already in the group weight
          float w = Wg;
          if (m.weighting == 1) {
            if (d <= -m.delta)
              w = 0.0f;
            else if (d < -m.eps)
              w = __fmul_rn(Wg, __fdiv_rn(__fadd_rn(d, m.delta), __fsub_rn(m.delta, m.eps)));
          }
          if (w > 0.0f && sb != kInvalid) {
            const uint32_t l = (uint32_t)((((dda.cz & (B - 1)) << blog | (dda.cy & (B - 1))) << blog) | (dda.cx & (B - 1)));
            vid = (sb << m.b3log) | l;  // scratch voxel
            fx_split(w, &qv[0], &qv[2]);
            fx_split(__fmul_rn(w, d), &qv[1], &qv[3]);
            ++nrec;
          }
          if (left == 0) {
            active = false;
          } else {
            const int ax = dda.step();
            --left;
            if (ax == dsel && ++dk == K) {
              active = false;  // the next cell starts the ray's next segment
            } else {
              // block transition: a 6-connected step into the face neighbour, whose scratch
              // block this lane loaded when it entered the current block
              bool moved = false;
              if (ax == 0) {
                const int nb = dda.cx >> blog;
                if (nb != bcx) {
                  bcx = nb;
                  sb = nx;
                  moved = true;
                }
              } else if (ax == 1) {
                const int nb = dda.cy >> blog;
                if (nb != bcy) {
                  bcy = nb;
                  sb = ny;
                  moved = true;
                }
              } else {
                const int nb = dda.cz >> blog;
                if (nb != bcz) {
                  bcz = nb;
                  sb = nz;
                  moved = true;
                }
              }
              if (moved && sb != kInvalid) {
                const uint32_t* row = &m.snbr[(size_t)sb * 27];
                nx = __ldcg(&row[(dda.sx + 1) * 9 + 4]);
                ny = __ldcg(&row[9 + (dda.sy + 1) * 3 + 1]);
                nz = __ldcg(&row[13 + dda.sz]);
              }
            }
          }
        }
        const unsigned peers = __match_any_sync(kFull, vid);
        const bool alone = (peers == (1u << lane)) || vid == kInvalid;
        if (__all_sync(kFull, alone)) {
          if (vid != kInvalid) accumulate(m, vid, qv);
        } else {
          for (int j = 0; j < 4; ++j) sh_v[j][wid][lane] = qv[j];
          __syncwarp();
          if (vid != kInvalid && lane == __ffs(peers) - 1) {
            long long sum[4] = {0, 0, 0, 0};
            for (unsigned pm = peers; pm; pm &= pm - 1) {
              const int src = __ffs(pm) - 1;
              for (int j = 0; j < 4; ++j) sum[j] += sh_v[j][wid][src];
            }
            accumulate(m, vid, sum);
          }
          __syncwarp();
        }
      }
    }
    __syncwarp();
  }
  if (nrec) atomicAdd(&map_of(b, rec_map).ctr->nrecords, nrec);
}

// ------------------------------------------------------------------------------------ A5
// Appends vid to the scan's updated list and, if `queue`, to the ESDF dirty list: one leader
// per group of lanes of the same map issues both counter atomics back to back.
__device__ __forceinline__ void append_updated_dirty(const DevMap& m, uint32_t vid, bool queue) {
  const unsigned active = __activemask();
  const unsigned peers = __match_any_sync(active, (unsigned long long)(uintptr_t)m.ctr);
  const unsigned qpeers = peers & __ballot_sync(active, queue);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  const unsigned below = (1u << lane) - 1u;
  unsigned bu = 0, bd = 0;
  if (lane == leader) {
    bu = atomicAdd(&m.ctr->nupdated, (unsigned)__popc(peers));
    if (qpeers) bd = atomicAdd(&m.ctr->ndirty, (unsigned)__popc(qpeers));
  }
  bu = __shfl_sync(peers, bu, leader);
  bd = __shfl_sync(peers, bd, leader);
  m.updated[bu + __popc(peers & below)] = vid;
  if (queue) m.dirty[bd + __popc(qpeers & below)] = vid;
}

// Touch flags per lane in k_apply: 16 (one 16-byte load) where the scan's records are sparse
// in its scratch blocks (thin lines of voxels per block), 4 where they are dense.
__device__ __forceinline__ unsigned apply_flags_per_lane(const DevMap& m, bool wide) {
  const unsigned long long vox = (unsigned long long)scratch_blocks(m) << m.b3log;
  return wide && 2ull * __ldcg(&m.ctr->nrecords) < vox ? 16u : 4u;
}

// Every voxel that received records this scan gets the Eq. (3) merge, its sums and touch flag
// are cleared, and it joins the scan's updated list and (once) the queue of the next ESDF
// update. Each lane reads the touch flags of 4 or 16 consecutive scratch voxels; the warp
// compacts the touched ones (possibly of two maps) and gives each lane one at a time.
// One map per launch: the updated and queued voxels of a CTA are collected in shared memory and
// each list's space is reserved with one atomic per CTA flush, not one per warp round (the two
// counters of a map would otherwise take tens of thousands of serialised atomics per scan).
constexpr int kApplyBuf = 2048;

__global__ void __launch_bounds__(kThreads) k_apply(Batch b, unsigned warp_slots) {
  __shared__ unsigned pfx[kMaxBatch + 1];
  __shared__ uint32_t s_upd[kApplyBuf], s_dty[kApplyBuf];
  __shared__ unsigned s_cnt[2], s_base[2];
  const int lane = threadIdx.x & 31;
  const int nm = nmaps_of(b);
  // 16 flags per lane only when the launch has enough scratch voxels to keep every resident
  // warp busy several times over with them
  const unsigned vall = cta_prefix(pfx, b, [&](unsigned mi) { return scratch_blocks(map_of(b, mi)) << map_of(b, mi).b3log; });
  const bool wide = vall >= 16u * 32u * 4u * warp_slots;
  __syncthreads();
  const unsigned total = cta_prefix(pfx, b, [&](unsigned mi) {
    const DevMap& m = map_of(b, mi);
    return (scratch_blocks(m) << m.b3log) / apply_flags_per_lane(m, wide);  // B^3 >= 64
  });
  const unsigned stride = gridDim.x * blockDim.x;
  // 4 flags per lane at most: one CTA round appends at most kThreads * 4 voxels to each list
  const bool buffered = nm == 1 && !wide;
  static_assert(kApplyBuf >= 2 * kThreads * 4, "a CTA round fits the half-full buffer");
  if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0u;
  __syncthreads();
  auto flush = [&]() {  // all threads of the CTA
    __syncthreads();
    const DevMap& m = map_of(b, 0);
    if (threadIdx.x == 0) {
      s_base[0] = s_cnt[0] ? atomicAdd(&m.ctr->nupdated, s_cnt[0]) : 0u;
      s_base[1] = s_cnt[1] ? atomicAdd(&m.ctr->ndirty, s_cnt[1]) : 0u;
    }
    __syncthreads();
    for (unsigned j = threadIdx.x; j < s_cnt[0]; j += kThreads) m.updated[s_base[0] + j] = s_upd[j];
    for (unsigned j = threadIdx.x; j < s_cnt[1]; j += kThreads) m.dirty[s_base[1] + j] = s_dty[j];
    __syncthreads();
    if (threadIdx.x == 0) s_cnt[0] = s_cnt[1] = 0u;
    __syncthreads();
  };
  for (unsigned cbase = blockIdx.x * blockDim.x; cbase < total; cbase += stride) {
    const unsigned base = cbase + (threadIdx.x & ~31u);
    const unsigned i = base + lane;
    unsigned mi = 0, v0 = 0, bits = 0;
    uint32_t slot = 0;
    if (i < total) {
      mi = map_index(pfx, nm, i);
      const DevMap& m = map_of(b, mi);
      const unsigned V = apply_flags_per_lane(m, wide);
      v0 = (i - pfx[mi]) * V;  // first scratch voxel of this lane (V voxels of one scratch block)
      slot = m.slist[v0 >> m.b3log];  // loaded with the flags, not after them
      if (V == 16) {
        uint4* f = reinterpret_cast<uint4*>(m.stouch + v0);
        const uint4 w = *f;
        if (w.x | w.y | w.z | w.w) {
          *f = make_uint4(0u, 0u, 0u, 0u);
          const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
          for (int q = 0; q < 4; ++q)
            bits |= ((ws[q] & 1u) | ((ws[q] >> 7) & 2u) | ((ws[q] >> 14) & 4u) | ((ws[q] >> 21) & 8u)) << (4 * q);
        }
      } else {
        uint32_t* f = reinterpret_cast<uint32_t*>(m.stouch + v0);
        const uint32_t w = *f;
        if (w) {
          *f = 0u;
          bits = (w & 1u) | ((w >> 7) & 2u) | ((w >> 14) & 4u) | ((w >> 21) & 8u);
        }
      }
    }
    int first = 0;
    const int tot = warp_segments(__popc(bits), lane, &first);
    for (int t0 = 0; t0 < tot; t0 += 32) {
      const int t = t0 + lane;
      const int own = segment_owner(first, t);
      int n = t - __shfl_sync(kFull, first, own);
      const unsigned ob = __shfl_sync(kFull, bits, own);
      const unsigned omi = __shfl_sync(kFull, mi, own);
      const unsigned ov0 = __shfl_sync(kFull, v0, own);
      const uint32_t oslot = __shfl_sync(kFull, slot, own);
      if (t >= tot) continue;
      int j = 0;  // position of the (n+1)-th set bit of ob
      while (!(ob >> j & 1u) || n-- > 0) ++j;
      const DevMap& m = map_of(b, omi);
      const unsigned sv = ov0 + (unsigned)j;  // scratch voxel
      const uint32_t vid = (oslot << m.b3log) | (sv & ((1u << m.b3log) - 1u));
      // the sums, {D, W} and the queue flag are independent loads, issued together
      ulonglong2* a = reinterpret_cast<ulonglong2*>(&m.sacc[4 * (size_t)sv]);
      const ulonglong2 hi = a[0], lo = a[1];
      const float2 tv = m.tsdf[vid];
      const uint8_t vf = m.vflags[vid];
      a[0] = make_ulonglong2(0ull, 0ull);
      a[1] = make_ulonglong2(0ull, 0ull);
      const float Sw = __fadd_rn(__fmul_rn(__ll2float_rn((long long)hi.x), kAccInvScale),
                                 __fmul_rn(__ll2float_rn((long long)lo.x), kAccLoInvScale));
      const float Swd = __fadd_rn(__fmul_rn(__ll2float_rn((long long)hi.y), kAccInvScale),
                                  __fmul_rn(__ll2float_rn((long long)lo.y), kAccLoInvScale));
      // Eq. (3): D <- (W D + sum w d) / (W + sum w), W <- min(W + sum w, W_max)
      const float Wn = __fadd_rn(tv.y, Sw);
      const float D = __fdiv_rn(__fadd_rn(__fmul_rn(tv.y, tv.x), Swd), Wn);
      m.tsdf[vid] = make_float2(D, fminf(Wn, m.wmax));
      const bool queue = !(vf & kQueuedForEsdf);
      if (queue) m.vflags[vid] = (uint8_t)(vf | kQueuedForEsdf);
      if (buffered) {
        const unsigned act = __activemask();
        const unsigned qm = __ballot_sync(act, queue);
        const int leader = __ffs(act) - 1;
        const unsigned below = (1u << lane) - 1u;
        unsigned bu = 0, bd = 0;
        if (lane == leader) {
          bu = atomicAdd(&s_cnt[0], (unsigned)__popc(act));
          if (qm) bd = atomicAdd(&s_cnt[1], (unsigned)__popc(qm));
        }
        bu = __shfl_sync(act, bu, leader);
        bd = __shfl_sync(act, bd, leader);
        s_upd[bu + __popc(act & below)] = vid;
        if (queue) s_dty[bd + __popc(qm & below)] = vid;
      } else {
        append_updated_dirty(m, vid, queue);
      }
    }
    if (buffered) {
      __syncthreads();
      if (s_cnt[0] > (unsigned)(kApplyBuf - kThreads * 4)) flush();
    }
  }
  if (buffered) flush();
}

// ------------------------------------------------------------------------------ reset
// Empties a map for reuse without a host round trip: the used sizes (blocks, the last scan's
// scratch blocks) are read on the device; the counters are cleared after this kernel.
__global__ void __launch_bounds__(kThreads) k_reset_map(DevMap m) {
  const size_t nb = min(__ldcg(&m.ctr->blocks), m.cap_blocks);
  const size_t B3 = (size_t)1 << m.b3log;
  const size_t V = nb * B3;
  const size_t SV = (size_t)min(__ldcg(&m.ctr->ntouched), m.scr_cap) * B3;
  const size_t H = (size_t)m.hmask + 1;
  const size_t tiles = nb << m.tile_shift;
  const size_t i0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
  for (size_t i = i0; i < H; i += st) {
    m.hkeys[i] = kEmptyKey;
    m.hvals[i] = kInvalid;
    m.hclaim[i] = 0u;
  }
  for (size_t i = i0; i < nb; i += st) {
    m.bcoord[i] = make_int3(0, 0, 0);
    m.sinfo[i] = 0ull;
    m.mdirty[i] = 0u;
  }
  for (size_t i = i0; i < nb * 27; i += st) m.nbr[i] = kInvalid;
  for (size_t i = i0; i < tiles; i += st) {
    m.bstamp_r[i] = 0u;
    m.bstamp_l[i] = 0u;
  }
  for (size_t i = i0; i < V; i += st) {
    m.tsdf[i] = make_float2(0.0f, 0.0f);
    m.esdf[i] = 0ull;
    m.vflags[i] = 0u;
  }
  for (size_t i = i0; i < V / 32; i += st) {
    m.rbits0[i] = 0u;
    m.rbits1[i] = 0u;
    m.lbits0[i] = 0u;
    m.lbits1[i] = 0u;
    m.pbits[i] = 0u;
  }
  for (size_t i = i0; i < SV; i += st) {
    m.stouch[i] = 0u;
    reinterpret_cast<ulonglong2*>(m.sacc)[2 * i] = make_ulonglong2(0ull, 0ull);
    reinterpret_cast<ulonglong2*>(m.sacc)[2 * i + 1] = make_ulonglong2(0ull, 0ull);
  }
}

// ------------------------------------------------------------------------ import (restore)
__global__ void __launch_bounds__(kThreads) k_import_alloc(DevMap m, const int* __restrict__ vox, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    block_insert(m, vox[3 * i] >> m.blog, vox[3 * i + 1] >> m.blog, vox[3 * i + 2] >> m.blog);
}

__global__ void __launch_bounds__(kThreads) k_import_set(DevMap m, const int* __restrict__ vox, const float* __restrict__ D,
                                                        const float* __restrict__ W, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int x = vox[3 * i], y = vox[3 * i + 1], z = vox[3 * i + 2];
    const uint32_t slot = block_lookup(m, x >> m.blog, y >> m.blog, z >> m.blog);
    if (slot == kInvalid) continue;
    const int B = m.B;
    const uint32_t vid = (slot << m.b3log) | (uint32_t)((((z & (B - 1)) << m.blog | (y & (B - 1))) << m.blog) | (x & (B - 1)));
    m.tsdf[vid] = make_float2(D[i], W[i]);
    m.mdirty[slot] = 1u;
    const unsigned u = atomicAdd(&m.ctr->nupdated, 1u);
    m.updated[u] = vid;
    if (!(m.vflags[vid] & kQueuedForEsdf)) {
      m.vflags[vid] |= kQueuedForEsdf;
      const unsigned j = atomicAdd(&m.ctr->ndirty, 1u);
      m.dirty[j] = vid;
    }
  }
}

int grid_for(long long items, int num_sms, int per_sm) {
  long long g = (items + kThreads - 1) / kThreads;
  const long long cap = (long long)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

Batch single_batch(const DevMap& m, const float* pts, int n, const Pose& T, unsigned epoch) {
  Batch b;
  std::memset(&b, 0, sizeof(b));
  b.maps = nullptr;
  b.scans = nullptr;
  b.queries = nullptr;
  b.nmaps = 1;
  b.one = m;
  b.one_scan.pts = pts;
  b.one_scan.n = (unsigned)n;
  b.one_scan.epoch = epoch;
  std::memcpy(b.one_scan.T, T.T, sizeof(T.T));
  return b;
}

cudaError_t launch_init_groups(GroupEntry* tab, uint32_t entries, cudaStream_t s, LaunchHook* hook) {
  hook->begin(kKInitGroups, s);
  k_init_groups<<<(entries + kThreads - 1) / kThreads > 65535 ? 65535 : (entries + kThreads - 1) / kThreads, kThreads, 0, s>>>(tab, entries);
  hook->end(kKInitGroups, s);
  return cudaGetLastError();
}

cudaError_t launch_reset_counters(const Batch& b, const LaunchCfg& cfg, LaunchHook* hook) {
  hook->begin(kKReset, cfg.stream);
  k_reset_counters<<<1, kThreads, 0, cfg.stream>>>(b);
  hook->end(kKReset, cfg.stream);
  return cudaGetLastError();
}

cudaError_t launch_integrate(const Batch& b, const LaunchCfg& cfg, LaunchHook* hook) {
  const cudaStream_t s = cfg.stream;
  // single-map launches size the point grid by the scan; batched launches use the tuned grid
  // (all kernels stride over their device-side work counts)
  static int occ_bin = 0;
  if (!occ_bin) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_bin, k_bin_points, kThreads, 0);
    if (occ_bin < 1) occ_bin = 1;
  }
  // grids of at most the resident CTAs (every CTA first builds the per-map prefix)
  const int bin_per_sm = std::min(occ_bin, cfg.tune.bin_ctas_per_sm);
  const int gpts = b.maps ? cfg.num_sms * bin_per_sm : grid_for(b.one_scan.n, cfg.num_sms, bin_per_sm);
  // the ray kernels run a grid of at most their resident CTAs over all SMs and cut the rays
  // into warp tasks sized for that many warps
  static int occ_group = 0, occ_rays = 0, occ_rays_b = 0;
  if (!occ_group) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_group, k_group_rays, kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_rays, k_integrate_rays<VBX_RAYS_MIN_CTAS>, kThreads, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_rays_b, k_integrate_rays<VBX_RAYS_MIN_CTAS_BATCH>, kThreads, 0);
    if (occ_group < 1) occ_group = 1;
    if (occ_rays < 1) occ_rays = 1;
    if (occ_rays_b < 1) occ_rays_b = 1;
  }
  const bool batched = b.maps != nullptr;
  const int ggroup = cfg.num_sms * std::min(occ_group, cfg.tune.bin_ctas_per_sm);
  const int grays = cfg.num_sms * std::min(batched ? occ_rays_b : occ_rays, cfg.tune.rays_ctas_per_sm);
  hook->begin(kKBin, s);
  k_bin_points<<<gpts, kThreads, 0, s>>>(b);
  hook->end(kKBin, s);
  hook->begin(kKGroupRays, s);
  k_group_rays<<<ggroup, kThreads, 0, s>>>(b, (unsigned)(ggroup * kWarps));
  hook->end(kKGroupRays, s);
  hook->begin(kKLink, s);
  k_link_blocks<<<cfg.num_sms * 4, kThreads, 0, s>>>(b);
  hook->end(kKLink, s);
  hook->begin(kKScratchLinks, s);
  k_scratch_links<<<cfg.num_sms * 4, kThreads, 0, s>>>(b);
  hook->end(kKScratchLinks, s);
  hook->begin(kKIntegrateRays, s);
  if (batched)
    k_integrate_rays<VBX_RAYS_MIN_CTAS_BATCH><<<grays, kThreads, 0, s>>>(b, (unsigned)(grays * kWarps));
  else
    k_integrate_rays<VBX_RAYS_MIN_CTAS><<<grays, kThreads, 0, s>>>(b, (unsigned)(grays * kWarps));
  hook->end(kKIntegrateRays, s);
  hook->begin(kKApply, s);
  static int occ_apply = 0;
  if (!occ_apply) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_apply, k_apply, kThreads, 0);
    if (occ_apply < 1) occ_apply = 1;
  }
  const int gapply = cfg.num_sms * std::min(occ_apply, cfg.tune.apply_ctas_per_sm);
  k_apply<<<gapply, kThreads, 0, s>>>(b, (unsigned)(gapply * kWarps));
  hook->end(kKApply, s);
  return cudaGetLastError();
}

cudaError_t launch_reset_map(const DevMap& m, const LaunchCfg& cfg) {
  k_reset_map<<<cfg.num_sms * 8, kThreads, 0, cfg.stream>>>(m);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(m.ctr, 0, sizeof(Counters), cfg.stream);
}

cudaError_t launch_import(const DevMap& m, const int* vox, const float* D, const float* W, int n,
                          const LaunchCfg& cfg, LaunchHook* hook) {
  const cudaStream_t s = cfg.stream;
  const int g = grid_for(n, cfg.num_sms, 16);
  hook->begin(kKImportAlloc, s);
  k_import_alloc<<<g, kThreads, 0, s>>>(m, vox, n);
  hook->end(kKImportAlloc, s);
  hook->begin(kKLink, s);
  k_link_blocks<<<cfg.num_sms * 4, kThreads, 0, s>>>(single_batch(m, nullptr, 0, Pose{}));
  hook->end(kKLink, s);
  hook->begin(kKImportSet, s);
  k_import_set<<<g, kThreads, 0, s>>>(m, vox, D, W, n);
  hook->end(kKImportSet, s);
  return cudaGetLastError();
}


// -------------------------------------------------------------------------------------------
// Integration without device allocation.
//
// Callers that cannot allocate device memory while they run (a robot's real-time loop, where
// cudaMalloc/cudaFree synchronise the whole device and can stall for milliseconds past the
// control deadline; or a process that committed its whole device-memory budget at start-up)
// integrate scans through this path. vbx_integrate_scan keeps its per-scan scratch (point
// group table, group list, ray buffer) in map-owned buffers that it grows with cudaMalloc when
// a scan has more points than before; here the same scratch lives in one file-scope device
// array instead, sized for at most kNoAllocMaxPoints points, so no call allocates.
// Every GPU that loads the library holds this array (about 9.3 MiB) until the process exits.
// All calls share it and it keeps the previous call's contents: the group table is cleared at
// the start of every call, the other buffers are fully written before they are read. Two calls
// whose work overlaps on the GPU (different streams, or different maps used concurrently)
// race on the array; callers serialise them.

namespace {
constexpr uint32_t kNoAllocGroupEntries = 2u * (uint32_t)kNoAllocMaxPoints;
constexpr size_t kNoAllocGroupBytes = (size_t)kNoAllocGroupEntries * sizeof(GroupEntry);
constexpr size_t kNoAllocListBytes = (size_t)kNoAllocMaxPoints * sizeof(uint32_t);
constexpr size_t kNoAllocRayBytes = (size_t)kNoAllocMaxPoints * sizeof(float4);
constexpr size_t kNoAllocBytes = kNoAllocGroupBytes + kNoAllocListBytes + kNoAllocRayBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch, resolved once per device with that device current.
// In host code the symbol itself is only a host-side stand-in, never a device address.
constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;
}  // namespace

cudaError_t noalloc_scratch_setup(int device, void** ptr) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = p;
  }
  *ptr = g_noalloc_ptr[device];
  return cudaSuccess;
}

cudaError_t launch_integrate_noalloc(const DevMap& m, void* scratch, const float* pts, int n, const Pose& T,
                                     unsigned epoch, const LaunchCfg& cfg, LaunchHook* hook) {
  DevMap ms = m;
  unsigned char* base = static_cast<unsigned char*>(scratch);
  ms.gtab = reinterpret_cast<GroupEntry*>(base);
  ms.gmask = kNoAllocGroupEntries - 1;
  ms.glist = reinterpret_cast<uint32_t*>(base + kNoAllocGroupBytes);
  ms.rays = reinterpret_cast<float4*>(base + kNoAllocGroupBytes + kNoAllocListBytes);
  cudaError_t e = launch_init_groups(ms.gtab, kNoAllocGroupEntries, cfg.stream, hook);
  if (e != cudaSuccess) return e;
  return launch_integrate(single_batch(ms, pts, n, T, epoch), cfg, hook);
}

}  // namespace vbx
