// esdf.cu -- incremental ESDF update from the updated TSDF voxels (Sec. V-A, Algorithm 1 of
// Oleynikova et al. 2017), as one cooperative persistent kernel:
//   A6 classify : every TSDF voxel updated since the last call takes one branch of the first
//                 loop of Algorithm 1 (fixed band |D| < gamma, leaving the band, new voxel,
//                 sign flip) and seeds the raise and lower frontiers
//   A7 raise    : synchronous rounds (one warp per popped voxel, one lane per direction);
//                 a popped non-fixed voxel is reset to +-d_max, its
//                 children (neighbours whose parent direction points back at it) form the
//                 next raise frontier and all other observed neighbours join the lower frontier
//   A8 lower    : synchronous rounds; each popped voxel (one warp, one lane per direction)
//                 relaxes its observed, non-fixed,
//                 same-sign 26-neighbours with quasi-Euclidean steps; the neighbour's
//                 {distance, parent} word is lowered with a 64-bit atomicMin whose high half
//                 is the float's bit pattern (monotone in |d| for a fixed sign)
// The paper processes the open set with a priority queue or a FIFO; synchronous frontier
// rounds reach the same fixpoint (the lower wave computes the greatest fixpoint below the
// post-raise values of a monotone relaxation, which does not depend on the processing
// order). Frontier pushes are de-duplicated per round with monotone epoch stamps and
// appended with one atomic per coalesced warp group.
#include <cooperative_groups.h>
#include <cstdlib>
#include <cuda_runtime.h>

#include "launch.h"
#include "vbx_internal.cuh"

namespace cg = cooperative_groups;

namespace vbx {

namespace {

constexpr int kThreads = 256;
constexpr unsigned kMaxRounds = 1u << 16;

// Appends vid to a frontier unless it is already in the frontier of this epoch.
__device__ __forceinline__ void push(uint32_t* buf, unsigned* count, uint32_t* stamps, uint32_t vid, unsigned epoch) {
  if (atomicMax(&stamps[vid], epoch) >= epoch) return;
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(count, g.size());
  base = g.shfl(base, 0);
  buf[base + g.thread_rank()] = vid;
}

__device__ __forceinline__ float step_len(const DevMap& m, int k) {
  const int n1 = (k / 9 != 1) + ((k / 3) % 3 != 1) + (k % 3 != 1);
  return n1 == 1 ? m.L1 : (n1 == 2 ? m.L2 : m.L3);
}

__global__ void __launch_bounds__(kThreads) k_esdf(DevMap m) {
  Counters* c = m.ctr;
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nthreads = gridDim.x * blockDim.x;
  const unsigned lane = threadIdx.x & 31u;
  const unsigned gwarp = tid >> 5, nwarps = nthreads >> 5;
  const int kdir = lane < 13 ? (int)lane : (int)lane + 1;  // lanes 0..25 -> the 26 directions
  const float klen = lane < 26 ? step_len(m, kdir) : 0.0f;
  const unsigned base = __ldcg(&c->epoch);
  const unsigned e0 = base + 1;  // epoch of the frontiers seeded by classification
  const float dmax = m.dmax;

  // ---------------------------------------------------------------- A6: classification
  const unsigned nd = __ldcg(&c->ndirty);
  unsigned seeds = 0;
  for (unsigned i = tid; i < nd; i += nthreads) {
    const uint32_t vid = m.dirty[i];
    m.vflags[vid] = (uint8_t)(m.vflags[vid] & ~kQueuedForEsdf);
    const float2 t = m.tsdf[vid];
    if (!(t.y > 0.0f)) continue;
    const float Df = t.x == 0.0f ? 0.0f : t.x;  // sign(0) = +1
    const bool neg = Df < 0.0f;
    const float sdmax = neg ? -dmax : dmax;
    const unsigned long long w = __ldcg(&m.esdf[vid]);
    const unsigned fl = ew_flags(w);
    const bool obs = (fl & kObserved) != 0;
    const float de = ew_d(w);
    if (fabsf(Df) < m.gamma) {  // isFixed, evaluated on the TSDF voxel
      ++seeds;
      const bool lower_only = !obs || (((de < 0.0f) == neg) && fabsf(Df) <= fabsf(de));
      m.esdf[vid] = ew_pack(Df, kObserved | kFixed, kNoParent);
      if (!lower_only) push(m.rfront0, &c->rc[0], m.stamp_r, vid, e0);
      push(m.lfront0, &c->lc[0], m.stamp_l, vid, e0);
    } else if (fl & kFixed) {  // leaves the fixed band
      m.esdf[vid] = ew_pack(sdmax, kObserved, kNoParent);
      push(m.rfront0, &c->rc[0], m.stamp_r, vid, e0);
    } else if (!obs) {  // newly observed: its observed neighbours will lower it
      m.esdf[vid] = ew_pack(sdmax, kObserved, kNoParent);
      for (int k = 0; k < 27; ++k) {
        if (k == 13) continue;
        const uint32_t n = neighbor_vid(m, vid, k);
        if (n == kInvalid) continue;
        if (ew_flags(__ldcg(&m.esdf[n])) & kObserved) push(m.lfront0, &c->lc[0], m.stamp_l, n, e0);
      }
    } else if ((de < 0.0f) != neg) {  // sign flip of a propagated voxel
      m.esdf[vid] = ew_pack(sdmax, kObserved, kNoParent);
      push(m.rfront0, &c->rc[0], m.stamp_r, vid, e0);
    }
  }
  if (seeds) atomicAdd(&c->seeds, seeds);
  if (!grid_barrier(&c->bar, gridDim.x, &c->error)) return;

  // ------------------------------------------------------------------------ A7: raise
  unsigned long long pops = 0;
  unsigned r = 0;
  for (;; ++r) {
    const unsigned cnt = __ldcg(&c->rc[r % 3]);
    if (cnt == 0 || (__ldcg(&c->error) & kErrTimeout)) break;
    if (r >= kMaxRounds) {
      if (tid == 0) atomicOr(&c->error, kErrTimeout);
      break;
    }
    if (tid == 0) c->rc[(r + 2) % 3] = 0;
    const uint32_t* cur = (r & 1) ? m.rfront1 : m.rfront0;
    uint32_t* nxt = (r & 1) ? m.rfront0 : m.rfront1;
    unsigned* ncnt = &c->rc[(r + 1) % 3];
    const unsigned ep = base + 2 + r;
    for (unsigned i = gwarp; i < cnt; i += nwarps) {  // one warp per voxel, one lane per direction
      const uint32_t vid = cur[i];
      const unsigned long long w = __ldcg(&m.esdf[vid]);
      const unsigned fl = ew_flags(w);
      if (lane == 0) {
        ++pops;
        if (!(fl & kFixed)) m.esdf[vid] = ew_pack(ew_d(w) < 0.0f ? -dmax : dmax, fl, kNoParent);
      }
      if (lane < 26) {
        const uint32_t n = neighbor_vid(m, vid, kdir);
        if (n != kInvalid) {
          const unsigned long long nw = __ldcg(&m.esdf[n]);
          const unsigned nfl = ew_flags(nw);
          if (nfl & kObserved) {
            if (!(nfl & kFixed) && ew_parent(nw) == (unsigned)(26 - kdir))
              push(nxt, ncnt, m.stamp_r, n, ep);
            else
              push(m.lfront0, &c->lc[0], m.stamp_l, n, e0);
          }
        }
      }
    }
    if (!grid_barrier(&c->bar, gridDim.x, &c->error)) return;
  }
  const unsigned raise_rounds = r;
  if (pops) atomicAdd(&c->raise_pops, pops);

  // ------------------------------------------------------------------------ A8: lower
  pops = 0;
  unsigned l = 0;
  for (;; ++l) {
    const unsigned cnt = __ldcg(&c->lc[l % 3]);
    if (cnt == 0 || (__ldcg(&c->error) & kErrTimeout)) break;
    if (l >= kMaxRounds) {
      if (tid == 0) atomicOr(&c->error, kErrTimeout);
      break;
    }
    if (tid == 0) c->lc[(l + 2) % 3] = 0;
    const uint32_t* cur = (l & 1) ? m.lfront1 : m.lfront0;
    uint32_t* nxt = (l & 1) ? m.lfront0 : m.lfront1;
    unsigned* ncnt = &c->lc[(l + 1) % 3];
    const unsigned ep = base + 2 + l;
    for (unsigned i = gwarp; i < cnt; i += nwarps) {  // one warp per voxel, one lane per direction
      const uint32_t vid = cur[i];
      const unsigned long long w = __ldcg(&m.esdf[vid]);
      if (!(ew_flags(w) & kObserved)) continue;
      if (lane == 0) ++pops;
      if (lane >= 26) continue;
      const float dv = ew_d(w);
      const bool neg = dv < 0.0f;
      const uint32_t n = neighbor_vid(m, vid, kdir);
      if (n == kInvalid) continue;
      const unsigned long long nw = __ldcg(&m.esdf[n]);
      const unsigned nfl = ew_flags(nw);
      if ((nfl & (kObserved | kFixed)) != kObserved) continue;
      const float dn = ew_d(nw);
      if ((dn < 0.0f) != neg) continue;
      const float cand = __fadd_rn(fabsf(dv), klen);
      if (cand < fabsf(dn)) {
        const unsigned long long old = atomicMin(&m.esdf[n], ew_pack(neg ? -cand : cand, nfl, (unsigned)(26 - kdir)));
        if (fabsf(ew_d(old)) > cand) push(nxt, ncnt, m.stamp_l, n, ep);
      }
    }
    if (!grid_barrier(&c->bar, gridDim.x, &c->error)) return;
  }
  if (pops) atomicAdd(&c->lower_pops, pops);
  if (tid == 0) {
    c->esdf_in = nd;
    c->raise_rounds = raise_rounds;
    c->lower_rounds = l;
    c->epoch = base + 3 + (raise_rounds > l ? raise_rounds : l);
    c->ndirty = 0;
  }
}

}  // namespace

int esdf_max_blocks_per_sm() {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_esdf, kThreads, 0) != cudaSuccess) return 0;
  return nb;
}

cudaError_t launch_esdf(const DevMap& m, const LaunchCfg& cfg, LaunchHook* hook) {
  static int per_sm = -1;
  if (per_sm < 0) {
    per_sm = esdf_max_blocks_per_sm();
    // resident CTAs per SM of the cooperative grid: 2 by default (fastest of 1, 2, 4 on the
    // room workload), VBX_ESDF_CTAS_PER_SM to tune
    int want = 2;
    if (const char* e = getenv("VBX_ESDF_CTAS_PER_SM")) want = atoi(e) > 0 ? atoi(e) : want;
    if (per_sm > want) per_sm = want;
  }
  if (per_sm <= 0) return cudaErrorCooperativeLaunchTooLarge;
  dim3 grid(cfg.num_sms * per_sm), block(kThreads);
  DevMap arg = m;
  void* args[] = {&arg};
  hook->begin(kKEsdf, cfg.stream);
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_esdf, grid, block, args, 0, cfg.stream);
  hook->end(kKEsdf, cfg.stream);
  return e;
}

}  // namespace vbx
