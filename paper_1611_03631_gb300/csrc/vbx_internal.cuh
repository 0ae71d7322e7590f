// vbx_internal.cuh -- device-side layout and helpers of the GB300 map update.
//
// HBM layout of one map (all arrays indexed by pool slot or by voxel id):
//   block hash     : hkeys[H] u64 packed block key (EMPTY = ~0), hvals[H] u32 pool slot,
//                    hclaim[H] u32 scan epoch of the last scan whose rays entered the block
//   per block      : bcoord[slot] int3, nbr[slot*27 + k] u32 slot of the neighbour block in
//                    direction k = (dx+1)*9 + (dy+1)*3 + (dz+1) (k = 13 is the block itself),
//                    sinfo[slot] u64 {scan epoch << 32 | scratch block} of the block,
//                    mdirty[slot] u8 (TSDF changed since the last mesh extraction),
//                    mlist[i] u32 blocks listed by the current mesh extraction
//   per voxel      : voxel id vid = slot * B^3 + ((lz*B + ly)*B + lx)
//                    tsdf[vid]   float2 (D, W)                          8 B
//                    esdf[vid]   u64 packed {d f32 | flags u8 | parent u8} 8 B
//                    vflags[vid] u8 (bit0 queued for the ESDF)
//                    rbits/lbits[2][vid/32] u32 raise / lower frontier bitmasks (current, next)
//                    dirty list slot (u32)
//   per ESDF tile  : bstamp_r/bstamp_l[item] u32 epochs de-duplicating tile activations, item =
//                    slot << tile_shift | tile (a tile is the block, or an 8^3 octant of a 16^3 one)
//   per-scan sums  : scratch blocks, one per block the scan's rays enter (scr_cap of them):
//                    slist_h[i] / slist[i] u32 hash entry and pool slot of scratch block i,
//                    sacc[4*sv] i64 sums of w and w*d of scratch voxel sv = i * B^3 + local,
//                    each an exact two-part fixed point number (2^-28 part, 2^-60 part),
//                    stouch[sv] u8: the voxel received a record (all zero between scans)
//   lists          : updated (last scan), dirty (since last ESDF); the ESDF's active
//                    (map, block) lists live in the launch group's EsdfCtl
//   per-scan points: group hash table (64 B entries), group list, rays (float4)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vbx {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr uint32_t kInvalid = 0xffffffffu;
constexpr int kSub = 65536;  // fixed-point units per voxel for ray endpoints and offsets
// Per-voxel sums are exact: a float32 record x is split into hi = trunc(x * 2^28) and
// lo = rint(frac(x * 2^28) * 2^32), i.e. units of 2^-28 and 2^-60; both are summed with 64-bit
// integer atomics, so the sums do not depend on the order of the records.
constexpr float kAccScale = 268435456.0f;  // 2^28
constexpr float kAccInvScale = 1.0f / 268435456.0f;
constexpr float kAccLoScale = 4294967296.0f;  // 2^32
constexpr float kAccLoInvScale = 1.0f / 1152921504606846976.0f;  // 2^-60

// sticky device error bits
constexpr unsigned kErrPoolFull = 1u;
constexpr unsigned kErrHashFull = 2u;
constexpr unsigned kErrTimeout = 4u;
constexpr unsigned kErrGroupTable = 8u;
constexpr unsigned kErrScratchFull = 16u;

// ESDF voxel word: bits 63..32 float d, bits 15..8 flags, bits 7..0 parent direction
constexpr unsigned kObserved = 1u;
constexpr unsigned kFixed = 2u;
constexpr unsigned kHasSite = 4u;  // Euclidean variant: the word holds the offset to its site
constexpr unsigned kNoParent = 255u;
constexpr uint8_t kQueuedForEsdf = 1u;
constexpr uint8_t kSiteRaised = 2u;  // Euclidean variant: a site raised by this ESDF update

struct __align__(16) GroupEntry {
  unsigned long long key;       // packed voxel key, kEmptyKey when free
  unsigned long long sw;        // sum of integer point weights
  unsigned long long swo_lo[3]; // sum of weight * sub-voxel offset, low 64 bits per axis
  unsigned int swo_hi[3];       // carries into bit 64 and up
  unsigned int n;               // number of points
};
static_assert(sizeof(GroupEntry) == 64, "group entry is one 64-byte sector pair");

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

// Per-scan counters are contiguous so that one memset clears them.
struct Counters {
  // ---- per scan (cleared by vbx_integrate_scan)
  unsigned int ngroups;
  unsigned int nnew;
  unsigned int nupdated;
  unsigned int npoints_valid;
  unsigned int ntouched;  // blocks entered by the scan's rays (scratch blocks claimed)
  unsigned int nvseg;     // voxel-traversal segments of the scan's rays
  unsigned long long nrecords;
  // ---- persistent
  unsigned int blocks;
  unsigned int error;
  unsigned int ndirty;
  unsigned int epoch;
  // ---- per ESDF update (cleared by vbx_update_esdf)
  unsigned int raise_rounds;
  unsigned int lower_rounds;
  unsigned long long raise_pops;
  unsigned long long lower_pops;
  unsigned int seeds;
  unsigned int esdf_in;
  unsigned int esdf_block_visits;  // staged tile-rounds
  unsigned int esdf_local_iters;   // local relaxation iterations summed over tile-rounds
  unsigned int esdf_phase_ns[3];   // device time of classification, raise and lower phases
  // ---- per mesh extraction (cleared by vbx_extract_mesh)
  unsigned long long mesh_tris;    // triangles of the listed blocks
  unsigned int mesh_blocks;        // blocks listed for meshing
  unsigned int mesh_pad;
};

// Control block of one ESDF launch: one map, or a batch of maps updated by the same
// cooperative kernel. Active lists hold (map index, block slot) pairs; counts rotate over
// three slots so that the count of the next round can be cleared while the current one is
// read.
struct EsdfCtl {
  GridBarrier bar;
  unsigned int rcnt[3];
  unsigned int lcnt[3];
  unsigned int rnext[3];  // next unclaimed entry of the round's raise / lower list (CTAs claim
  unsigned int lnext[3];  // tiles one at a time, so a round is not paced by a static split)
  // lower wave as one asynchronous work queue (no rounds): consumer tickets, tickets produced
  // beyond the initial list, and items finished
  unsigned int qhead;
  unsigned int qtail;
  unsigned int qdone;
  unsigned int error;
  unsigned int cap;  // capacity of each active list
  uint2* ract0;
  uint2* ract1;
  uint2* lact0;
  uint2* lact1;
  // lower-wave queue ring (entries past the initial list) and its per-slot publish / read tags;
  // rcap >= cap + 27 x (largest grid), so a producer never waits on a slot no CTA will read
  unsigned int rcap;
  unsigned int calls;  // launches so far (tags carry it, so stale tags never match)
  uint2* lring;
  unsigned long long* ltag;
};

struct DevMap {
  // parameters (float32, as the map holds them)
  float v, delta, eps, gamma, wmax, dmax;
  float max_range2;  // <= 0: no range limit
  float range_lim2;  // (16384 v)^2: points farther than 2^14 voxels are dropped
  float L1, L2, L3;  // quasi-Euclidean step lengths v, v*sqrt(2), v*sqrt(3)
  int euclid;        // 1: full Euclidean ESDF (the word holds the offset to the site)
  int B, blog, b3log;
  int tile_shift;  // log2 of the ESDF tiles per block: 3 for B = 16 (8^3 octants), else 0
  int weighting, grouped;
  int esdf_mode;  // 0: fixed band |D| < gamma; 1: occupancy (D < 0 occupied at distance 0)
  // block hash
  unsigned long long* hkeys;
  uint32_t* hvals;
  uint32_t* hclaim;
  uint32_t hmask;
  // pool
  uint32_t cap_blocks;
  int3* bcoord;
  uint32_t* nbr;
  unsigned long long* sinfo;
  float2* tsdf;
  // per-scan sums (scratch blocks)
  uint32_t scr_cap;
  uint32_t* slist_h;
  uint32_t* slist;
  uint32_t* snbr;  // per scratch block of the current scan: the scratch block of each of its 27
                   // neighbours (kInvalid if that block has none this scan)
  unsigned long long* sacc;
  uint8_t* stouch;
  unsigned long long* esdf;
  uint8_t* vflags;
  uint32_t* rbits0;
  uint32_t* rbits1;
  uint32_t* lbits0;
  uint32_t* lbits1;
  // quasi-Euclidean ESDF update: voxels (raised, or newly observed) that take their value from
  // their neighbours when the lower wave first stages their tile; each bit is set together with
  // the voxel's lower-frontier bit and taken by that staging
  uint32_t* pbits;
  uint32_t* bstamp_r;
  uint32_t* bstamp_l;
  // mesh: per block, whether its TSDF may have changed since the last extraction; the blocks
  // listed by the current extraction
  uint8_t* mdirty;
  uint32_t* mlist;
  // lists
  uint32_t* updated;
  uint32_t* dirty;
  uint32_t* newblk;
  // per-scan scratch
  GroupEntry* gtab;
  uint32_t gmask;
  uint32_t* glist;
  float4* rays;
  Counters* ctr;
};

// ---------------------------------------------------------------------------------------
// keys and hashing

__device__ __forceinline__ unsigned long long pack_key(int x, int y, int z) {
  return ((unsigned long long)(uint32_t)(x + (1 << 20)) << 42) | ((unsigned long long)(uint32_t)(y + (1 << 20)) << 21) |
         (unsigned long long)(uint32_t)(z + (1 << 20));
}

__device__ __forceinline__ int3 unpack_key(unsigned long long k) {
  return make_int3((int)((k >> 42) & 0x1fffff) - (1 << 20), (int)((k >> 21) & 0x1fffff) - (1 << 20),
                   (int)(k & 0x1fffff) - (1 << 20));
}

__device__ __forceinline__ uint32_t hash64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return (uint32_t)k;
}

__device__ __forceinline__ int floor_div_pow2(int a, int log2b) { return a >> log2b; }  // arithmetic shift = floor

// Block hash lookup (no insertion); kInvalid when absent or not allocated.
__device__ __forceinline__ uint32_t block_lookup(const DevMap& m, int bx, int by, int bz) {
  const unsigned long long key = pack_key(bx, by, bz);
  uint32_t h = hash64(key) & m.hmask;
  for (uint32_t probe = 0; probe <= m.hmask; ++probe) {
    const unsigned long long k = __ldcg(&m.hkeys[h]);
    if (k == key) return __ldcg(&m.hvals[h]);
    if (k == kEmptyKey) return kInvalid;
    h = (h + 1) & m.hmask;
  }
  return kInvalid;
}

// Lock-free find-or-insert (Sec. III: O(1) hashed block insertion). The thread that claims an
// empty slot with atomicCAS takes a pool slot and publishes it; others see the key and move on.
// Slots are read only by later kernels, so nobody waits here. Returns the hash entry of the
// block (its pool slot may not be published yet), or kInvalid if the table is full.
__device__ __forceinline__ uint32_t block_insert(const DevMap& m, int bx, int by, int bz) {
  const unsigned long long key = pack_key(bx, by, bz);
  uint32_t h = hash64(key) & m.hmask;
  for (uint32_t probe = 0; probe <= m.hmask; ++probe) {
    unsigned long long k = __ldcg(&m.hkeys[h]);
    if (k == key) return h;
    if (k == kEmptyKey) {
      k = atomicCAS(&m.hkeys[h], kEmptyKey, key);
      if (k == kEmptyKey) {
        const uint32_t slot = atomicAdd(&m.ctr->blocks, 1u);
        if (slot >= m.cap_blocks) {
          m.hvals[h] = kInvalid;
          atomicOr(&m.ctr->error, kErrPoolFull);
          return h;
        }
        m.hvals[h] = slot;
        m.bcoord[slot] = make_int3(bx, by, bz);
        const uint32_t i = atomicAdd(&m.ctr->nnew, 1u);
        m.newblk[i] = slot;
        return h;
      }
      if (k == key) return h;
    }
    h = (h + 1) & m.hmask;
  }
  atomicOr(&m.ctr->error, kErrHashFull);
  return kInvalid;
}

// ---------------------------------------------------------------------------------------
// ESDF voxel word

__device__ __forceinline__ unsigned long long ew_pack(float d, unsigned flags, unsigned parent) {
  return ((unsigned long long)__float_as_uint(d) << 32) | ((unsigned long long)(flags & 0xffu) << 8) |
         (unsigned long long)(parent & 0xffu);
}
__device__ __forceinline__ float ew_d(unsigned long long w) { return __uint_as_float((uint32_t)(w >> 32)); }
__device__ __forceinline__ unsigned ew_flags(unsigned long long w) { return (unsigned)(w >> 8) & 0xffu; }
__device__ __forceinline__ unsigned ew_parent(unsigned long long w) { return (unsigned)w & 0xffu; }
// Euclidean variant: {d | oz (i8) | oy (i8) | flags | ox (i8)}, the offset from the voxel to its
// site in voxels (|offset| <= d_max / v < 127)
__device__ __forceinline__ unsigned long long ew_pack_site(float d, unsigned flags, int ox, int oy, int oz) {
  return ((unsigned long long)__float_as_uint(d) << 32) | ((unsigned long long)((unsigned)oz & 0xffu) << 24) |
         ((unsigned long long)((unsigned)oy & 0xffu) << 16) | ((unsigned long long)(flags & 0xffu) << 8) |
         (unsigned long long)((unsigned)ox & 0xffu);
}
__device__ __forceinline__ int3 ew_site(unsigned long long w) {
  return make_int3((int)(signed char)(w & 0xffu), (int)(signed char)((w >> 16) & 0xffu), (int)(signed char)((w >> 24) & 0xffu));
}

// Voxel id of the 26-neighbour in direction k (kInvalid if its block does not exist).
__device__ __forceinline__ uint32_t neighbor_vid(const DevMap& m, uint32_t vid, int k) {
  const int B = m.B, blog = m.blog;
  uint32_t slot = vid >> m.b3log;
  const uint32_t l = vid & ((1u << m.b3log) - 1u);
  int x = (int)(l & (B - 1)) + (k / 9 - 1);
  int y = (int)((l >> blog) & (B - 1)) + ((k / 3) % 3 - 1);
  int z = (int)(l >> (2 * blog)) + (k % 3 - 1);
  const int bx = x < 0 ? -1 : (x >= B ? 1 : 0);
  const int by = y < 0 ? -1 : (y >= B ? 1 : 0);
  const int bz = z < 0 ? -1 : (z >= B ? 1 : 0);
  if (bx | by | bz) {
    slot = __ldg(&m.nbr[(size_t)slot * 27 + (bx + 1) * 9 + (by + 1) * 3 + (bz + 1)]);
    if (slot == kInvalid) return kInvalid;
    x -= bx * B;
    y -= by * B;
    z -= bz * B;
  }
  return (slot << m.b3log) | (uint32_t)((((z << blog) | y) << blog) | x);
}

// ---------------------------------------------------------------------------------------
// Ray setup shared by the block and voxel traversals (identical float32 operations in both
// kernels, no contraction): s -> e = pbar + delta * (pbar - s)/|pbar - s|, both quantised to
// 1/65536 voxel.
struct RayGeom {
  float p[3];   // pbar
  float g[3];   // pbar - s
  long long S[3];
  long long E[3];
};

__device__ __forceinline__ bool ray_setup(const float pbar[3], const float s[3], float v, float delta, RayGeom* r) {
  for (int a = 0; a < 3; ++a) {
    r->p[a] = pbar[a];
    r->g[a] = __fsub_rn(pbar[a], s[a]);
  }
  const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(r->g[0], r->g[0]), __fmul_rn(r->g[1], r->g[1])), __fmul_rn(r->g[2], r->g[2]));
  const float len = __fsqrt_rn(n2);
  if (!(len > 0.0f)) return false;
  for (int a = 0; a < 3; ++a) {
    const float u = __fdiv_rn(r->g[a], len);
    const float e = __fadd_rn(pbar[a], __fmul_rn(delta, u));
    r->S[a] = __float2ll_rn(__fmul_rn(__fdiv_rn(s[a], v), 65536.0f));
    r->E[a] = __float2ll_rn(__fmul_rn(__fdiv_rn(e, v), 65536.0f));
  }
  return true;
}

// Incremental integer 3-D DDA over cells of size F fixed-point units (F = 65536 for voxels,
// 65536*B for blocks). The next face crossing of axis a is at t_a = num_a / den_a; instead of
// comparing the ratios at every step, the three pairwise cross differences
// C_ab = num_a*den_b - num_b*den_a are kept and updated by additions when an axis steps.
// Ties go to x, then y, then z. With ray ends at most 2^14 voxels apart (points farther away
// are dropped) every numerator, denominator and product stays below 2^62.
struct Dda {
  int cx, cy, cz;     // current cell
  int sx, sy, sz;     // step direction per axis (+1 / -1)
  int rx, ry, rz;     // remaining steps per axis
  long long ix, iy, iz;  // F * den per axis
  long long cxy, cxz, cyz;

  __host__ __device__ __forceinline__ void init(const long long S[3], const long long E[3], int log2F) {
    long long num[3], den[3];
    init(S, E, log2F, num, den);
  }
  // Also returns the first-crossing numerators and the denominators (for seeking).
  __host__ __device__ __forceinline__ void init(const long long S[3], const long long E[3], int log2F, long long num[3],
                                                long long den[3]) {
    int c[3], st[3], rem[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      c[a] = (int)(S[a] >> log2F);
      const int ce = (int)(E[a] >> log2F);
      st[a] = E[a] >= S[a] ? 1 : -1;
      den[a] = E[a] >= S[a] ? E[a] - S[a] : S[a] - E[a];
      rem[a] = ce >= c[a] ? ce - c[a] : c[a] - ce;
      num[a] = st[a] > 0 ? (((long long)c[a] + 1) << log2F) - S[a] : S[a] - ((long long)c[a] << log2F);
    }
    cx = c[0], cy = c[1], cz = c[2];
    sx = st[0], sy = st[1], sz = st[2];
    rx = rem[0], ry = rem[1], rz = rem[2];
    ix = den[0] << log2F, iy = den[1] << log2F, iz = den[2] << log2F;
    cxy = num[0] * den[1] - num[1] * den[0];
    cxz = num[0] * den[2] - num[2] * den[0];
    cyz = num[1] * den[2] - num[2] * den[1];
  }
  __host__ __device__ __forceinline__ int steps() const { return rx + ry + rz; }
  // Advances one cell; returns the axis stepped (0, 1, 2).
  __host__ __device__ __forceinline__ int step() {
    const bool vx = rx > 0, vy = ry > 0, vz = rz > 0;
    if (vx && (!vy || cxy <= 0) && (!vz || cxz <= 0)) {
      cxy += iy;
      cxz += iz;
      cx += sx;
      rx -= 1;
      return 0;
    }
    if (vy && (!vz || cyz <= 0)) {
      cxy -= ix;
      cyz += iz;
      cy += sy;
      ry -= 1;
      return 1;
    }
    cxz -= ix;
    cyz -= iy;
    cz += sz;
    rz -= 1;
    return 2;
  }
};

// Work splitting of long rays: the traversal of a ray is cut at every K-th crossing of its
// dominant axis d (the axis with the most steps, ties to the lower axis); segment s starts in
// the cell entered by the (s*K)-th crossing of d and ends before the ((s+1)*K)-th. The state at
// a cut has a closed form: after n_a crossings per axis, cell_a = c_a + s_a n_a,
// rem_a -= n_a and C_ab += n_a F den_b - n_b F den_a, and n_b for b != d counts the crossings
// of b that the DDA orders before the cut (earlier, or at the same parameter on a lower axis).
struct DdaSeg {
  Dda q0;  // state at the start of the ray
  long long num0[3], den[3];
  int log2F;
  int d;  // dominant axis

  __host__ __device__ __forceinline__ void init(const long long S[3], const long long E[3], int lf) {
    log2F = lf;
    q0.init(S, E, lf, num0, den);
    d = 0;
    if (q0.ry > q0.rx) d = 1;
    if (q0.rz > (d == 0 ? q0.rx : q0.ry)) d = 2;
  }
  __host__ __device__ __forceinline__ int rem(int a) const { return a == 0 ? q0.rx : (a == 1 ? q0.ry : q0.rz); }
  __host__ __device__ __forceinline__ int segments(int K) const { return rem(d) / K + 1; }
  // DDA state at the start of segment s (0 <= s < segments(K)); *left = steps after it.
  __host__ __device__ __forceinline__ Dda seek(int s, int K, int* left) const {
    Dda q = q0;
    if (s == 0) {
      *left = q0.steps();
      return q;
    }
    const long long F = 1ll << log2F;
    // (selected without indexing by d, so that the arrays stay in registers)
    const long long num_d = d == 0 ? num0[0] : (d == 1 ? num0[1] : num0[2]);
    const long long den_d = d == 0 ? den[0] : (d == 1 ? den[1] : den[2]);
    const long long j = (long long)s * K;     // crossings of d up to and including the cut
    const long long tn = num_d + (j - 1) * F;  // the cut is at t = tn / den_d
    const long long fd = den_d << log2F;
    long long n[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      if (b == d) {
        n[b] = j;
        continue;
      }
      const int rb = rem(b);
      long long cnt = 0;
      if (rb > 0) {
        // crossing i of b precedes the cut iff (num0_b + i F) den_d < tn den_b
        // (or equal, for b before d in the tie order)
        const long long r = tn * den[b] - num0[b] * den_d;
        if (b < d)
          cnt = r < 0 ? 0 : r / fd + 1;
        else
          cnt = r <= 0 ? 0 : (r - 1) / fd + 1;
        if (cnt > rb) cnt = rb;
      }
      n[b] = cnt;
    }
    q.cx += q.sx * (int)n[0];
    q.cy += q.sy * (int)n[1];
    q.cz += q.sz * (int)n[2];
    q.rx -= (int)n[0];
    q.ry -= (int)n[1];
    q.rz -= (int)n[2];
    q.cxy += n[0] * q.iy - n[1] * q.ix;
    q.cxz += n[0] * q.iz - n[2] * q.ix;
    q.cyz += n[1] * q.iz - n[2] * q.iy;
    *left = q.steps();
    return q;
  }
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t) : : "memory");
  return t;
}

// ---------------------------------------------------------------------------------------
// grid-wide barrier for cooperative launches, with a bounded wait

__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned int nblocks, unsigned* err) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* genp = &bar->gen;
    const unsigned int g = *genp;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      while (*genp == g) {
        if (++spins > (1ll << 25)) {
          atomicOr(err, kErrTimeout);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

}  // namespace vbx
