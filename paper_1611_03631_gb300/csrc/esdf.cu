// esdf.cu -- incremental ESDF update from the updated TSDF voxels (Sec. V-A, Algorithm 1 of
// Oleynikova et al. 2017), as one cooperative persistent kernel over a group of maps:
//   A6 classify : every TSDF voxel updated since the last call takes one branch of the first
//                 loop of Algorithm 1 (fixed band |D| < gamma, leaving the band, new voxel,
//                 sign flip) and seeds the raise and lower frontiers
//   A7 raise    : active tiles (a block, or an 8^3 octant of a 16^3 block), in global rounds
//                 or from a work queue; a CTA stages one tile and its one-voxel halo in shared
//                 memory and raises within the tile until no child is left there: a raised
//                 non-fixed voxel is reset to +-d_max, neighbours whose parent direction points
//                 back at it are raised next, and the raised voxel itself joins the lower
//                 frontier marked to pull; children in the halo go to their own tile
//   A8 lower    : active tiles, likewise; a voxel marked to pull (raised, or newly observed)
//                 first takes the best offer of its neighbours (what their pushes would give
//                 it), then the CTA relaxes the staged tile to local convergence (observed,
//                 non-fixed, same-sign 26-neighbours, quasi-Euclidean steps, 64-bit atomicMin
//                 on {distance bits, flags, parent} in shared memory) and writes every changed
//                 voxel back with a global 64-bit atomicMin; halo voxels that improved are
//                 pushed to their own tile
// Frontiers are per-voxel bitmasks plus lists (rounds) or a ticket queue (single maps) of active
// (map, tile) pairs, de-duplicated with monotone epoch stamps. The paper processes the open set
// with a priority queue or a FIFO; any processing order reaches the same fixpoint (after the
// raise phase the lower wave computes the greatest fixpoint below the current values of a
// monotone relaxation), so the block-staged schedules give the batch-recompute result.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "launch.h"
#include "vbx_internal.cuh"

namespace cg = cooperative_groups;

namespace vbx {

namespace {

constexpr unsigned kMaxRounds = 1u << 16;
constexpr int kMaxLocalIters = 1 << 15;

// Shared-memory layout of one staged tile: an S^3 sub-block (S = min(B, 8); a 16^3 block is
// staged as eight 8^3 octants, so a round has more independent work items) with its one-voxel
// halo (tile edge T = S + 2).
struct Tile {
  unsigned long long* w;  // T^3 ESDF words, halo included
  uint16_t* a;            // active interior voxels (tile cell index), current
  uint16_t* b;            // active interior voxels, next
  uint32_t* in;           // 2 x S^3 bits: already queued for the next local iteration (by parity)
  uint32_t* chg;          // T^3 bits: word changed in this tile-round
  uint32_t* nslot;        // 27 pool slots of the block and its neighbours
  unsigned* cnt;          // [0..2] rotating list counts (read j%3, append (j+1)%3, clear
                          // (j+2)%3), [3] neighbour tiles to activate in the next-round list,
                          // [4] neighbour tiles whose lower frontier was seeded (bit k = direction
                          // k of the neighbour tile relative to this one)
  uint32_t* lseed;        // T^3 bits: cells the raise wave reset (they join the lower wave and pull)
  int* doff;              // [27] tile cell offset of direction k
  unsigned char* dcls;    // [27] 1, 2 or 3: axes direction k moves along (step v, v*sqrt2, v*sqrt3)
};

#ifndef VBX_TILE_EDGE
#define VBX_TILE_EDGE 8
#endif
constexpr int kTileEdge = VBX_TILE_EDGE;  // sub-block edge S for B >= 8

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

__host__ __device__ inline size_t tile_bytes(int S) {
  const size_t T = S + 2, T3 = T * T * T, S3 = (size_t)S * S * S;
  return align16(T3 * 8) + align16(S3 * 2) * 2 + align16(S3 / 4 < 16 ? 16 : S3 / 4) + align16((T3 + 31) / 32 * 4) +
         align16(27 * 4) + 32 + align16(27 * 4) + 32 + align16((T3 + 31) / 32 * 4);
}

__device__ inline Tile carve(unsigned char* base, int S) {
  const size_t T = S + 2, T3 = T * T * T, S3 = (size_t)S * S * S;
  Tile t;
  size_t off = 0;
  t.w = reinterpret_cast<unsigned long long*>(base + off);
  off += align16(T3 * 8);
  t.a = reinterpret_cast<uint16_t*>(base + off);
  off += align16(S3 * 2);
  t.b = reinterpret_cast<uint16_t*>(base + off);
  off += align16(S3 * 2);
  t.in = reinterpret_cast<uint32_t*>(base + off);
  off += align16(S3 / 4 < 16 ? 16 : S3 / 4);
  t.chg = reinterpret_cast<uint32_t*>(base + off);
  off += align16((T3 + 31) / 32 * 4);
  t.nslot = reinterpret_cast<uint32_t*>(base + off);
  off += align16(27 * 4);
  t.cnt = reinterpret_cast<unsigned*>(base + off);
  off += 32;
  t.doff = reinterpret_cast<int*>(base + off);
  off += align16(27 * 4);
  t.dcls = base + off;
  off += 32;
  t.lseed = reinterpret_cast<uint32_t*>(base + off);
  return t;
}

// Appends v to a shared-memory list with one atomic per coalesced group of lanes.
__device__ __forceinline__ void smem_append(uint16_t* list, unsigned* count, uint16_t v) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned base = 0;
  if (g.thread_rank() == 0) base = atomicAdd(count, g.size());
  base = g.shfl(base, 0);
  list[base + g.thread_rank()] = v;
}

__device__ __forceinline__ void set_bit(uint32_t* bits, uint32_t i) { atomicOr(&bits[i >> 5], 1u << (i & 31)); }

// Adds one to a global counter with one atomic per group of converged lanes that share it (a
// counter that every seed voxel of a scan bumps would otherwise serialise in its L2 slice).
__device__ __forceinline__ void count_one(unsigned* ctr) {
  cg::coalesced_group g = cg::coalesced_threads();
  unsigned* lead = g.shfl(ctr, 0);
  if (g.all(lead == ctr)) {
    if (g.thread_rank() == 0) atomicAdd(ctr, g.size());
  } else {
    atomicAdd(ctr, 1u);
  }
}

// Puts (map, tile) on an active list unless it is already there for this epoch.
__device__ __forceinline__ void activate(uint2* list, unsigned* count, uint32_t* stamps, uint32_t item, unsigned epoch,
                                         unsigned mi) {
  if (__ldcg(&stamps[item]) >= epoch) return;
  if (atomicMax(&stamps[item], epoch) >= epoch) return;
  const unsigned i = atomicAdd(count, 1u);
  list[i] = make_uint2(mi, item);
}

// Tile item (slot * tiles per block + tile index) of a voxel id.
__device__ __forceinline__ uint32_t tile_item_of(const DevMap& m, uint32_t vid) {
  const uint32_t slot = vid >> m.b3log;
  if (m.tile_shift == 0) return slot;
  const uint32_t l = vid & ((1u << m.b3log) - 1u);
  const int B = m.B, blog = m.blog;
  const uint32_t x = l & (B - 1), y = (l >> blog) & (B - 1), z = l >> (2 * blog);
  return (slot << 3) | ((z >> 3) << 2) | ((y >> 3) << 1) | (x >> 3);
}

// ---- tile geometry, templated on the block edge B and the tile edge S so that all index
// arithmetic is by compile-time constants

template <int B, int S>
struct Geo {
  static constexpr int T = S + 2;
  static constexpr int T3 = T * T * T;
  static constexpr int S3 = S * S * S;
  static constexpr int O = B / S;  // tiles per block and axis (1 or 2)
  static constexpr int LOGB = B == 4 ? 2 : (B == 8 ? 3 : 4);
  static constexpr int LOGS = S == 4 ? 2 : (S == 8 ? 3 : 4);
  static_assert((1 << LOGB) == B && (1 << LOGS) == S && S <= B, "tile and block edges are 4, 8 or 16");
  __device__ static __forceinline__ int cell_of_local(int l) {
    return (((l >> (2 * LOGS)) + 1) * T + (((l >> LOGS) & (S - 1)) + 1)) * T + ((l & (S - 1)) + 1);
  }
  __device__ static __forceinline__ int off(int k) { return (k % 3 - 1) * T * T + ((k / 3) % 3 - 1) * T + (k / 9 - 1); }
  __device__ static __forceinline__ void xyz(int c, int* x, int* y, int* z) {
    *x = c % T - 1;
    *y = (c / T) % T - 1;
    *z = c / (T * T) - 1;
  }
};

struct TileRef {
  uint32_t slot;  // pool slot of the block
  int ox, oy, oz;  // tile origin inside the block
  int tx, ty, tz;  // tile coordinates inside the block (0..O-1)
};

template <int B, int S>
__device__ __forceinline__ TileRef tile_ref(uint32_t item) {
  using G = Geo<B, S>;
  TileRef r;
  if (G::O == 1) {
    r.slot = item;
    r.tx = r.ty = r.tz = 0;
  } else {
    r.slot = item >> 3;
    r.tx = item & 1;
    r.ty = (item >> 1) & 1;
    r.tz = (item >> 2) & 1;
  }
  r.ox = r.tx * S;
  r.oy = r.ty * S;
  r.oz = r.tz * S;
  return r;
}

// Voxel id of tile cell c (tile coordinates -1..S per axis); kInvalid if its block is absent.
template <int B, int S>
__device__ __forceinline__ uint32_t cell_vid(const Tile& t, const TileRef& r, int c) {
  using G = Geo<B, S>;
  int x, y, z;
  G::xyz(c, &x, &y, &z);
  x += r.ox;
  y += r.oy;
  z += r.oz;
  const int bx = x < 0 ? -1 : (x >= B ? 1 : 0);
  const int by = y < 0 ? -1 : (y >= B ? 1 : 0);
  const int bz = z < 0 ? -1 : (z >= B ? 1 : 0);
  const uint32_t s = t.nslot[(bx + 1) * 9 + (by + 1) * 3 + (bz + 1)];
  if (s == kInvalid) return kInvalid;
  x -= bx * B;
  y -= by * B;
  z -= bz * B;
  return (s << (3 * G::LOGB)) | (uint32_t)((((z << G::LOGB) | y) << G::LOGB) | x);
}

// Direction (0..26) of the neighbour tile that holds tile cell c, relative to this tile.
template <int B, int S>
__device__ __forceinline__ int cell_tile_dir(int c) {
  using G = Geo<B, S>;
  int x, y, z;
  G::xyz(c, &x, &y, &z);
  const int dx = x < 0 ? -1 : (x >= S ? 1 : 0);
  const int dy = y < 0 ? -1 : (y >= S ? 1 : 0);
  const int dz = z < 0 ? -1 : (z >= S ? 1 : 0);
  return (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1);
}

template <int B, int S>
__device__ __forceinline__ bool cell_interior(int c) {
  using G = Geo<B, S>;
  int x, y, z;
  G::xyz(c, &x, &y, &z);
  return (unsigned)x < (unsigned)S && (unsigned)y < (unsigned)S && (unsigned)z < (unsigned)S;
}

template <int B, int S>
__device__ __forceinline__ int interior_local(int c) {
  using G = Geo<B, S>;
  int x, y, z;
  G::xyz(c, &x, &y, &z);
  return (((z << G::LOGS) | y) << G::LOGS) | x;
}

// Item of the neighbour tile in direction k of this tile (kInvalid if its block is absent).
template <int B, int S>
__device__ __forceinline__ uint32_t neighbor_tile_item(const Tile& t, const TileRef& r, int k) {
  using G = Geo<B, S>;
  int tx = r.tx + (k / 9 - 1), ty = r.ty + ((k / 3) % 3 - 1), tz = r.tz + (k % 3 - 1);
  const int bx = tx < 0 ? -1 : (tx >= G::O ? 1 : 0);
  const int by = ty < 0 ? -1 : (ty >= G::O ? 1 : 0);
  const int bz = tz < 0 ? -1 : (tz >= G::O ? 1 : 0);
  const uint32_t s = t.nslot[(bx + 1) * 9 + (by + 1) * 3 + (bz + 1)];
  if (s == kInvalid) return kInvalid;
  if (G::O == 1) return s;
  tx -= bx * G::O;
  ty -= by * G::O;
  tz -= bz * G::O;
  return (s << 3) | (uint32_t)((tz << 2) | (ty << 1) | tx);
}

// Voxel id and tile direction of tile coordinates (x, y, z) in [-1, S] (kInvalid if absent).
template <int B, int S>
__device__ __forceinline__ uint32_t coords_vid(const Tile& t, const TileRef& r, int x, int y, int z) {
  using G = Geo<B, S>;
  x += r.ox;
  y += r.oy;
  z += r.oz;
  const int bx = x < 0 ? -1 : (x >= B ? 1 : 0);
  const int by = y < 0 ? -1 : (y >= B ? 1 : 0);
  const int bz = z < 0 ? -1 : (z >= B ? 1 : 0);
  const uint32_t s = t.nslot[(bx + 1) * 9 + (by + 1) * 3 + (bz + 1)];
  if (s == kInvalid) return kInvalid;
  x -= bx * B;
  y -= by * B;
  z -= bz * B;
  return (s << (3 * G::LOGB)) | (uint32_t)((((z << G::LOGB) | y) << G::LOGB) | x);
}

template <int S>
__device__ __forceinline__ int coords_tile_dir(int x, int y, int z) {
  const int dx = x < 0 ? -1 : (x >= S ? 1 : 0);
  const int dy = y < 0 ? -1 : (y >= S ? 1 : 0);
  const int dz = z < 0 ? -1 : (z >= S ? 1 : 0);
  return (dx + 1) * 9 + (dy + 1) * 3 + (dz + 1);
}

// Stages tile `item` of map m: the current frontier bits of its interior (cleared in global
// memory, appended to the active list), then its words with the one-voxel halo (one tile row of
// T words per thread, the S interior words of a row read as 16-byte vectors).
template <int NT, int B, int S>
__device__ void stage_tile(const DevMap& m, const TileRef& r, uint32_t* cur_bits, const Tile& t, bool ordered,
                           bool pull = false) {
  using G = Geo<B, S>;
  if (threadIdx.x < 27) {
    const int k = threadIdx.x;
    t.nslot[k] = k == 13 ? r.slot : __ldcg(&m.nbr[(size_t)r.slot * 27 + k]);
    t.doff[k] = G::off(k);
    t.dcls[k] = (unsigned char)((k / 9 != 1) + ((k / 3) % 3 != 1) + (k % 3 != 1));
  }
  if (threadIdx.x < 8) t.cnt[threadIdx.x] = 0u;
  for (int i = threadIdx.x; i < (G::T3 + 31) / 32; i += NT) {
    t.chg[i] = 0u;
    t.lseed[i] = 0u;
  }
  for (int i = threadIdx.x; i < (2 * G::S3 + 31) / 32; i += NT) t.in[i] = 0u;
  __syncthreads();
  // with `pull` (lower wave): the first list is also recorded in the second half of t.in, and
  // the tile's pull marks are taken into a list in t.b (t.cnt[5] entries), which is free until
  // the first local iteration fills it
  uint32_t* first = t.in + (G::S3 / 32 > 0 ? G::S3 / 32 : 1);
  auto take_bits = [&]() {
    // frontier bits: tile row (z, y) = S consecutive bits of the block bitmap, inside one word
    for (int row = threadIdx.x; row < S * S; row += NT) {
      const int z = row / S, y = row % S;
      const uint32_t base = (r.slot << (3 * G::LOGB)) + (uint32_t)((((r.oz + z) << G::LOGB) | (r.oy + y)) << G::LOGB) + r.ox;
      uint32_t* wp = &cur_bits[base >> 5];
      const uint32_t mask = ((1u << S) - 1u) << (base & 31);
      const uint32_t fw = __ldcg(wp);
      const uint32_t pw = pull ? __ldcg(&m.pbits[base >> 5]) : 0u;
      if (fw & mask) {
        uint32_t chunk = (atomicAnd(wp, ~mask) & mask) >> (base & 31);
        const unsigned at = atomicAdd(&t.cnt[0], (unsigned)__popc(chunk));
        unsigned i = at;
        while (chunk) {
          const int x = __ffs(chunk) - 1;
          chunk &= chunk - 1;
          const int nl = (((z << G::LOGS) | y) << G::LOGS) | x;
          t.a[i++] = (uint16_t)G::cell_of_local(nl);
          if (pull) atomicOr(&first[nl >> 5], 1u << (nl & 31));
        }
      }
      if (pw & mask) {
        uint32_t chunk = (atomicAnd(&m.pbits[base >> 5], ~mask) & mask) >> (base & 31);
        unsigned i = atomicAdd(&t.cnt[5], (unsigned)__popc(chunk));
        while (chunk) {
          const int x = __ffs(chunk) - 1;
          chunk &= chunk - 1;
          t.b[i++] = (uint16_t)G::cell_of_local((((z << G::LOGS) | y) << G::LOGS) | x);
        }
      }
    }
  };
  auto load_words = [&]() {
    for (int row = threadIdx.x; row < G::T * G::T; row += NT) {
      const int y = row % G::T - 1, z = row / G::T - 1;
      unsigned long long* dst = &t.w[row * G::T];
      const uint32_t vl = coords_vid<B, S>(t, r, -1, y, z);
      const uint32_t v0 = coords_vid<B, S>(t, r, 0, y, z);
      const uint32_t vr = coords_vid<B, S>(t, r, S, y, z);
      dst[0] = vl == kInvalid ? 0ull : __ldcg(&m.esdf[vl]);
      if (v0 == kInvalid) {
#pragma unroll
        for (int x = 0; x < S; ++x) dst[1 + x] = 0ull;
      } else {
        const ulonglong2* src = reinterpret_cast<const ulonglong2*>(&m.esdf[v0]);
#pragma unroll
        for (int j = 0; j < S / 2; ++j) {
          const ulonglong2 v = __ldcg(&src[j]);
          dst[1 + 2 * j] = v.x;
          dst[2 + 2 * j] = v.y;
        }
      }
      dst[S + 1] = vr == kInvalid ? 0ull : __ldcg(&m.esdf[vr]);
    }
  };
  if (ordered) {
    // asynchronous lower wave: the frontier bits are taken before the words are read. A
    // neighbour writes a voxel's word, fences, then sets its bit, so a bit taken here comes with
    // a word at least that low.
    take_bits();
    __threadfence();
    __syncthreads();
    load_words();
  } else {  // rounds: writers and readers are separated by a grid barrier
    load_words();
    take_bits();
  }
  __syncthreads();
}

// ---- the work queue of a wave (raise, then lower, for single maps). Tiles are taken one at a
// time by tickets (qhead); the first n0 tickets are the wave's initial list (built by
// classification, and for the lower wave also by raise), later ones are tiles
// pushed while the wave runs, each in ring slot (ticket - n0) mod rcap with a publish tag. A
// tile is stamped e0 (its map's epoch) while queued and e0 - 1 once taken, so it is queued at
// most once at a time and is queued again by any write that lands after it was staged.
constexpr long long kMaxWaitSpins = 1ll << 24;
// Largest number of maps with work in one launch for which the waves run as work queues.
#ifndef VBX_ESDF_QUEUE_MAPS
#define VBX_ESDF_QUEUE_MAPS 16
#endif
constexpr unsigned kMaxQueuedMaps = VBX_ESDF_QUEUE_MAPS;

struct WaveQueue {
  EsdfCtl* ctl;
  const uint2* init;  // the initial list (raise: ract0, lower: lact0)
  unsigned n0;        // its length
  unsigned tag_epoch;  // 2 x this launch's call number + phase (0 raise, 1 lower)
};

__device__ __forceinline__ unsigned long long q_pub_tag(unsigned ep, unsigned h) {
  return ((unsigned long long)(2u * ep) << 32) | (0x80000000u | (h & 0x7fffffffu));
}
__device__ __forceinline__ unsigned long long q_read_tag(unsigned ep, unsigned h) {
  return ((unsigned long long)(2u * ep + 1u) << 32) | (0x80000000u | (h & 0x7fffffffu));
}

// Queues tile `item` of map mi unless it is queued already (one thread). The caller makes the
// frontier bits it set for this tile visible first (each writing thread fences, then a CTA
// barrier), so that a tile found still queued here is staged after those bits landed.
__device__ void q_push(const WaveQueue& q, unsigned mi, uint32_t item, uint32_t* stamps, unsigned e0) {
  if (__ldcg(&stamps[item]) >= e0) return;
  if (atomicMax(&stamps[item], e0) >= e0) return;
  EsdfCtl* ctl = q.ctl;
  const unsigned h = q.n0 + atomicAdd(&ctl->qtail, 1u);
  const unsigned slot = (h - q.n0) % ctl->rcap;
  unsigned long long* tag = &ctl->ltag[slot];
  if (h - q.n0 >= ctl->rcap) {  // the ticket that used this slot before must have been read
    const unsigned long long want = q_read_tag(q.tag_epoch, h - ctl->rcap);
    long long spins = 0;
    while (*(volatile unsigned long long*)tag != want) {
      if (++spins > kMaxWaitSpins || *(volatile unsigned*)&ctl->error) {
        atomicOr(&ctl->error, kErrTimeout);
        return;
      }
      __nanosleep(64);
    }
  }
  ctl->lring[slot] = make_uint2(mi, item);
  __threadfence();
  // fire and forget: termination counts tickets (qtail, whose increment has completed), not
  // publications, so a late tag only keeps the ticket's taker waiting a little longer
  atomicExch(tag, q_pub_tag(q.tag_epoch, h));
}

// Reads the published tile of ring ticket h and marks the slot free for reuse.
__device__ __forceinline__ void q_read_slot(const WaveQueue& q, unsigned h, uint2* out) {
  EsdfCtl* ctl = q.ctl;
  const unsigned slot = (h - q.n0) % ctl->rcap;
  __threadfence();
  *out = __ldcg(&ctl->lring[slot]);  // L2: the producer's store on another SM
  __threadfence();
  atomicExch(&ctl->ltag[slot], q_read_tag(q.tag_epoch, h));
}

// Resolves ticket h without waiting (one thread): 1 with the tile in *out, 0 if its tile has not
// been published yet.
__device__ int q_try(const WaveQueue& q, unsigned h, uint2* out) {
  if (h < q.n0) {
    *out = __ldcg(&q.init[h]);
    return 1;
  }
  const unsigned slot = (h - q.n0) % q.ctl->rcap;
  if (*(volatile unsigned long long*)&q.ctl->ltag[slot] != q_pub_tag(q.tag_epoch, h)) return 0;
  q_read_slot(q, h, out);
  return 1;
}

// Waits for ticket h (one thread): 1 with the tile in *out, 0 once the queue has drained (every
// produced ticket finished, so no tile can be queued any more), -1 on error.
__device__ int q_wait(const WaveQueue& q, unsigned h, uint2* out) {
  EsdfCtl* ctl = q.ctl;
  if (h < q.n0) {
    *out = __ldcg(&q.init[h]);
    return 1;
  }
  const unsigned slot = (h - q.n0) % ctl->rcap;
  unsigned long long* tag = &ctl->ltag[slot];
  const unsigned long long want = q_pub_tag(q.tag_epoch, h);
  long long spins = 0;
  for (;;) {
    if (*(volatile unsigned long long*)tag == want) break;
    // finished items are read strictly before produced tickets: if every ticket produced so far
    // had finished when qdone was read, no tile was being processed then, so none can be
    // queued later (a pushing tile is counted finished only after its tickets are visible)
    const unsigned done = *(volatile unsigned*)&ctl->qdone;
    __threadfence();
    const unsigned made = q.n0 + *(volatile unsigned*)&ctl->qtail;
    if (done == made && h >= made) return 0;
    if (*(volatile unsigned*)&ctl->error) return -1;
    if (++spins > kMaxWaitSpins) {
      atomicOr(&ctl->error, kErrTimeout);
      return -1;
    }
    __nanosleep(64);
  }
  q_read_slot(q, h, out);
  return 1;
}

// The CTA's next ticket, taken while its current tile is written back (by kAheadThread, of a warp
// that has no push to make), so that taking it and reading its tile overlap with the write-back's
// fences instead of following them. Holding a ticket that long delays its tile by at most one
// write-back.
struct QueueAhead {
  unsigned h;
  int st;  // 0 none, 1 ticket h taken, 2 ticket h's tile in e
  uint2 e;
};
constexpr int kAheadThread = 32;

__device__ __forceinline__ void q_ahead_resolve(const WaveQueue& q, unsigned h, QueueAhead* a) {
  uint2 e = make_uint2(0u, 0u);
  a->st = q_try(q, h, &e) ? 2 : 1;
  a->h = h;
  a->e = e;
}

// Next tile of the CTA (thread 0): the one taken ahead, else a fresh ticket; as q_wait.
__device__ int q_next(const WaveQueue& q, QueueAhead* a, uint2* out) {
  const int st = a->st;
  a->st = 0;
  if (st == 2) {
    *out = a->e;
    return 1;
  }
  return q_wait(q, st == 1 ? a->h : atomicAdd(&q.ctl->qhead, 1u), out);
}

struct RoundArgs {
  unsigned mi;       // map index in the group
  unsigned ep_next;  // activation epoch of the next round
  unsigned e0;       // epoch of the frontiers seeded by classification
  uint32_t* nxt_bits;
  uint2* nxt_list;
  unsigned* nxt_cnt;
  const WaveQueue* q;  // asynchronous waves: where neighbour tiles are queued
  QueueAhead* ahead;   // and where the CTA's next ticket is taken ahead
};

// A7 for one staged tile (all threads of the CTA).
template <int NT, int B, int S>
__device__ void raise_tile(const DevMap& m, uint32_t item, uint32_t* cur_bits, const RoundArgs& ra, EsdfCtl* ctl,
                           unsigned char* smem) {
  using G = Geo<B, S>;
  const Tile t = carve(smem, S);
  const TileRef r = tile_ref<B, S>(item);
  stage_tile<NT, B, S>(m, r, cur_bits, t, false);
  const float dmax = m.dmax;
  unsigned iters = 0;
  unsigned long long pops = 0;
  for (int it = 0;; ++it) {
    const unsigned na = t.cnt[it % 3];
    if (na == 0) break;
    if (it > kMaxLocalIters) {
      if (threadIdx.x == 0) atomicOr(&ctl->error, kErrTimeout);
      break;
    }
    ++iters;
    const uint16_t* cur = (it & 1) ? t.b : t.a;
    uint16_t* nxt = (it & 1) ? t.a : t.b;
    unsigned* ncnt = &t.cnt[(it + 1) % 3];
    uint32_t* inb = t.in + (it & 1) * (G::S3 / 32 > 0 ? G::S3 / 32 : 1);
    pops += na;
    if (threadIdx.x == 0) t.cnt[(it + 2) % 3] = 0u;
    for (int j = threadIdx.x; j < (G::S3 + 31) / 32; j += NT)
      t.in[((it + 1) & 1) * (G::S3 / 32 > 0 ? G::S3 / 32 : 1) + j] = 0u;
    // reset the raised voxels; each joins the lower frontier itself and takes its new value from
    // its neighbours when the lower wave stages its tile (its other observed neighbours, whose
    // values stand, would otherwise all be popped to offer it theirs). No barrier before the
    // child tests below: a test that still sees the old parent of a voxel raised in this same
    // iteration raises it once more, which only costs a pop.
    for (unsigned i = threadIdx.x; i < na; i += NT) {
      const int c = cur[i];
      const unsigned long long w = t.w[c];
      const unsigned fl = ew_flags(w);
      if (!(fl & kFixed)) {
        t.w[c] = ew_pack(ew_d(w) < 0.0f ? -dmax : dmax, fl, kNoParent);
        atomicOr(&t.chg[c >> 5], 1u << (c & 31));
        atomicOr(&t.lseed[c >> 5], 1u << (c & 31));
      }
    }
    for (unsigned p = threadIdx.x; p < na * 26u; p += NT) {
      const unsigned i = p / 26u;
      const int kk = (int)(p - i * 26u);
      const int k = kk < 13 ? kk : kk + 1;
      const int c = cur[i];
      const int nc = c + t.doff[k];
      const unsigned long long nw = t.w[nc];
      const unsigned nfl = ew_flags(nw);
      if (!(nfl & kObserved)) continue;
      if (!(nfl & kFixed) && ew_parent(nw) == (unsigned)(26 - k)) {  // a child: raise it
        if (cell_interior<B, S>(nc)) {
          const int nl = interior_local<B, S>(nc);
          const uint32_t bit = 1u << (nl & 31);
          if (!(atomicOr(&inb[nl >> 5], bit) & bit)) smem_append(nxt, ncnt, (uint16_t)nc);
        } else {
          set_bit(ra.nxt_bits, cell_vid<B, S>(t, r, nc));
          atomicOr(&t.cnt[3], 1u << cell_tile_dir<B, S>(nc));
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // drained during the write-back's fences
    atomicAdd(&m.ctr->esdf_local_iters, iters);
    if (pops) atomicAdd(&m.ctr->raise_pops, pops);
    atomicAdd(&m.ctr->esdf_block_visits, 1u);
  }
  unsigned ahead = 0;  // the CTA's next ticket
  if (ra.q && threadIdx.x == kAheadThread) ahead = atomicAdd(&ra.q->ctl->qhead, 1u);
  // write back the raised voxels (raise rounds never lower words, plain stores suffice); each
  // joins the lower frontier and pulls
  for (int c = threadIdx.x; c < G::T3; c += NT) {
    if (t.chg[c >> 5] & (1u << (c & 31))) m.esdf[cell_vid<B, S>(t, r, c)] = t.w[c];
    if (t.lseed[c >> 5] & (1u << (c & 31))) {
      const uint32_t vid = cell_vid<B, S>(t, r, c);
      set_bit(m.pbits, vid);
      set_bit(m.lbits0, vid);
      atomicOr(&t.cnt[4], 1u << cell_tile_dir<B, S>(c));
    }
  }
  __syncthreads();
  // activate the tiles that received raise (next round, or the queue) or lower (seed) bits
  if (ra.q) {  // the raise bits set by any thread precede the pushes' stamp checks
    __threadfence();
    __syncthreads();
  }
  if (threadIdx.x < 27) {
    const int k = threadIdx.x;
    const bool rz = t.cnt[3] >> k & 1u, lz = t.cnt[4] >> k & 1u;
    if (rz || lz) {
      const uint32_t nit = neighbor_tile_item<B, S>(t, r, k);
      if (nit != kInvalid) {
        if (rz) {
          if (ra.q)
            q_push(*ra.q, ra.mi, nit, m.bstamp_r, ra.e0);
          else
            activate(ra.nxt_list, ra.nxt_cnt, m.bstamp_r, nit, ra.ep_next, ra.mi);
        }
        if (lz) activate(ctl->lact0, &ctl->lcnt[0], m.bstamp_l, nit, ra.e0, ra.mi);
      }
    }
  }
  if (ra.q && threadIdx.x == kAheadThread) q_ahead_resolve(*ra.q, ahead, ra.ahead);
  __syncthreads();
}

// A8 for one staged tile (all threads of the CTA).
template <int NT, int B, int S>
__device__ void lower_tile(const DevMap& m, uint32_t item, uint32_t* cur_bits, const RoundArgs& ra, EsdfCtl* ctl,
                           unsigned char* smem) {
  using G = Geo<B, S>;
  const Tile t = carve(smem, S);
  const TileRef r = tile_ref<B, S>(item);
  stage_tile<NT, B, S>(m, r, cur_bits, t, ra.q != nullptr, true);
  const float L1 = m.L1, L2 = m.L2, L3 = m.L3;
  // a voxel lowered to |d| with |d| + v >= d_max cannot lower any neighbour (no value exceeds
  // d_max), so it is written back but not put on a frontier
  const float reach = m.dmax;
  // Voxels marked to pull (raised, or newly observed; staging listed the marks it took in t.b)
  // take the best offer of their observed same-sign neighbours: the least word {|d_n| + step,
  // flags, direction}, the choice the atomicMin of pushes from all those neighbours would make.
  // A mark is set with the voxel's frontier bit before the wave, so the staging that takes one
  // normally takes the other; if the value drops and another visit took the frontier bit, this
  // visit's first list gets the voxel too.
  {
    const uint32_t* first = t.in + (G::S3 / 32 > 0 ? G::S3 / 32 : 1);
    for (unsigned i = threadIdx.x; i < t.cnt[5]; i += NT) {
      {
        const int c = t.b[i];
        const unsigned long long w = t.w[c];
        const unsigned fl = ew_flags(w);
        const bool neg = ew_d(w) < 0.0f;
        unsigned long long best = w;
        for (int k = 0; k < 27; ++k) {
          if (k == 13) continue;
          const unsigned long long nw = t.w[c + t.doff[k]];
          const float dn = ew_d(nw);
          if (!(ew_flags(nw) & kObserved) || (dn < 0.0f) != neg) continue;
          const int n1 = t.dcls[k];
          const float cand = __fadd_rn(fabsf(dn), n1 == 1 ? L1 : (n1 == 2 ? L2 : L3));
          const unsigned long long cw = ew_pack(neg ? -cand : cand, fl, (unsigned)k);
          if (cw < best) best = cw;
        }
        if (best < w) {
          atomicMin(&t.w[c], best);
          atomicOr(&t.chg[c >> 5], 1u << (c & 31));
          const int nl = interior_local<B, S>(c);
          if (!(first[nl >> 5] & (1u << (nl & 31)))) smem_append(t.a, &t.cnt[0], (uint16_t)c);
        }
      }
    }
    __syncthreads();
  }
  // First-list voxels with |d| + v >= d_max cannot lower any neighbour (no value exceeds d_max):
  // above all new or raised voxels inside a new or raised region, which found no offer. They
  // leave the list (through t.b, free again) before their 26 neighbour checks.
  {
    for (unsigned i = threadIdx.x; i < t.cnt[0]; i += NT) {
      const int c = t.a[i];
      if (__fadd_rn(fabsf(ew_d(t.w[c])), L1) < reach) smem_append(t.b, &t.cnt[6], (uint16_t)c);
    }
    __syncthreads();
    const unsigned n = t.cnt[6];
    for (unsigned i = threadIdx.x; i < n; i += NT) t.a[i] = t.b[i];
    __syncthreads();
    if (threadIdx.x == 0) t.cnt[0] = n;
    __syncthreads();
  }
  // this lane's direction for the visit (lanes 26-31 take direction 0 and stay idle)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int k = (lane < 13 ? lane : lane + 1) % 27;
  const int dk = t.doff[k];
  const float Lk = t.dcls[k] == 1 ? L1 : (t.dcls[k] == 2 ? L2 : L3);
  unsigned iters = 0;
  unsigned long long pops = 0;
  for (int it = 0;; ++it) {
    const unsigned na = t.cnt[it % 3];
    if (na == 0) break;
    if (it > kMaxLocalIters) {
      if (threadIdx.x == 0) atomicOr(&ctl->error, kErrTimeout);
      break;
    }
    ++iters;
    const uint16_t* cur = (it & 1) ? t.b : t.a;
    uint16_t* nxt = (it & 1) ? t.a : t.b;
    unsigned* ncnt = &t.cnt[(it + 1) % 3];
    uint32_t* inb = t.in + (it & 1) * (G::S3 / 32 > 0 ? G::S3 / 32 : 1);
    pops += na;
    if (threadIdx.x == 0) t.cnt[(it + 2) % 3] = 0u;
    for (int j = threadIdx.x; j < (G::S3 + 31) / 32; j += NT)
      t.in[((it + 1) & 1) * (G::S3 / 32 > 0 ? G::S3 / 32 : 1) + j] = 0u;
    // one voxel per warp, one of its 26 directions per lane (lanes 26-31 idle): the voxel's word
    // is one broadcast, and each lane's offset and step stay in registers for the whole visit
    for (unsigned i = (unsigned)wid; i < na; i += NT / 32) {
      const int c = cur[i];
      const unsigned long long w = t.w[c];
      if (lane >= 26 || !(ew_flags(w) & kObserved)) continue;
      const float dv = ew_d(w);
      const bool neg = dv < 0.0f;
      const int nc = c + dk;
      const unsigned long long nw = t.w[nc];
      const unsigned nfl = ew_flags(nw);
      if ((nfl & (kObserved | kFixed)) != kObserved) continue;
      const float dn = ew_d(nw);
      if ((dn < 0.0f) != neg) continue;
      const float cand = __fadd_rn(fabsf(dv), Lk);
      if (!(cand < fabsf(dn))) continue;
      const unsigned long long old = atomicMin(&t.w[nc], ew_pack(neg ? -cand : cand, nfl, (unsigned)(26 - k)));
      if (!(fabsf(ew_d(old)) > cand)) continue;
      atomicOr(&t.chg[nc >> 5], 1u << (nc & 31));
      if (cell_interior<B, S>(nc) && __fadd_rn(cand, L1) < reach) {
        const int nl = interior_local<B, S>(nc);
        const uint32_t bit = 1u << (nl & 31);
        if (!(atomicOr(&inb[nl >> 5], bit) & bit)) smem_append(nxt, ncnt, (uint16_t)nc);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // drained during the write-back's fences
    atomicAdd(&m.ctr->esdf_local_iters, iters);
    if (pops) atomicAdd(&m.ctr->lower_pops, pops);
    atomicAdd(&m.ctr->esdf_block_visits, 1u);
  }
  const bool async = ra.q != nullptr;
  unsigned ahead = 0;  // the CTA's next ticket
  if (async && threadIdx.x == kAheadThread) ahead = atomicAdd(&ra.q->ctl->qhead, 1u);
  // write back: the global word keeps the smaller value (fire-and-forget atomicMin); a halo
  // voxel this tile lowered is pushed to its own tile for the next round (a push of a voxel
  // that another tile lowered even further is redundant work, never wrong)
  for (int c = threadIdx.x; c < G::T3; c += NT) {
    if (!(t.chg[c >> 5] & (1u << (c & 31)))) continue;
    const uint32_t vid = cell_vid<B, S>(t, r, c);
    const unsigned long long w = t.w[c];
    atomicMin(&m.esdf[vid], w);
    if (ra.q == nullptr && !cell_interior<B, S>(c) && __fadd_rn(fabsf(ew_d(w)), L1) < reach) {
      set_bit(ra.nxt_bits, vid);  // rounds: the bit goes with the value
      atomicOr(&t.cnt[3], 1u << cell_tile_dir<B, S>(c));
    }
  }
  // asynchronous wave: values before frontier bits (a tile that takes a bit must find the word
  // at least that low), and bits before the pushes of the tiles that own them
  if (async) {
    __threadfence();
    __syncthreads();
    for (int c = threadIdx.x; c < G::T3; c += NT) {
      if (!(t.chg[c >> 5] & (1u << (c & 31))) || cell_interior<B, S>(c)) continue;
      if (!(__fadd_rn(fabsf(ew_d(t.w[c])), L1) < reach)) continue;
      set_bit(ra.nxt_bits, cell_vid<B, S>(t, r, c));
      atomicOr(&t.cnt[3], 1u << cell_tile_dir<B, S>(c));
    }
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x < 27 && (t.cnt[3] >> threadIdx.x & 1u)) {
    const uint32_t nit = neighbor_tile_item<B, S>(t, r, threadIdx.x);
    if (nit != kInvalid) {
      if (async)
        q_push(*ra.q, ra.mi, nit, m.bstamp_l, ra.e0);
      else
        activate(ra.nxt_list, ra.nxt_cnt, m.bstamp_l, nit, ra.ep_next, ra.mi);
    }
  }
  if (async && threadIdx.x == kAheadThread) q_ahead_resolve(*ra.q, ahead, ra.ahead);
  __syncthreads();
}

// BE: the block edge the kernel was compiled for (0: any, chosen per tile from the map)
template <int NT, int BE>
__device__ __forceinline__ void raise_dispatch(const DevMap& m, uint32_t item, uint32_t* cur_bits, const RoundArgs& ra,
                                               EsdfCtl* ctl, unsigned char* smem) {
  if constexpr (BE == 4) {
    raise_tile<NT, 4, 4>(m, item, cur_bits, ra, ctl, smem);
  } else if constexpr (BE == 8) {
    raise_tile<NT, 8, 8>(m, item, cur_bits, ra, ctl, smem);
  } else if constexpr (BE == 16) {
    raise_tile<NT, 16, kTileEdge>(m, item, cur_bits, ra, ctl, smem);
  } else {
    switch (m.B) {
      case 4: raise_tile<NT, 4, 4>(m, item, cur_bits, ra, ctl, smem); break;
      case 8: raise_tile<NT, 8, 8>(m, item, cur_bits, ra, ctl, smem); break;
      default: raise_tile<NT, 16, kTileEdge>(m, item, cur_bits, ra, ctl, smem); break;
    }
  }
}

// BE: the block edge the kernel was compiled for (0: any, chosen per tile from the map)
template <int NT, int BE>
__device__ __forceinline__ void lower_dispatch(const DevMap& m, uint32_t item, uint32_t* cur_bits, const RoundArgs& ra,
                                               EsdfCtl* ctl, unsigned char* smem) {
  if constexpr (BE == 4) {
    lower_tile<NT, 4, 4>(m, item, cur_bits, ra, ctl, smem);
  } else if constexpr (BE == 8) {
    lower_tile<NT, 8, 8>(m, item, cur_bits, ra, ctl, smem);
  } else if constexpr (BE == 16) {
    lower_tile<NT, 16, kTileEdge>(m, item, cur_bits, ra, ctl, smem);
  } else {
    switch (m.B) {
      case 4: lower_tile<NT, 4, 4>(m, item, cur_bits, ra, ctl, smem); break;
      case 8: lower_tile<NT, 8, 8>(m, item, cur_bits, ra, ctl, smem); break;
      default: lower_tile<NT, 16, kTileEdge>(m, item, cur_bits, ra, ctl, smem); break;
    }
  }
}

__device__ __forceinline__ unsigned upper_index(const unsigned* pfx, int n, unsigned i) {
  // largest mi with pfx[mi] <= i
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pfx[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  return (unsigned)lo;
}

// NT threads per CTA, at least MINB CTAs per SM worth of registers: the 128- and 256-thread
// batch shapes are held to 12 and 6 per SM (more tiles in flight per SM outweigh a few spilled
// registers). BE != 0 compiles the kernel for one map of block edge BE whose waves run as work
// queues (a single map's large update, 256 x 8 per SM): without the other tile geometries and the
// round schedule it fits 32 registers with about 50 B of spills (the general kernel: over 450 B).
template <int NT, int MINB, int BE>
__global__ void __launch_bounds__(NT, MINB) k_esdf(const DevMap* __restrict__ maps, int nmaps, EsdfCtl* ctl, int allow_async) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ unsigned pfx[kMaxBatch + 1];
  __shared__ QueueAhead sh_ahead;
  __shared__ unsigned sh_item;
  __shared__ int sh_state;
  __shared__ uint2 sh_e;
  __shared__ unsigned long long sh_t[4];  // phase boundaries, taken by thread 0 of each CTA
  __shared__ unsigned sh_active;          // maps with dirty voxels in this launch
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nthreads = gridDim.x * blockDim.x;
  if (threadIdx.x == 0) sh_t[0] = global_ns();
  if (tid == 0) atomicAdd(&ctl->calls, 1u);  // read by every CTA after the first grid barrier

  // ---------------------------------------------------------------- A6: classification
  // exclusive prefix of the maps' dirty counts: warp 0 scans kMaxBatch / 32 counts per lane
  if (threadIdx.x < 32) {
    constexpr int per = kMaxBatch / 32;
    unsigned v[per];
    unsigned sum = 0;
#pragma unroll
    for (int j = 0; j < per; ++j) {
      const int mi = (int)threadIdx.x * per + j;
      v[j] = mi < nmaps ? __ldcg(&maps[mi].ctr->ndirty) : 0u;
      sum += v[j];
    }
    unsigned incl = sum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned up = __shfl_up_sync(0xffffffffu, incl, off);
      if ((int)threadIdx.x >= off) incl += up;
    }
    unsigned run = incl - sum;
    unsigned act = 0;
#pragma unroll
    for (int j = 0; j < per; ++j) act += v[j] > 0u ? 1u : 0u;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) act += __shfl_xor_sync(0xffffffffu, act, off);
    if (threadIdx.x == 0) sh_active = act;
    if (threadIdx.x == 0) pfx[0] = 0u;
#pragma unroll
    for (int j = 0; j < per; ++j) {
      run += v[j];
      pfx[threadIdx.x * per + j + 1] = run;
    }
  }
  __syncthreads();
  const unsigned total = pfx[nmaps];
  // Schedule of the raise and lower waves (every CTA decides alike, from the same counts): with
  // few maps at work, rounds would hold a few tiles each and wait for their slowest one, so the
  // waves run as work queues; with many, rounds are full and cheaper.
  const bool async_lower = BE != 0 || (allow_async && sh_active <= kMaxQueuedMaps);
  // the queue's ring must hold every tile plus 27 pushes per CTA in flight
  if (async_lower && ctl->rcap < ctl->cap + 27u * gridDim.x) {
    if (tid == 0) atomicOr(&ctl->error, kErrTimeout);
    return;
  }
  for (unsigned i = tid; i < total; i += nthreads) {
    const unsigned mi = upper_index(pfx, nmaps, i);
    const DevMap& m = maps[mi];
    const uint32_t vid = m.dirty[i - pfx[mi]];
    const unsigned e0 = __ldcg(&m.ctr->epoch) + 1;
    const float dmax = m.dmax;
    m.vflags[vid] = (uint8_t)(m.vflags[vid] & ~kQueuedForEsdf);
    const float2 t = m.tsdf[vid];
    if (!(t.y > 0.0f)) continue;
    const float Df = t.x == 0.0f ? 0.0f : t.x;  // sign(0) = +1
    // fixed band |D| < gamma (Sec. V-A), or occupancy: D < 0 is occupied at distance 0 and
    // every other observed voxel is positive (the occupancy ESDF of Sec. VI-B)
    const bool occ = m.esdf_mode == 1;
    const bool neg = !occ && Df < 0.0f;
    const bool fixed_now = occ ? Df < 0.0f : fabsf(Df) < m.gamma;
    const float seedv = occ ? 0.0f : Df;
    const float sdmax = neg ? -dmax : dmax;
    const unsigned long long w = __ldcg(&m.esdf[vid]);
    const unsigned fl = ew_flags(w);
    const bool obs = (fl & kObserved) != 0;
    const float de = ew_d(w);
    const uint32_t slot = tile_item_of(m, vid);
    if (fixed_now) {  // isFixed, evaluated on the TSDF voxel
      count_one(&m.ctr->seeds);
      const bool lower_only = !obs || (((de < 0.0f) == neg) && fabsf(seedv) <= fabsf(de));
      m.esdf[vid] = ew_pack(seedv, kObserved | kFixed, kNoParent);
      if (!lower_only) {
        set_bit(m.rbits0, vid);
        activate(ctl->ract0, &ctl->rcnt[0], m.bstamp_r, slot, e0, mi);
      }
      set_bit(m.lbits0, vid);
      activate(ctl->lact0, &ctl->lcnt[0], m.bstamp_l, slot, e0, mi);
    } else if (fl & kFixed) {  // leaves the fixed band
      m.esdf[vid] = ew_pack(sdmax, kObserved, kNoParent);
      set_bit(m.rbits0, vid);
      activate(ctl->ract0, &ctl->rcnt[0], m.bstamp_r, slot, e0, mi);
    } else if (!obs) {
      // newly observed: it joins the lower frontier itself and takes its value from its
      // neighbours when the lower wave stages its tile (one pull instead of a frontier entry for
      // every neighbour that could lower it)
      m.esdf[vid] = ew_pack(sdmax, kObserved, kNoParent);
      set_bit(m.pbits, vid);
      set_bit(m.lbits0, vid);
      activate(ctl->lact0, &ctl->lcnt[0], m.bstamp_l, slot, e0, mi);
    } else if ((de < 0.0f) != neg) {  // sign flip of a propagated voxel
      m.esdf[vid] = ew_pack(sdmax, kObserved, kNoParent);
      set_bit(m.rbits0, vid);
      activate(ctl->ract0, &ctl->rcnt[0], m.bstamp_r, slot, e0, mi);
    }
  }
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->error)) return;
  if (threadIdx.x == 0) sh_t[1] = global_ns();

  // ------------------------------------------------------------------------ A7: raise
  // The raised set is the closure over parent directions from the classified voxels, and
  // parent directions do not change while the wave runs, so its result does not depend on the
  // schedule either: rounds for batches, the work queue for single maps (then the queue's
  // counters are reset between two grid barriers for the lower wave).
  unsigned r = 0;
  if (async_lower) {
    WaveQueue q;
    q.ctl = ctl;
    q.init = ctl->ract0;
    q.n0 = __ldcg(&ctl->rcnt[0]);
    q.tag_epoch = 2u * __ldcg(&ctl->calls);
    r = q.n0 > 0 ? 1u : 0u;  // reported as one raise "round"
    if (threadIdx.x == 0) sh_ahead.st = 0;
    for (;;) {
      if (threadIdx.x == 0) {
        uint2 e = make_uint2(0u, 0u);
        const int st = q_next(q, &sh_ahead, &e);
        if (st == 1) {
          const DevMap& m = maps[e.x];
          atomicExch(&m.bstamp_r[e.y], __ldcg(&m.ctr->epoch));  // e0 - 1: no longer queued
          __threadfence();  // and the CTA barrier below orders this before the tile's bit reads
        }
        sh_state = st;
        sh_e = e;
      }
      __syncthreads();
      const int st = sh_state;
      const uint2 e = sh_e;
      if (st != 1) break;
      const DevMap& m = maps[e.x];
      RoundArgs ra;
      ra.mi = e.x;
      ra.e0 = __ldcg(&m.ctr->epoch) + 1;
      ra.ep_next = ra.e0;
      ra.nxt_bits = m.rbits0;
      ra.nxt_list = nullptr;
      ra.nxt_cnt = nullptr;
      ra.q = &q;
      ra.ahead = &sh_ahead;
      raise_dispatch<NT, BE>(m, e.y, m.rbits0, ra, ctl, dsm);
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&ctl->qdone, 1u);
      }
    }
    if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->error)) return;
    if (tid == 0) {
      ctl->qhead = 0u;
      ctl->qtail = 0u;
      ctl->qdone = 0u;
    }
    if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->error)) return;
  } else {
    for (;; ++r) {
      const unsigned cnt = __ldcg(&ctl->rcnt[r % 3]);
      if (cnt == 0 || __ldcg(&ctl->error)) break;
      if (r >= kMaxRounds) {
        if (tid == 0) atomicOr(&ctl->error, kErrTimeout);
        break;
      }
      if (tid == 0) {
        ctl->rcnt[(r + 2) % 3] = 0;
        ctl->rnext[(r + 2) % 3] = 0;
      }
      const uint2* cur = (r & 1) ? ctl->ract1 : ctl->ract0;
      for (;;) {
        if (threadIdx.x == 0) sh_item = atomicAdd(&ctl->rnext[r % 3], 1u);
        __syncthreads();
        const unsigned item = sh_item;
        __syncthreads();
        if (item >= cnt) break;
        const uint2 e = cur[item];
        const DevMap& m = maps[e.x];
        RoundArgs ra;
        ra.mi = e.x;
        ra.e0 = __ldcg(&m.ctr->epoch) + 1;
        ra.ep_next = ra.e0 + 1 + r;
        ra.nxt_bits = (r & 1) ? m.rbits0 : m.rbits1;
        ra.nxt_list = (r & 1) ? ctl->ract0 : ctl->ract1;
        ra.nxt_cnt = &ctl->rcnt[(r + 1) % 3];
        ra.q = nullptr;
        ra.ahead = nullptr;
        raise_dispatch<NT, BE>(m, e.y, (r & 1) ? m.rbits1 : m.rbits0, ra, ctl, dsm);
      }
      if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->error)) return;
    }
  }
  const unsigned raise_rounds = r;
  if (threadIdx.x == 0) sh_t[2] = global_ns();

  // ------------------------------------------------------------------------ A8: lower
  // Two schedules reach the same fixpoint (the lower wave is a monotone relaxation: values only
  // decrease, by global atomicMin, so neither the processing order nor two CTAs working on
  // neighbouring tiles at once change the result):
  //  * rounds (batches): all tiles active in a round, then a grid barrier; many maps keep every
  //    round full of tiles;
  //  * one asynchronous work queue (single maps, whose rounds hold about one tile per SM): each
  //    CTA takes a tile, un-stamps it (a write into it from then on queues it again), relaxes it
  //    to local convergence and queues the neighbour tiles whose voxels it lowered, with no grid
  //    barrier; the phase ends when every produced ticket has finished.
  unsigned l = 0;
  if (async_lower) {
    WaveQueue q;
    q.ctl = ctl;
    q.init = ctl->lact0;
    q.n0 = __ldcg(&ctl->lcnt[0]);
    q.tag_epoch = 2u * __ldcg(&ctl->calls) + 1u;
    l = q.n0 > 0 ? 1u : 0u;  // reported as one lower "round"
    if (threadIdx.x == 0) sh_ahead.st = 0;
    for (;;) {
      if (threadIdx.x == 0) {
        uint2 e = make_uint2(0u, 0u);
        const int st = q_next(q, &sh_ahead, &e);
        if (st == 1) {
          const DevMap& m = maps[e.x];
          atomicExch(&m.bstamp_l[e.y], __ldcg(&m.ctr->epoch));  // e0 - 1: no longer queued
          // the un-stamping is ordered (this fence, then the CTA barrier) before the CTA's reads
          // of the tile's frontier bits: a neighbour that sets a bit after those reads then sees
          // the tile as not queued
          __threadfence();
        }
        sh_state = st;
        sh_e = e;
      }
      __syncthreads();
      const int st = sh_state;
      const uint2 e = sh_e;
      if (st != 1) break;
      const DevMap& m = maps[e.x];
      RoundArgs ra;
      ra.mi = e.x;
      ra.e0 = __ldcg(&m.ctr->epoch) + 1;
      ra.ep_next = ra.e0;
      ra.nxt_bits = m.lbits0;
      ra.nxt_list = nullptr;
      ra.nxt_cnt = nullptr;
      ra.q = &q;
      ra.ahead = &sh_ahead;
      lower_dispatch<NT, BE>(m, e.y, m.lbits0, ra, ctl, dsm);
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&ctl->qdone, 1u);
      }
    }
  } else {
    for (;; ++l) {
      const unsigned cnt = __ldcg(&ctl->lcnt[l % 3]);
      if (cnt == 0 || __ldcg(&ctl->error)) break;
      if (l >= kMaxRounds) {
        if (tid == 0) atomicOr(&ctl->error, kErrTimeout);
        break;
      }
      if (tid == 0) {
        ctl->lcnt[(l + 2) % 3] = 0;
        ctl->lnext[(l + 2) % 3] = 0;
      }
      const uint2* cur = (l & 1) ? ctl->lact1 : ctl->lact0;
      for (;;) {
        if (threadIdx.x == 0) sh_item = atomicAdd(&ctl->lnext[l % 3], 1u);
        __syncthreads();
        const unsigned item = sh_item;
        __syncthreads();
        if (item >= cnt) break;
        const uint2 e = cur[item];
        const DevMap& m = maps[e.x];
        RoundArgs ra;
        ra.mi = e.x;
        ra.e0 = __ldcg(&m.ctr->epoch) + 1;
        ra.ep_next = ra.e0 + 1 + l;
        ra.nxt_bits = (l & 1) ? m.lbits0 : m.lbits1;
        ra.nxt_list = (l & 1) ? ctl->lact0 : ctl->lact1;
        ra.nxt_cnt = &ctl->lcnt[(l + 1) % 3];
        ra.q = nullptr;
        ra.ahead = nullptr;
        lower_dispatch<NT, BE>(m, e.y, (l & 1) ? m.lbits1 : m.lbits0, ra, ctl, dsm);
      }
      if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->error)) return;
    }
  }
  if (threadIdx.x == 0) sh_t[3] = global_ns();
  __syncthreads();
  for (unsigned i = tid; i < (unsigned)nmaps; i += nthreads) {
    Counters* c = maps[i].ctr;
    c->esdf_phase_ns[0] = (unsigned)(sh_t[1] - sh_t[0]);
    c->esdf_phase_ns[1] = (unsigned)(sh_t[2] - sh_t[1]);
    c->esdf_phase_ns[2] = (unsigned)(sh_t[3] - sh_t[2]);
    c->esdf_in = pfx[i + 1] - pfx[i];
    c->raise_rounds = raise_rounds;
    c->lower_rounds = l;
    c->epoch = c->epoch + 3 + (raise_rounds > l ? raise_rounds : l);
    c->ndirty = 0;
    if (__ldcg(&ctl->error) & kErrTimeout) atomicOr(&c->error, kErrTimeout);
  }
}

// ------------------------------------------------------------------------------------------
// Full Euclidean variant (Sec. V-A: the parent holds the full offset to the site instead of a
// neighbour direction), one map per launch. Reading R13:
//  * a site s (a fixed voxel) offers voxel n the distance |d_s| + v ||n - s||, each float32
//    operation rounded once: fl(|d_s| + fl(v * sqrt(fl(q)))), q the squared offset in voxels;
//  * classification follows the first loop of Algorithm 1, except that a fixed voxel whose
//    value changes at all, or that leaves the band, is raised (voxels measured to it would
//    otherwise keep a distance computed from its old value);
//  * raise: a voxel is a child of a raised site iff it is measured to it; every voxel of the
//    map is checked once (a lookup of its site's raised flag), children are reset to +-d_max
//    without a site, and their observed neighbours join the lower wave;
//  * lower: the tile work queue of the quasi-Euclidean wave, where a voxel offers its site
//    (itself if fixed) to its observed, non-fixed, same-sign neighbours.
// Nearest-site propagation through neighbours depends on the processing order, so the result
// is one of several correct ones: every voxel's distance is exactly the offer of its stored
// site, which is a fixed voxel of its sign, and no neighbour's site offers it less.

__device__ __forceinline__ float site_offer(float v, float ds, int ox, int oy, int oz) {
  const int q = ox * ox + oy * oy + oz * oz;
  return __fadd_rn(ds, __fmul_rn(v, __fsqrt_rn((float)q)));
}

// Voxel id of global voxel coordinates (kInvalid if the block is not allocated).
__device__ __forceinline__ uint32_t voxel_at(const DevMap& m, int x, int y, int z) {
  const uint32_t slot = block_lookup(m, x >> m.blog, y >> m.blog, z >> m.blog);
  if (slot == kInvalid || slot >= m.cap_blocks) return kInvalid;
  const int B = m.B;
  return (slot << m.b3log) | (uint32_t)((((z & (B - 1)) << m.blog | (y & (B - 1))) << m.blog) | (x & (B - 1)));
}

__device__ __forceinline__ int3 voxel_coords(const DevMap& m, uint32_t vid) {
  const int3 bc = m.bcoord[vid >> m.b3log];
  const uint32_t l = vid & ((1u << m.b3log) - 1u);
  const int B = m.B;
  return make_int3(bc.x * B + (int)(l & (B - 1)), bc.y * B + (int)((l >> m.blog) & (B - 1)), bc.z * B + (int)(l >> (2 * m.blog)));
}

// Puts the observed 26-neighbours of vid on the lower frontier (they offer their sites to it).
__device__ void mark_observed_neighbours(const DevMap& m, uint32_t vid, EsdfCtl* ctl, unsigned e0) {
  uint32_t last = kInvalid;
  for (int k = 0; k < 27; ++k) {
    if (k == 13) continue;
    const uint32_t n = neighbor_vid(m, vid, k);
    if (n == kInvalid) continue;
    if (ew_flags(__ldcg(&m.esdf[n])) & kObserved) {
      set_bit(m.lbits0, n);
      const uint32_t nb = tile_item_of(m, n);
      if (nb != last) activate(ctl->lact0, &ctl->lcnt[0], m.bstamp_l, nb, e0, 0u);
      last = nb;
    }
  }
}

// Shared memory of a Euclidean lower tile: the tile of the quasi-Euclidean wave, then per active
// voxel of the current local iteration its site's |d| and offset.
__host__ __device__ inline size_t euclid_tile_bytes(int S) { return tile_bytes(S) + align16((size_t)S * S * S * 8); }

// A8 with R13 for one staged tile (all threads of the CTA); the work-queue schedule only.
template <int NT, int B, int S>
__device__ void lower_tile_euclid(const DevMap& m, uint32_t item, const RoundArgs& ra, EsdfCtl* ctl, unsigned char* smem) {
  using G = Geo<B, S>;
  const Tile t = carve(smem, S);
  float* sds = reinterpret_cast<float*>(smem + tile_bytes(S));  // site |d| per active voxel (< 0: none)
  int* soff = reinterpret_cast<int*>(sds + G::S3);              // packed site offset per active voxel
  const TileRef r = tile_ref<B, S>(item);
  stage_tile<NT, B, S>(m, r, m.lbits0, t, true);
  const int3 bc = m.bcoord[r.slot];
  const int gx = bc.x * B + r.ox, gy = bc.y * B + r.oy, gz = bc.z * B + r.oz;  // global origin of the tile
  const float v = m.v;
  unsigned long long pops = 0;
  for (int it = 0;; ++it) {
    const unsigned na = t.cnt[it % 3];
    if (na == 0) break;
    if (it > kMaxLocalIters) {
      if (threadIdx.x == 0) atomicOr(&ctl->error, kErrTimeout);
      break;
    }
    const uint16_t* cur = (it & 1) ? t.b : t.a;
    uint16_t* nxt = (it & 1) ? t.a : t.b;
    unsigned* ncnt = &t.cnt[(it + 1) % 3];
    uint32_t* inb = t.in + (it & 1) * (G::S3 / 32 > 0 ? G::S3 / 32 : 1);
    pops += na;
    if (threadIdx.x == 0) t.cnt[(it + 2) % 3] = 0u;
    for (int j = threadIdx.x; j < (G::S3 + 31) / 32; j += NT) t.in[((it + 1) & 1) * (G::S3 / 32 > 0 ? G::S3 / 32 : 1) + j] = 0u;
    // the site each active voxel offers: itself if fixed, else its stored site (a fixed voxel,
    // whose value does not change during the wave)
    for (unsigned i = threadIdx.x; i < na; i += NT) {
      const int c = cur[i];
      const unsigned long long w = t.w[c];
      const unsigned fl = ew_flags(w);
      float ds = -1.0f;
      int3 o = make_int3(0, 0, 0);
      if (fl & kFixed) {
        ds = fabsf(ew_d(w));
      } else if ((fl & (kObserved | kHasSite)) == (kObserved | kHasSite)) {
        o = ew_site(w);
        int x, y, z;
        G::xyz(c, &x, &y, &z);
        const uint32_t sv = voxel_at(m, gx + x + o.x, gy + y + o.y, gz + z + o.z);
        if (sv != kInvalid) {
          const unsigned long long sw = __ldcg(&m.esdf[sv]);
          if (ew_flags(sw) & kFixed) ds = fabsf(ew_d(sw));
        }
      }
      sds[i] = ds;
      soff[i] = (o.x & 0xff) | ((o.y & 0xff) << 8) | ((o.z & 0xff) << 16);
    }
    __syncthreads();
    for (unsigned p = threadIdx.x; p < na * 26u; p += NT) {
      const unsigned i = p / 26u;
      const float ds = sds[i];
      if (!(ds >= 0.0f)) continue;
      const int kk = (int)(p - i * 26u);
      const int k = kk < 13 ? kk : kk + 1;
      const int c = cur[i];
      const unsigned long long w = t.w[c];
      const bool neg = ew_d(w) < 0.0f;
      const int nc = c + t.doff[k];
      const unsigned long long nw = t.w[nc];
      const unsigned nfl = ew_flags(nw);
      if ((nfl & (kObserved | kFixed)) != kObserved) continue;
      const float dn = ew_d(nw);
      if ((dn < 0.0f) != neg) continue;
      const int so = soff[i];
      // offset from the neighbour to the site: the voxel's offset minus the step to the neighbour
      const int ox = (int)(signed char)(so & 0xff) - (k / 9 - 1);
      const int oy = (int)(signed char)((so >> 8) & 0xff) - ((k / 3) % 3 - 1);
      const int oz = (int)(signed char)((so >> 16) & 0xff) - (k % 3 - 1);
      const float cand = site_offer(v, ds, ox, oy, oz);
      if (!(cand < fabsf(dn))) continue;
      const unsigned long long old = atomicMin(&t.w[nc], ew_pack_site(neg ? -cand : cand, nfl | kHasSite, ox, oy, oz));
      if (!(fabsf(ew_d(old)) > cand)) continue;
      atomicOr(&t.chg[nc >> 5], 1u << (nc & 31));
      if (cell_interior<B, S>(nc)) {
        const int nl = interior_local<B, S>(nc);
        const uint32_t bit = 1u << (nl & 31);
        if (!(atomicOr(&inb[nl >> 5], bit) & bit)) smem_append(nxt, ncnt, (uint16_t)nc);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // drained during the write-back's fences
    if (pops) atomicAdd(&m.ctr->lower_pops, pops);
    atomicAdd(&m.ctr->esdf_block_visits, 1u);
  }
  unsigned ahead = 0;  // the CTA's next ticket
  if (threadIdx.x == kAheadThread) ahead = atomicAdd(&ra.q->ctl->qhead, 1u);
  // write back (global atomicMin), then frontier bits of lowered halo voxels, then the pushes
  for (int c = threadIdx.x; c < G::T3; c += NT) {
    if (!(t.chg[c >> 5] & (1u << (c & 31)))) continue;
    atomicMin(&m.esdf[cell_vid<B, S>(t, r, c)], t.w[c]);
  }
  __threadfence();
  __syncthreads();
  for (int c = threadIdx.x; c < G::T3; c += NT) {
    if (!(t.chg[c >> 5] & (1u << (c & 31))) || cell_interior<B, S>(c)) continue;
    set_bit(m.lbits0, cell_vid<B, S>(t, r, c));
    atomicOr(&t.cnt[3], 1u << cell_tile_dir<B, S>(c));
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x < 27 && (t.cnt[3] >> threadIdx.x & 1u)) {
    const uint32_t nit = neighbor_tile_item<B, S>(t, r, threadIdx.x);
    if (nit != kInvalid) q_push(*ra.q, 0u, nit, m.bstamp_l, ra.e0);
  }
  if (threadIdx.x == kAheadThread) q_ahead_resolve(*ra.q, ahead, ra.ahead);
  __syncthreads();
}

template <int NT>
__global__ void __launch_bounds__(NT, 1) k_esdf_euclid(const DevMap* __restrict__ maps, EsdfCtl* ctl) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ QueueAhead sh_ahead;
  __shared__ int sh_state;
  __shared__ uint2 sh_e;
  __shared__ unsigned long long sh_t[4];
  const DevMap& m = maps[0];
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nthreads = gridDim.x * blockDim.x;
  if (threadIdx.x == 0) sh_t[0] = global_ns();
  if (tid == 0) atomicAdd(&ctl->calls, 1u);
  if (ctl->rcap < ctl->cap + 27u * gridDim.x) {
    if (tid == 0) atomicOr(&ctl->error, kErrTimeout);
    return;
  }
  const unsigned ndirty = __ldcg(&m.ctr->ndirty);
  const unsigned e0 = __ldcg(&m.ctr->epoch) + 1;
  const float dmax = m.dmax;
  // ---- classification (first loop of Algorithm 1, R6 and R13)
  for (unsigned i = tid; i < ndirty; i += nthreads) {
    const uint32_t vid = m.dirty[i];
    m.vflags[vid] = (uint8_t)(m.vflags[vid] & ~kQueuedForEsdf);
    const float2 tv = m.tsdf[vid];
    if (!(tv.y > 0.0f)) continue;
    const float Df = tv.x == 0.0f ? 0.0f : tv.x;  // sign(0) = +1
    const bool occ = m.esdf_mode == 1;
    const bool neg = !occ && Df < 0.0f;
    const bool fixed_now = occ ? Df < 0.0f : fabsf(Df) < m.gamma;
    const float seedv = occ ? 0.0f : Df;
    const float sdmax = neg ? -dmax : dmax;
    const unsigned long long w = __ldcg(&m.esdf[vid]);
    const unsigned fl = ew_flags(w);
    const bool obs = (fl & kObserved) != 0;
    const float de = ew_d(w);
    if (fixed_now) {
      count_one(&m.ctr->seeds);
      if (obs && (fl & kFixed) && __float_as_uint(de) != __float_as_uint(seedv)) {
        m.vflags[vid] = (uint8_t)(m.vflags[vid] | kSiteRaised);
        atomicAdd(&ctl->rcnt[0], 1u);
      }
      m.esdf[vid] = ew_pack_site(seedv, kObserved | kFixed, 0, 0, 0);
      set_bit(m.lbits0, vid);
      activate(ctl->lact0, &ctl->lcnt[0], m.bstamp_l, tile_item_of(m, vid), e0, 0u);
    } else if (fl & kFixed) {  // leaves the band: raised, and its neighbours offer their sites
      m.vflags[vid] = (uint8_t)(m.vflags[vid] | kSiteRaised);
      atomicAdd(&ctl->rcnt[0], 1u);
      m.esdf[vid] = ew_pack_site(sdmax, kObserved, 0, 0, 0);
      mark_observed_neighbours(m, vid, ctl, e0);
    } else if (!obs || (de < 0.0f) != neg) {  // new voxel, or sign flip (nothing is measured to it)
      m.esdf[vid] = ew_pack_site(sdmax, kObserved, 0, 0, 0);
      mark_observed_neighbours(m, vid, ctl, e0);
    }
  }
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->error)) return;
  if (threadIdx.x == 0) sh_t[1] = global_ns();
  // ---- raise (R13): every voxel measured to a raised site is reset
  const bool any_raised = __ldcg(&ctl->rcnt[0]) > 0u;
  if (any_raised) {
    const uint32_t V = min(__ldcg(&m.ctr->blocks), m.cap_blocks) << m.b3log;
    unsigned long long nraised = 0;
    for (uint32_t vid = tid; vid < V; vid += nthreads) {
      const unsigned long long w = __ldcg(&m.esdf[vid]);
      const unsigned fl = ew_flags(w);
      if ((fl & (kObserved | kFixed | kHasSite)) != (kObserved | kHasSite)) continue;
      const int3 c = voxel_coords(m, vid);
      const int3 o = ew_site(w);
      const uint32_t sv = voxel_at(m, c.x + o.x, c.y + o.y, c.z + o.z);
      if (sv != kInvalid && !(__ldcg(&m.vflags[sv]) & kSiteRaised) && (ew_flags(__ldcg(&m.esdf[sv])) & kFixed)) continue;
      m.esdf[vid] = ew_pack_site(ew_d(w) < 0.0f ? -dmax : dmax, kObserved, 0, 0, 0);
      ++nraised;
      mark_observed_neighbours(m, vid, ctl, e0);
    }
    if (nraised) atomicAdd(&m.ctr->raise_pops, nraised);
    if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->error)) return;
    for (unsigned i = tid; i < ndirty; i += nthreads) {
      const uint32_t vid = m.dirty[i];
      m.vflags[vid] = (uint8_t)(m.vflags[vid] & ~kSiteRaised);
    }
  }
  if (!grid_barrier(&ctl->bar, gridDim.x, &ctl->error)) return;
  if (threadIdx.x == 0) sh_t[2] = global_ns();
  // ---- lower: the tile work queue with site offers
  WaveQueue q;
  q.ctl = ctl;
  q.init = ctl->lact0;
  q.n0 = __ldcg(&ctl->lcnt[0]);
  q.tag_epoch = 2u * __ldcg(&ctl->calls) + 1u;
  if (threadIdx.x == 0) sh_ahead.st = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      uint2 e = make_uint2(0u, 0u);
      const int st = q_next(q, &sh_ahead, &e);
      if (st == 1) {
        atomicExch(&m.bstamp_l[e.y], __ldcg(&m.ctr->epoch));  // e0 - 1: no longer queued
        __threadfence();  // and the CTA barrier below orders this before the tile's bit reads
      }
      sh_state = st;
      sh_e = e;
    }
    __syncthreads();
    const int st = sh_state;
    const uint2 e = sh_e;
    if (st != 1) break;
    RoundArgs ra;
    ra.mi = 0;
    ra.e0 = e0;
    ra.ep_next = e0;
    ra.nxt_bits = m.lbits0;
    ra.nxt_list = nullptr;
    ra.nxt_cnt = nullptr;
    ra.q = &q;
    ra.ahead = &sh_ahead;
    switch (m.B) {
      case 4: lower_tile_euclid<NT, 4, 4>(m, e.y, ra, ctl, dsm); break;
      case 8: lower_tile_euclid<NT, 8, 8>(m, e.y, ra, ctl, dsm); break;
      default: lower_tile_euclid<NT, 16, kTileEdge>(m, e.y, ra, ctl, dsm); break;
    }
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&ctl->qdone, 1u);
    }
  }
  if (threadIdx.x == 0) sh_t[3] = global_ns();
  __syncthreads();
  if (tid == 0) {
    Counters* c = m.ctr;
    c->esdf_phase_ns[0] = (unsigned)(sh_t[1] - sh_t[0]);
    c->esdf_phase_ns[1] = (unsigned)(sh_t[2] - sh_t[1]);
    c->esdf_phase_ns[2] = (unsigned)(sh_t[3] - sh_t[2]);
    c->esdf_in = ndirty;
    c->raise_rounds = any_raised ? 1u : 0u;
    c->lower_rounds = q.n0 > 0 ? 1u : 0u;
    c->epoch = c->epoch + 4;
    c->ndirty = 0;
    if (__ldcg(&ctl->error) & kErrTimeout) atomicOr(&c->error, kErrTimeout);
  }
}

}  // namespace

size_t esdf_smem_bytes(int max_B) { return tile_bytes(max_B < kTileEdge ? max_B : kTileEdge); }

namespace {

template <int NT, int MINB>
const void* esdf_single_kernel(int be) {
  switch (be) {
    case 4: return (const void*)k_esdf<NT, MINB, 4>;
    case 8: return (const void*)k_esdf<NT, MINB, 8>;
    case 16: return (const void*)k_esdf<NT, MINB, 16>;
    default: return nullptr;
  }
}

// be: the block edge of a single map whose waves run as work queues (0 for a batch)
const void* esdf_kernel(int threads, int ctas_per_sm, int be) {
  // (the 512 x 2 shape of small single-map updates keeps the general kernel: compiled for one
  // block edge it ran the room frames' ESDF 2.5 % slower)
  if (be != 0 && threads == 256 && ctas_per_sm == 8) return esdf_single_kernel<256, 8>(be);
  switch (threads) {
    case 128: return (const void*)k_esdf<128, 12, 0>;
    case 256: return ctas_per_sm > 0 && ctas_per_sm <= 4 ? (const void*)k_esdf<256, 4, 0> : (const void*)k_esdf<256, 6, 0>;
    case 512: return (const void*)k_esdf<512, 2, 0>;
    case 1024: return (const void*)k_esdf<1024, 1, 0>;
    default: return nullptr;
  }
}

}  // namespace

int esdf_grid(int num_sms, int max_B, int ctas_per_sm, int threads, int be) {
  const void* k = esdf_kernel(threads, ctas_per_sm, be);
  if (!k) return 0;
  const size_t smem = esdf_smem_bytes(max_B);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, threads, smem) != cudaSuccess) return 0;
  if (ctas_per_sm > 0 && nb > ctas_per_sm) nb = ctas_per_sm;
  return nb * num_sms;
}

cudaError_t launch_esdf(const DevMap* maps_dev, int nmaps, int max_B, EsdfCtl* ctl, const LaunchCfg& cfg,
                        LaunchHook* hook, bool allow_async) {
  if (nmaps <= 0 || nmaps > kMaxBatch) return cudaErrorInvalidValue;
  const int threads = cfg.tune.esdf_threads;
  // one map whose waves run as work queues gets the kernel compiled for its block edge
  const int be = nmaps == 1 && allow_async ? max_B : 0;
  const void* k = esdf_kernel(threads, cfg.tune.esdf_ctas_per_sm, be);
  if (!k) return cudaErrorInvalidValue;
  const int grid = esdf_grid(cfg.num_sms, max_B, cfg.tune.esdf_ctas_per_sm, threads, be);
  if (grid <= 0) return cudaErrorCooperativeLaunchTooLarge;
  const size_t smem = esdf_smem_bytes(max_B);
  int async = allow_async ? 1 : 0;
  void* args[] = {(void*)&maps_dev, (void*)&nmaps, (void*)&ctl, (void*)&async};
  hook->begin(kKEsdf, cfg.stream);
  cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(grid), dim3(threads), args, smem, cfg.stream);
  hook->end(kKEsdf, cfg.stream);
  return e;
}

// Euclidean variant of one map (R13): cooperative launch of 512-thread CTAs.
cudaError_t launch_esdf_euclid(const DevMap* map_dev, int B, EsdfCtl* ctl, const LaunchCfg& cfg, LaunchHook* hook) {
  const void* k = (const void*)k_esdf_euclid<512>;
  const size_t smem = euclid_tile_bytes(B < kTileEdge ? B : kTileEdge);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return cudaErrorInvalidValue;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 512, smem) != cudaSuccess || nb < 1) return cudaErrorCooperativeLaunchTooLarge;
  nb = nb > 2 ? 2 : nb;
  void* args[] = {(void*)&map_dev, (void*)&ctl};
  hook->begin(kKEsdf, cfg.stream);
  cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(nb * cfg.num_sms), dim3(512), args, smem, cfg.stream);
  hook->end(kKEsdf, cfg.stream);
  return e;
}

}  // namespace vbx
