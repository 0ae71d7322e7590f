// api.cu -- the C ABI declared in include/vbx.h: map lifetime, argument validation, device
// memory, per-scan scratch, launch bookkeeping (counting and optional event timing), sticky
// device errors, and host-side export/import of map contents.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/vbx.h"
#include "launch.h"
#include "vbx_internal.cuh"

namespace vbx {
const char* const kKernelNames[kNumKernels] = {"reset_counters", "bin_points",  "group_rays",  "link_blocks",
                                               "integrate_rays", "apply",       "esdf",        "query",
                                               "import_alloc",   "import_set",  "init_groups", "mesh_select",
                                               "mesh_blocks",    "mesh_clear",  "scratch_links"};
}  // namespace vbx

namespace {

thread_local std::string g_last_error;

// Slots of the lower wave's queue ring: every tile once plus 27 pushes in flight per CTA, for the
// largest grid (32 resident CTAs per SM).
uint64_t lower_ring_slots(uint64_t tiles, int num_sms) { return tiles + 27ull * 32ull * (uint64_t)(num_sms > 0 ? num_sms : 1); }
std::atomic<long long> g_total_launches{0};

vbx_status fail(vbx_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

vbx_status cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(VBX_ERR_OUT_OF_MEMORY, "%s: %s", where, cudaGetErrorString(e));
  return fail(VBX_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

struct PendingTiming {
  int kernel;
  cudaEvent_t start, stop;
};

struct MapHook : vbx::LaunchHook {
  long long launches = 0;
  bool profile = false;
  std::vector<PendingTiming> pending;
  std::vector<cudaEvent_t> free_events;
  cudaEvent_t cur_start = nullptr;
  double ms[vbx::kNumKernels] = {0};
  long long count[vbx::kNumKernels] = {0};

  cudaEvent_t get_event() {
    if (!free_events.empty()) {
      cudaEvent_t e = free_events.back();
      free_events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void begin(int, cudaStream_t s) override {
    ++launches;
    g_total_launches.fetch_add(1);
    if (profile) {
      cur_start = get_event();
      cudaEventRecord(cur_start, s);
    }
  }
  void end(int kernel, cudaStream_t s) override {
    if (profile && cur_start) {
      cudaEvent_t stop = get_event();
      cudaEventRecord(stop, s);
      pending.push_back(PendingTiming{kernel, cur_start, stop});
      cur_start = nullptr;
    }
  }
  void collect() {
    for (auto& p : pending) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, p.start, p.stop) == cudaSuccess) {
        ms[p.kernel] += t;
        count[p.kernel] += 1;
      }
      free_events.push_back(p.start);
      free_events.push_back(p.stop);
    }
    pending.clear();
  }
  ~MapHook() override {
    for (auto& p : pending) {
      cudaEventDestroy(p.start);
      cudaEventDestroy(p.stop);
    }
    for (auto e : free_events) cudaEventDestroy(e);
  }
};

uint32_t next_pow2(uint64_t x) {
  uint64_t p = 1;
  while (p < x) p <<= 1;
  return (uint32_t)p;
}

int ilog2(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

}  // namespace

struct vbx_map_s {
  vbx::DevMap d{};
  int device = 0;
  int num_sms = 0;
  vbx_map_options opt{};
  float voxel_size = 0, truncation = 0, max_esdf_dist = 0;
  int B = 0;
  vbx::DevMap* d_dev = nullptr;   // device copy of d (kernels that take map arrays read it)
  vbx::EsdfCtl* ctl_dev = nullptr;  // ESDF control block of this map's own updates
  int64_t pts_cap = 0;
  int64_t last_points_in = 0;
  uint32_t gtab_entries = 0;
  uint64_t version = 0;  // bumped whenever d (and so d_dev) changes
  uint32_t scan_epoch = 0;  // epoch of the last integrated scan (claims of scratch blocks)
  std::vector<void*> allocs;
  MapHook hook;

  vbx::LaunchCfg cfg(void* stream) const { return vbx::LaunchCfg{num_sms, (cudaStream_t)stream, vbx::kMapTuning}; }
  // dirty voxels of the last ESDF update, copied back asynchronously after each update (pinned;
  // read without waiting, so it may lag by an update): picks the next update's launch shape
  unsigned* h_last_esdf_in = nullptr;

  std::vector<size_t> alloc_bytes;

  template <typename T>
  cudaError_t alloc(T** p, size_t count, int fill_byte) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16));
    if (e != cudaSuccess) return e;
    allocs.push_back(q);
    alloc_bytes.push_back(std::max<size_t>(count * sizeof(T), 16));
    e = cudaMemset(q, fill_byte, std::max<size_t>(count * sizeof(T), 16));
    *p = (T*)q;
    return e;
  }
  void release(void* p) {
    if (!p) return;
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (it != allocs.end()) {
      alloc_bytes.erase(alloc_bytes.begin() + (it - allocs.begin()));
      allocs.erase(it);
    }
    cudaFree(p);
  }
  ~vbx_map_s() {
    for (void* p : allocs) cudaFree(p);
    if (h_last_esdf_in) cudaFreeHost(h_last_esdf_in);
  }
};

namespace {

vbx_status read_error(vbx_map_t m, cudaStream_t s) {
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
  unsigned err = 0;
  e = cudaMemcpy(&err, &m->d.ctr->error, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read error word");
  if (!err) return VBX_OK;
  unsigned zero = 0;
  cudaMemcpy(&m->d.ctr->error, &zero, sizeof(unsigned), cudaMemcpyHostToDevice);
  if (err & vbx::kErrTimeout) return fail(VBX_ERR_TIMEOUT, "device loop exceeded its round or wait budget");
  if (err & vbx::kErrPoolFull) return fail(VBX_ERR_OUT_OF_MEMORY, "block pool exhausted (block_capacity)");
  if (err & vbx::kErrHashFull) return fail(VBX_ERR_HASH_FULL, "block hash probe limit reached");
  if (err & vbx::kErrGroupTable) return fail(VBX_ERR_HASH_FULL, "per-scan group table full");
  if (err & vbx::kErrScratchFull)
    return fail(VBX_ERR_OUT_OF_MEMORY, "the scan entered more blocks than scratch_blocks; it was not integrated");
  return fail(VBX_ERR_CUDA, "unknown device error 0x%x", err);
}

vbx_status ensure_scratch(vbx_map_t m, int64_t n, cudaStream_t s) {
  if (n <= m->pts_cap && m->d.gtab) return VBX_OK;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "scratch resize sync");
  m->release(m->d.gtab);
  m->release(m->d.glist);
  m->release(m->d.rays);
  m->d.gtab = nullptr;
  m->d.glist = nullptr;
  m->d.rays = nullptr;
  const int64_t cap = std::max<int64_t>(next_pow2((uint64_t)std::max<int64_t>(n, 1024)), m->pts_cap);
  const uint32_t entries = next_pow2((uint64_t)cap * 2);
  if ((e = m->alloc(&m->d.gtab, entries, 0)) != cudaSuccess) return cuda_fail(e, "group table");
  if ((e = m->alloc(&m->d.glist, (size_t)cap, 0)) != cudaSuccess) return cuda_fail(e, "group list");
  if ((e = m->alloc(&m->d.rays, (size_t)cap, 0)) != cudaSuccess) return cuda_fail(e, "ray buffer");
  m->d.gmask = entries - 1;
  m->gtab_entries = entries;
  m->pts_cap = cap;
  e = vbx::launch_init_groups(m->d.gtab, entries, s, &m->hook);
  if (e != cudaSuccess) return cuda_fail(e, "group table init");
  if (m->d_dev) {
    e = cudaMemcpy(m->d_dev, &m->d, sizeof(vbx::DevMap), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "device map descriptor");
  }
  m->version += 1;
  return VBX_OK;
}

// Epoch of the next scan of m. Epochs only grow, so a block's scratch claim from an earlier
// scan never matches; on wrap-around the claim and epoch arrays are cleared first.
cudaError_t next_scan_epoch(vbx_map_t m, cudaStream_t s, unsigned* ep) {
  if (m->scan_epoch == 0xffffffffu) {
    cudaError_t e = cudaMemsetAsync(m->d.hclaim, 0, ((size_t)m->d.hmask + 1) * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->d.sinfo, 0, (size_t)m->d.cap_blocks * 8, s);
    if (e != cudaSuccess) return e;
    m->scan_epoch = 0;
  }
  *ep = ++m->scan_epoch;
  return cudaSuccess;
}

}  // namespace

extern "C" {

vbx_status vbx_default_options(vbx_map_options* opt) {
  if (!opt) return fail(VBX_ERR_INVALID_ARG, "opt is NULL");
  std::memset(opt, 0, sizeof(*opt));
  opt->weighting = 0;
  opt->grouped = 1;
  return VBX_OK;
}

vbx_status vbx_create_map(float voxel_size, int voxels_per_block, float truncation, float max_esdf_dist,
                          const vbx_map_options* opt_in, vbx_map_t* out) {
  if (!out) return fail(VBX_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!(voxel_size > 0.0f) || !std::isfinite(voxel_size))
    return fail(VBX_ERR_INVALID_ARG, "voxel_size must be a positive finite number");
  if (voxels_per_block != 4 && voxels_per_block != 8 && voxels_per_block != 16)
    return fail(VBX_ERR_INVALID_ARG, "voxels_per_block must be 4, 8 or 16");
  if (!(truncation >= voxel_size) || !(truncation <= 64.0f * voxel_size))
    return fail(VBX_ERR_INVALID_ARG, "truncation must lie in [voxel_size, 64 * voxel_size]");
  if (!(max_esdf_dist > 0.0f) || !std::isfinite(max_esdf_dist))
    return fail(VBX_ERR_INVALID_ARG, "max_esdf_dist must be a positive finite number");
  vbx_map_options opt;
  vbx_default_options(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.weighting != 0 && opt.weighting != 1) return fail(VBX_ERR_INVALID_ARG, "weighting must be 0 or 1");
  if (opt.esdf_mode != 0 && opt.esdf_mode != 1) return fail(VBX_ERR_INVALID_ARG, "esdf_mode must be 0 or 1");
  if (opt.euclidean != 0 && opt.euclidean != 1) return fail(VBX_ERR_INVALID_ARG, "euclidean must be 0 or 1");
  if (opt.euclidean && !(max_esdf_dist <= 126.0f * voxel_size))
    return fail(VBX_ERR_INVALID_ARG, "euclidean maps need max_esdf_dist <= 126 * voxel_size (site offsets are 8-bit)");
  const float eps = opt.eps > 0.0f ? opt.eps : voxel_size;
  if (opt.weighting == 1 && !(eps < truncation)) return fail(VBX_ERR_INVALID_ARG, "eps must be below truncation");
  const int B = voxels_per_block;
  const int64_t B3 = (int64_t)B * B * B;
  int64_t cap = opt.block_capacity > 0 ? opt.block_capacity : (int64_t(1) << 25) / B3;
  if (cap * B3 >= (int64_t(1) << 32) - 1) return fail(VBX_ERR_INVALID_ARG, "block_capacity * B^3 must stay below 2^32");

  vbx_map_s* m = new vbx_map_s();
  cudaError_t e = cudaGetDevice(&m->device);
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "cudaGetDevice");
  }
  int coop = 0;
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, m->device);
  if (!coop) {
    delete m;
    return fail(VBX_ERR_CUDA, "device does not support cooperative launches");
  }
  m->opt = opt;
  m->voxel_size = voxel_size;
  m->truncation = truncation;
  m->max_esdf_dist = max_esdf_dist;
  m->B = B;
  vbx::DevMap& d = m->d;
  d.v = voxel_size;
  d.delta = truncation;
  d.eps = eps;
  d.gamma = opt.fixed_band > 0.0f ? opt.fixed_band : voxel_size;
  d.wmax = opt.w_max > 0.0f ? opt.w_max : 1e4f;
  d.dmax = max_esdf_dist;
  d.max_range2 = (opt.max_range > 0.0f && std::isfinite(opt.max_range)) ? opt.max_range * opt.max_range : 0.0f;
  const float lim = 16384.0f * voxel_size;
  d.range_lim2 = lim * lim;
  d.L1 = voxel_size;
  d.L2 = voxel_size * 1.41421356237309515f;
  d.L3 = voxel_size * 1.73205080756887719f;
  d.B = B;
  d.blog = ilog2(B);
  d.b3log = 3 * d.blog;
#ifndef VBX_TILE_EDGE
#define VBX_TILE_EDGE 8
#endif
  d.tile_shift = (B == 16 && VBX_TILE_EDGE == 8) ? 3 : 0;  // ESDF tiles of 8^3 voxels
  d.weighting = opt.weighting;
  d.esdf_mode = opt.esdf_mode;
  d.euclid = opt.euclidean;
  d.grouped = opt.grouped ? 1 : 0;
  d.cap_blocks = (uint32_t)cap;
  const uint32_t H = next_pow2((uint64_t)cap * 2);
  d.hmask = H - 1;
  const size_t V = (size_t)cap * B3;
#define VBX_ALLOC(ptr, count, fill)                           \
  do {                                                        \
    if ((e = m->alloc(&(ptr), (count), (fill))) != cudaSuccess) { \
      delete m;                                               \
      return cuda_fail(e, "allocate " #ptr);                  \
    }                                                         \
  } while (0)
  const int64_t scr = opt.scratch_blocks > 0 ? std::min<int64_t>(opt.scratch_blocks, cap) : cap;
  d.scr_cap = (uint32_t)scr;
  const size_t SV = (size_t)scr * B3;  // scratch voxels
  VBX_ALLOC(d.hkeys, H, 0xff);
  VBX_ALLOC(d.hvals, H, 0xff);
  VBX_ALLOC(d.hclaim, H, 0);
  VBX_ALLOC(d.bcoord, (size_t)cap, 0);
  VBX_ALLOC(d.nbr, (size_t)cap * 27, 0xff);
  VBX_ALLOC(d.sinfo, (size_t)cap, 0);
  VBX_ALLOC(d.tsdf, V, 0);
  VBX_ALLOC(d.slist_h, (size_t)scr, 0);
  VBX_ALLOC(d.slist, (size_t)scr, 0);
  VBX_ALLOC(d.snbr, (size_t)scr * 27, 0xff);
  VBX_ALLOC(d.sacc, 4 * SV, 0);
  VBX_ALLOC(d.stouch, SV, 0);
  VBX_ALLOC(d.esdf, V, 0);
  VBX_ALLOC(d.vflags, V, 0);
  VBX_ALLOC(d.rbits0, V / 32, 0);
  VBX_ALLOC(d.rbits1, V / 32, 0);
  VBX_ALLOC(d.lbits0, V / 32, 0);
  VBX_ALLOC(d.lbits1, V / 32, 0);
  VBX_ALLOC(d.pbits, V / 32, 0);
  const size_t items = (size_t)cap << d.tile_shift;  // ESDF tiles
  VBX_ALLOC(d.bstamp_r, items, 0);
  VBX_ALLOC(d.bstamp_l, items, 0);
  VBX_ALLOC(d.updated, V, 0);
  VBX_ALLOC(d.dirty, V, 0);
  VBX_ALLOC(d.newblk, (size_t)cap, 0);
  VBX_ALLOC(d.mdirty, (size_t)cap, 0);
  VBX_ALLOC(d.mlist, (size_t)cap, 0);
  VBX_ALLOC(d.ctr, 1, 0);
  VBX_ALLOC(m->d_dev, 1, 0);
  VBX_ALLOC(m->ctl_dev, 1, 0);
  {
    vbx::EsdfCtl ctl{};
    ctl.cap = (unsigned)items;
    VBX_ALLOC(ctl.ract0, items, 0);
    VBX_ALLOC(ctl.ract1, items, 0);
    VBX_ALLOC(ctl.lact0, items, 0);
    VBX_ALLOC(ctl.lact1, items, 0);
    const uint64_t ring = lower_ring_slots(items, m->num_sms);
    ctl.rcap = (unsigned)ring;
    VBX_ALLOC(ctl.lring, ring, 0);
    VBX_ALLOC(ctl.ltag, ring, 0);
    if ((e = cudaMemcpy(m->ctl_dev, &ctl, sizeof(ctl), cudaMemcpyHostToDevice)) != cudaSuccess) {
      delete m;
      return cuda_fail(e, "esdf control block");
    }
  }
#undef VBX_ALLOC
  vbx_status st = ensure_scratch(m, opt.max_points > 0 ? opt.max_points : (int64_t(1) << 20), 0);
  if (st != VBX_OK) {
    delete m;
    return st;
  }
  if ((e = cudaMallocHost((void**)&m->h_last_esdf_in, sizeof(unsigned))) != cudaSuccess) {
    m->h_last_esdf_in = nullptr;
    delete m;
    return cuda_fail(e, "pinned update counter");
  }
  *m->h_last_esdf_in = 0u;
  if ((e = cudaMemcpy(m->d_dev, &m->d, sizeof(vbx::DevMap), cudaMemcpyHostToDevice)) != cudaSuccess) {
    delete m;
    return cuda_fail(e, "device map descriptor");
  }
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete m;
    return cuda_fail(e, "create sync");
  }
  *out = m;
  return VBX_OK;
}

vbx_status vbx_destroy_map(vbx_map_t map) {
  if (!map) return VBX_OK;
  cudaDeviceSynchronize();
  delete map;
  return VBX_OK;
}

vbx_status vbx_integrate_scan(vbx_map_t m, const float* points_dev, int64_t n, const float T[16], void* stream) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  if (n < 0 || n > (int64_t(1) << 28)) return fail(VBX_ERR_INVALID_ARG, "n must lie in [0, 2^28]");
  if (n > 0 && !points_dev) return fail(VBX_ERR_INVALID_ARG, "points_dev is NULL");
  if (!T) return fail(VBX_ERR_INVALID_ARG, "T_world_sensor is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(m->d.ctr, 0, offsetof(vbx::Counters, blocks), s);
  if (e != cudaSuccess) return cuda_fail(e, "reset scan counters");
  m->last_points_in = n;
  if (n == 0) return VBX_OK;
  vbx_status st = ensure_scratch(m, n, s);
  if (st != VBX_OK) return st;
  vbx::Pose pose;
  std::memcpy(pose.T, T, sizeof(pose.T));
  unsigned ep = 0;
  if ((e = next_scan_epoch(m, s, &ep)) != cudaSuccess) return cuda_fail(e, "scan epoch");
  e = vbx::launch_integrate(vbx::single_batch(m->d, points_dev, (int)n, pose, ep), m->cfg(stream), &m->hook);
  if (e != cudaSuccess) return cuda_fail(e, "integrate launch");
  return VBX_OK;
}

vbx_status vbx_integrate_scan_noalloc(vbx_map_t m, const float* points_dev, int64_t n, const float T[16],
                                      void* stream) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  if (n < 0 || n > vbx::kNoAllocMaxPoints)
    return fail(VBX_ERR_INVALID_ARG, "n = %lld outside [0, %d], the scratch limit of vbx_integrate_scan_noalloc",
                (long long)n, vbx::kNoAllocMaxPoints);
  if (n > 0 && !points_dev) return fail(VBX_ERR_INVALID_ARG, "points_dev is NULL");
  if (!T) return fail(VBX_ERR_INVALID_ARG, "T_world_sensor is NULL");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (device != m->device) return fail(VBX_ERR_INVALID_ARG, "the current device is not the map's device");
  void* scratch = nullptr;
  e = vbx::noalloc_scratch_setup(device, &scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaMemsetAsync(m->d.ctr, 0, offsetof(vbx::Counters, blocks), s);
  if (e != cudaSuccess) return cuda_fail(e, "reset scan counters");
  m->last_points_in = n;
  if (n == 0) return VBX_OK;
  vbx::Pose pose;
  std::memcpy(pose.T, T, sizeof(pose.T));
  unsigned ep = 0;
  if ((e = next_scan_epoch(m, s, &ep)) != cudaSuccess) return cuda_fail(e, "scan epoch");
  e = vbx::launch_integrate_noalloc(m->d, scratch, points_dev, (int)n, pose, ep, m->cfg(stream), &m->hook);
  if (e != cudaSuccess) return cuda_fail(e, "integrate launch");
  return VBX_OK;
}

vbx_status vbx_update_esdf(vbx_map_t m, void* stream) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t off = offsetof(vbx::Counters, raise_rounds);
  cudaError_t e = cudaMemsetAsync((char*)m->d.ctr + off, 0, sizeof(vbx::Counters) - off, s);
  if (e != cudaSuccess) return cuda_fail(e, "reset esdf counters");
  e = cudaMemsetAsync(m->ctl_dev, 0, offsetof(vbx::EsdfCtl, cap), s);
  if (e != cudaSuccess) return cuda_fail(e, "reset esdf control");
  if (m->opt.euclidean) {
    e = vbx::launch_esdf_euclid(m->d_dev, m->B, m->ctl_dev, m->cfg(stream), &m->hook);
  } else {  // one map: its rounds would hold about one tile per SM, so the waves run as work queues
    vbx::LaunchCfg cfg = m->cfg(stream);
    if (*(volatile unsigned*)m->h_last_esdf_in >= vbx::kMapLargeUpdate) cfg.tune = vbx::kMapTuningLarge;
    e = vbx::launch_esdf(m->d_dev, 1, m->B, m->ctl_dev, cfg, &m->hook, true);
  }
  if (e != cudaSuccess) return cuda_fail(e, "esdf cooperative launch");
  e = cudaMemcpyAsync(m->h_last_esdf_in, &m->d.ctr->esdf_in, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "esdf update count");
  return VBX_OK;
}

vbx_status vbx_query_distance_gradient(vbx_map_t m, const float* q_dev, int64_t n, float* dist_dev, float* grad_dev,
                                       uint8_t* status_dev, void* stream) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  if (n < 0 || n > (int64_t(1) << 30)) return fail(VBX_ERR_INVALID_ARG, "n must lie in [0, 2^30]");
  if (n > 0 && (!q_dev || !dist_dev || !grad_dev || !status_dev))
    return fail(VBX_ERR_INVALID_ARG, "query buffers must not be NULL");
  vbx::Batch b = vbx::single_batch(m->d, nullptr, 0, vbx::Pose{});
  b.one_query.q = q_dev;
  b.one_query.dist = dist_dev;
  b.one_query.grad = grad_dev;
  b.one_query.status = status_dev;
  b.one_query.n = (unsigned)n;
  cudaError_t e = vbx::launch_query(b, (unsigned)n, m->cfg(stream), &m->hook);
  if (e != cudaSuccess) return cuda_fail(e, "query launch");
  return VBX_OK;
}

vbx_status vbx_sync(vbx_map_t m, void* stream) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  return read_error(m, (cudaStream_t)stream);
}

vbx_status vbx_get_stats(vbx_map_t m, vbx_stats* out, void* stream) {
  if (!m || !out) return fail(VBX_ERR_INVALID_ARG, "map or out is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "stats sync");
  vbx::Counters c;
  e = cudaMemcpy(&c, m->d.ctr, sizeof(c), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "stats copy");
  std::memset(out, 0, sizeof(*out));
  out->points_in = m->last_points_in;
  out->points_valid = c.npoints_valid;
  out->rays = c.ngroups;
  out->records = (int64_t)c.nrecords;
  out->updated = c.nupdated;
  out->new_blocks = c.nnew;
  out->blocks = std::min<int64_t>(c.blocks, m->d.cap_blocks);
  out->esdf_in = c.esdf_in;
  out->seeds = c.seeds;
  out->raise_pops = (int64_t)c.raise_pops;
  out->lower_pops = (int64_t)c.lower_pops;
  out->raise_rounds = c.raise_rounds;
  out->lower_rounds = c.lower_rounds;
  out->launches = m->hook.launches;
  out->esdf_block_visits = c.esdf_block_visits;
  out->esdf_local_iters = c.esdf_local_iters;
  out->esdf_classify_ns = c.esdf_phase_ns[0];
  out->esdf_raise_ns = c.esdf_phase_ns[1];
  out->esdf_lower_ns = c.esdf_phase_ns[2];
  out->touched_blocks = c.ntouched;
  return read_error(m, (cudaStream_t)stream);
}

vbx_status vbx_num_blocks(vbx_map_t m, int64_t* n_out, void* stream) {
  if (!m || !n_out) return fail(VBX_ERR_INVALID_ARG, "map or n_out is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  unsigned b = 0;
  e = cudaMemcpy(&b, &m->d.ctr->blocks, sizeof(b), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "copy");
  *n_out = std::min<int64_t>(b, m->d.cap_blocks);
  return VBX_OK;
}

vbx_status vbx_export_blocks(vbx_map_t m, int32_t* keys, float* tsdf, float* esdf_d, uint8_t* parent, uint8_t* flags,
                             int64_t cap, void* stream) {
  int64_t nb = 0;
  vbx_status st = vbx_num_blocks(m, &nb, stream);
  if (st != VBX_OK) return st;
  if (cap < nb) return fail(VBX_ERR_INVALID_ARG, "cap %lld below the number of blocks %lld", (long long)cap, (long long)nb);
  const size_t B3 = (size_t)m->B * m->B * m->B;
  const size_t V = (size_t)nb * B3;
  cudaError_t e;
  if (keys && nb) {
    e = cudaMemcpy(keys, m->d.bcoord, (size_t)nb * sizeof(int3), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy keys");
  }
  if (tsdf && V) {
    e = cudaMemcpy(tsdf, m->d.tsdf, V * sizeof(float2), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy tsdf");
  }
  if ((esdf_d || parent || flags) && V) {
    std::vector<unsigned long long> w(V);
    e = cudaMemcpy(w.data(), m->d.esdf, V * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy esdf");
    for (size_t i = 0; i < V; ++i) {
      const uint32_t db = (uint32_t)(w[i] >> 32);
      float dv;
      std::memcpy(&dv, &db, sizeof(dv));
      if (esdf_d) esdf_d[i] = dv;
      if (parent) parent[i] = (uint8_t)(w[i] & 0xff);
      if (flags) flags[i] = (uint8_t)((w[i] >> 8) & 0xff);
    }
  }
  return read_error(m, (cudaStream_t)stream);
}

vbx_status vbx_export_sites(vbx_map_t m, int8_t* offsets, uint8_t* has_site, int64_t cap, void* stream) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  if (!m->opt.euclidean) return fail(VBX_ERR_INVALID_ARG, "the map is not a Euclidean map");
  int64_t nb = 0;
  vbx_status st = vbx_num_blocks(m, &nb, stream);
  if (st != VBX_OK) return st;
  if (cap < nb) return fail(VBX_ERR_INVALID_ARG, "cap %lld below the number of blocks %lld", (long long)cap, (long long)nb);
  const size_t V = (size_t)nb * m->B * m->B * m->B;
  if (V && (offsets || has_site)) {
    std::vector<unsigned long long> w(V);
    cudaError_t e = cudaMemcpy(w.data(), m->d.esdf, V * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy esdf");
    for (size_t i = 0; i < V; ++i) {
      const bool has = ((w[i] >> 8) & vbx::kHasSite) != 0;
      if (has_site) has_site[i] = has ? 1 : 0;
      if (offsets) {
        offsets[3 * i] = has ? (int8_t)(w[i] & 0xff) : 0;
        offsets[3 * i + 1] = has ? (int8_t)((w[i] >> 16) & 0xff) : 0;
        offsets[3 * i + 2] = has ? (int8_t)((w[i] >> 24) & 0xff) : 0;
      }
    }
  }
  return read_error(m, (cudaStream_t)stream);
}

vbx_status vbx_export_updated(vbx_map_t m, int32_t* vox, int64_t cap, int64_t* n_out, void* stream) {
  if (!m || !n_out) return fail(VBX_ERR_INVALID_ARG, "map or n_out is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  unsigned nu = 0, nb = 0;
  cudaMemcpy(&nu, &m->d.ctr->nupdated, sizeof(nu), cudaMemcpyDeviceToHost);
  cudaMemcpy(&nb, &m->d.ctr->blocks, sizeof(nb), cudaMemcpyDeviceToHost);
  nb = std::min<unsigned>(nb, m->d.cap_blocks);
  *n_out = nu;
  const int64_t k = std::min<int64_t>(cap, nu);
  if (k > 0 && vox) {
    std::vector<uint32_t> ids((size_t)k);
    std::vector<int3> bc(nb);
    e = cudaMemcpy(ids.data(), m->d.updated, (size_t)k * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "copy updated");
    if (nb) {
      e = cudaMemcpy(bc.data(), m->d.bcoord, (size_t)nb * sizeof(int3), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return cuda_fail(e, "copy keys");
    }
    const int B = m->B, blog = m->d.blog;
    for (int64_t i = 0; i < k; ++i) {
      const uint32_t slot = ids[i] >> m->d.b3log;
      const uint32_t l = ids[i] & ((1u << m->d.b3log) - 1u);
      const int3 b = slot < nb ? bc[slot] : int3{0, 0, 0};
      vox[3 * i + 0] = b.x * B + (int)(l & (B - 1));
      vox[3 * i + 1] = b.y * B + (int)((l >> blog) & (B - 1));
      vox[3 * i + 2] = b.z * B + (int)(l >> (2 * blog));
    }
  }
  return read_error(m, (cudaStream_t)stream);
}

vbx_status vbx_import_tsdf(vbx_map_t m, const int32_t* vox, const float* D, const float* W, int64_t n, void* stream) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  if (n < 0 || n > (int64_t(1) << 30)) return fail(VBX_ERR_INVALID_ARG, "n must lie in [0, 2^30]");
  if (n > 0 && (!vox || !D || !W)) return fail(VBX_ERR_INVALID_ARG, "import buffers must not be NULL");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(m->d.ctr, 0, offsetof(vbx::Counters, blocks), s);
  if (e != cudaSuccess) return cuda_fail(e, "reset scan counters");
  if (n == 0) return read_error(m, s);
  for (int64_t i = 0; i < 3 * n; ++i)
    if (vox[i] <= -(1 << 20) || vox[i] >= (1 << 20)) return fail(VBX_ERR_INVALID_ARG, "voxel coordinate out of range");
  int* dv = nullptr;
  float *dD = nullptr, *dW = nullptr;
  if ((e = cudaMalloc(&dv, (size_t)n * 3 * sizeof(int))) != cudaSuccess) return cuda_fail(e, "import buffers");
  if ((e = cudaMalloc(&dD, (size_t)n * sizeof(float))) != cudaSuccess) {
    cudaFree(dv);
    return cuda_fail(e, "import buffers");
  }
  if ((e = cudaMalloc(&dW, (size_t)n * sizeof(float))) != cudaSuccess) {
    cudaFree(dv);
    cudaFree(dD);
    return cuda_fail(e, "import buffers");
  }
  cudaMemcpyAsync(dv, vox, (size_t)n * 3 * sizeof(int), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dD, D, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(dW, W, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s);
  e = vbx::launch_import(m->d, dv, dD, dW, (int)n, m->cfg(stream), &m->hook);
  cudaError_t e2 = cudaStreamSynchronize(s);
  cudaFree(dv);
  cudaFree(dD);
  cudaFree(dW);
  if (e != cudaSuccess) return cuda_fail(e, "import launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "import sync");
  return read_error(m, s);
}

static_assert(sizeof(vbx_mesh_block) == sizeof(vbx::MeshBlockRec), "vbx_mesh_block layout");
static_assert(offsetof(vbx_mesh_block, first_triangle) == offsetof(vbx::MeshBlockRec, first), "vbx_mesh_block layout");

vbx_status vbx_extract_mesh(vbx_map_t m, int updated_only, int32_t* cells, float* verts, int64_t tri_cap,
                            vbx_mesh_block* blocks, int64_t block_cap, int64_t* n_tri_out, int64_t* n_blocks_out,
                            void* stream) {
  if (!m || !n_tri_out || !n_blocks_out) return fail(VBX_ERR_INVALID_ARG, "map or an output count is NULL");
  if (tri_cap < 0 || block_cap < 0) return fail(VBX_ERR_INVALID_ARG, "negative capacity");
  if (tri_cap > 0 && (!cells || !verts)) return fail(VBX_ERR_INVALID_ARG, "triangle buffers are NULL");
  if (block_cap > 0 && !blocks) return fail(VBX_ERR_INVALID_ARG, "block buffer is NULL");
  if (((uintptr_t)cells & 15u) || ((uintptr_t)blocks & 7u) || ((uintptr_t)verts & 3u))
    return fail(VBX_ERR_INVALID_ARG, "cells_dev must be 16-byte aligned (blocks_dev 8, verts_dev 4)");
  const cudaStream_t s = (cudaStream_t)stream;
  const size_t off = offsetof(vbx::Counters, mesh_tris);
  cudaError_t e = cudaMemsetAsync((char*)m->d.ctr + off, 0, sizeof(vbx::Counters) - off, s);
  if (e != cudaSuccess) return cuda_fail(e, "clear mesh counters");
  vbx::MeshOut o;
  o.cells = reinterpret_cast<int4*>(cells);
  o.verts = verts;
  o.tri_cap = (unsigned long long)tri_cap;
  o.blocks = reinterpret_cast<vbx::MeshBlockRec*>(blocks);
  o.block_cap = (unsigned long long)block_cap;
  if ((e = vbx::launch_mesh(m->d, updated_only == 0, o, m->cfg(stream), &m->hook)) != cudaSuccess)
    return cuda_fail(e, "mesh launch");
  vbx::Counters c;  // one copy brings the error word and the sizes
  if ((e = cudaMemcpyAsync(&c, m->d.ctr, sizeof(c), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return cuda_fail(e, "read mesh sizes");
  if (c.error) return read_error(m, s);
  const unsigned long long ntri = c.mesh_tris;
  const unsigned nblk = c.mesh_blocks;
  *n_tri_out = (int64_t)ntri;
  *n_blocks_out = (int64_t)nblk;
  if ((int64_t)ntri > tri_cap || (int64_t)nblk > block_cap)
    return fail(VBX_ERR_CAPACITY, "mesh needs %llu triangles and %u blocks (capacities %lld, %lld)", ntri, nblk,
                (long long)tri_cap, (long long)block_cap);
  if ((e = vbx::launch_mesh_clear(m->d, m->cfg(stream), &m->hook)) != cudaSuccess) return cuda_fail(e, "mesh clear");
  return VBX_OK;
}

vbx_status vbx_set_profiling(vbx_map_t m, int enable) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  m->hook.profile = enable != 0;
  return VBX_OK;
}

vbx_status vbx_get_kernel_times(vbx_map_t m, const char** names, double* ms, int64_t* launches, int cap, int* n_out,
                                void* stream) {
  if (!m || !n_out) return fail(VBX_ERR_INVALID_ARG, "map or n_out is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  m->hook.collect();
  *n_out = vbx::kNumKernels;
  for (int i = 0; i < vbx::kNumKernels && i < cap; ++i) {
    if (names) names[i] = vbx::kKernelNames[i];
    if (ms) ms[i] = m->hook.ms[i];
    if (launches) launches[i] = m->hook.count[i];
  }
  return VBX_OK;
}

vbx_status vbx_reset_kernel_times(vbx_map_t m) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  m->hook.collect();
  for (int i = 0; i < vbx::kNumKernels; ++i) {
    m->hook.ms[i] = 0.0;
    m->hook.count[i] = 0;
  }
  return VBX_OK;
}

// ------------------------------------------------------------------------------- batches

}  // extern "C"

struct vbx_batch_s {
  int count = 0;
  int device = 0;
  int num_sms = 0;
  int max_B = 4;
  int64_t max_queries = 0;
  std::vector<vbx_map_t> maps;
  // device descriptor block: DevMap[count] | ScanDesc[count] | QueryDesc[count]
  unsigned char* dev_block = nullptr;
  size_t block_bytes = 0;
  // pinned host copies of the descriptors, a ring of kStages: a step waits only for the step
  // issued kStages calls earlier, so a caller can keep several steps in flight
  static constexpr int kStages = 4;
  unsigned char* staging[kStages] = {};
  cudaEvent_t staged[kStages] = {};
  uint64_t steps = 0;
  vbx::EsdfCtl* ctl_dev = nullptr;
  std::vector<void*> dev_allocs;
  vbx::Tuning tune = vbx::kDefaultTuning;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graphs[kStages][8] = {};
  long long graph_kernels[kStages][8] = {};  // kernels captured into each graph
  uint64_t ctl_cap = 0;  // tiles the ESDF active lists hold (host copy of ctl.cap)
  MapHook hook;

  vbx::DevMap* maps_dev() const { return reinterpret_cast<vbx::DevMap*>(dev_block); }
  vbx::ScanDesc* scans_dev() const { return reinterpret_cast<vbx::ScanDesc*>(dev_block + count * sizeof(vbx::DevMap)); }
  vbx::QueryDesc* queries_dev() const {
    return reinterpret_cast<vbx::QueryDesc*>(dev_block + count * (sizeof(vbx::DevMap) + sizeof(vbx::ScanDesc)));
  }
  vbx::Batch batch_arg() const {
    vbx::Batch b;
    std::memset(&b, 0, sizeof(b));
    b.maps = maps_dev();
    b.scans = scans_dev();
    b.queries = queries_dev();
    b.nmaps = count;
    return b;
  }
  void drop_graphs() {
    for (auto& row : graphs)
      for (auto& g : row)
        if (g) {
          cudaGraphExecDestroy(g);
          g = nullptr;
        }
  }
  ~vbx_batch_s() {
    cudaDeviceSynchronize();
    drop_graphs();
    for (int k = 0; k < kStages; ++k) {
      if (staging[k]) cudaFreeHost(staging[k]);
      if (staged[k]) cudaEventDestroy(staged[k]);
    }
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (void* p : dev_allocs) cudaFree(p);
  }
};

namespace {

vbx_status batch_enqueue(vbx_batch_t b, int k, int flags, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(b->dev_block, b->staging[k], b->block_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "batch descriptors");
  const vbx::LaunchCfg cfg{b->num_sms, s, b->tune};
  const vbx::Batch arg = b->batch_arg();
  if (flags & (VBX_STEP_INTEGRATE | VBX_STEP_ESDF)) {
    if ((e = vbx::launch_reset_counters(arg, cfg, &b->hook)) != cudaSuccess) return cuda_fail(e, "batch reset");
  }
  if (flags & VBX_STEP_INTEGRATE) {
    if ((e = vbx::launch_integrate(arg, cfg, &b->hook)) != cudaSuccess) return cuda_fail(e, "batch integrate");
  }
  if (flags & VBX_STEP_ESDF) {
    if ((e = cudaMemsetAsync(b->ctl_dev, 0, offsetof(vbx::EsdfCtl, cap), s)) != cudaSuccess)
      return cuda_fail(e, "batch esdf reset");
    // the kernel keeps rounds when many maps have work (full rounds), queues when few do
    if ((e = vbx::launch_esdf(b->maps_dev(), b->count, b->max_B, b->ctl_dev, cfg, &b->hook, true)) != cudaSuccess)
      return cuda_fail(e, "batch esdf");
  }
  if (flags & VBX_STEP_QUERY) {
    const unsigned maxq = (unsigned)std::min<int64_t>(b->max_queries * b->count, (int64_t)UINT32_MAX);
    if ((e = vbx::launch_query(arg, maxq, cfg, &b->hook)) != cudaSuccess) return cuda_fail(e, "batch query");
  }
  return VBX_OK;
}

vbx_status batch_stage(vbx_batch_t b, const vbx_scan_in* scans, const vbx_query_io* queries, int flags, cudaStream_t s,
                       int* k_out) {
  for (int i = 0; i < b->count; ++i) {
    if (flags & VBX_STEP_INTEGRATE) {
      if (!scans) return fail(VBX_ERR_INVALID_ARG, "scans is NULL");
      if (scans[i].n < 0 || scans[i].n > b->maps[i]->pts_cap)
        return fail(VBX_ERR_INVALID_ARG, "slot %d: n = %lld outside [0, %lld], the map's per-scan capacity", i,
                    (long long)scans[i].n, (long long)b->maps[i]->pts_cap);
      if (scans[i].n > 0 && !scans[i].points_dev) return fail(VBX_ERR_INVALID_ARG, "slot %d: points_dev is NULL", i);
    }
    if (flags & VBX_STEP_QUERY) {
      if (!queries) return fail(VBX_ERR_INVALID_ARG, "queries is NULL");
      if (queries[i].n < 0 || queries[i].n > b->max_queries)
        return fail(VBX_ERR_INVALID_ARG, "slot %d: query n outside [0, max_queries]", i);
      if (queries[i].n > 0 && (!queries[i].q_dev || !queries[i].dist_dev || !queries[i].grad_dev || !queries[i].status_dev))
        return fail(VBX_ERR_INVALID_ARG, "slot %d: query buffers must not be NULL", i);
    }
  }
  const int k = (int)(b->steps % vbx_batch_s::kStages);
  cudaError_t e = cudaEventSynchronize(b->staged[k]);
  if (e != cudaSuccess) return cuda_fail(e, "batch staging wait");
  unsigned char* st = b->staging[k];
  auto* dm = reinterpret_cast<vbx::DevMap*>(st);
  auto* sd = reinterpret_cast<vbx::ScanDesc*>(st + b->count * sizeof(vbx::DevMap));
  auto* qd = reinterpret_cast<vbx::QueryDesc*>(st + b->count * (sizeof(vbx::DevMap) + sizeof(vbx::ScanDesc)));
  for (int i = 0; i < b->count; ++i) {
    dm[i] = b->maps[i]->d;
    vbx::ScanDesc d{};
    if ((flags & VBX_STEP_INTEGRATE) && scans) {
      if ((e = next_scan_epoch(b->maps[i], s, &d.epoch)) != cudaSuccess) return cuda_fail(e, "scan epoch");
      d.pts = scans[i].points_dev;
      d.n = (unsigned)scans[i].n;
      std::memcpy(d.T, scans[i].T_world_sensor, sizeof(d.T));
      b->maps[i]->last_points_in = scans[i].n;
    }
    sd[i] = d;
    vbx::QueryDesc q{};
    if ((flags & VBX_STEP_QUERY) && queries) {
      q.q = queries[i].q_dev;
      q.n = (unsigned)queries[i].n;
      q.dist = queries[i].dist_dev;
      q.grad = queries[i].grad_dev;
      q.status = queries[i].status_dev;
    }
    qd[i] = q;
  }
  *k_out = k;
  return VBX_OK;
}

vbx_status batch_run(vbx_batch_t b, const vbx_scan_in* scans, const vbx_query_io* queries, int flags, cudaStream_t s) {
  int k = 0;
  vbx_status st = batch_stage(b, scans, queries, flags, s, &k);
  if (st != VBX_OK) return st;
  const int f = flags & 7;
  cudaError_t e;
  if (flags & VBX_STEP_GRAPH) {
    if (!b->graphs[k][f]) {
      // capture on the batch's own stream (the legacy default stream cannot be captured)
      if ((e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return cuda_fail(e, "begin capture");
      const long long launches_before = b->hook.launches;
      st = batch_enqueue(b, k, f, b->cap_stream);
      b->graph_kernels[k][f] = b->hook.launches - launches_before;
      g_total_launches.fetch_sub(b->graph_kernels[k][f]);  // captured, not launched
      b->hook.launches = launches_before;
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(b->cap_stream, &g);
      if (st != VBX_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(e, "end capture");
      e = cudaGraphInstantiate(&b->graphs[k][f], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
    }
    if ((e = cudaGraphLaunch(b->graphs[k][f], s)) != cudaSuccess) return cuda_fail(e, "graph launch");
    // count the kernels the graph runs
    b->hook.launches += b->graph_kernels[k][f];
    g_total_launches.fetch_add(b->graph_kernels[k][f]);
  } else {
    st = batch_enqueue(b, k, f, s);
    if (st != VBX_OK) return st;
  }
  if ((e = cudaEventRecord(b->staged[k], s)) != cudaSuccess) return cuda_fail(e, "batch event");
  b->steps += 1;
  return VBX_OK;
}

}  // namespace

extern "C" {

vbx_status vbx_batch_create(const vbx_map_t* maps, int count, int64_t max_queries, vbx_batch_t* out) {
  if (!out) return fail(VBX_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!maps || count < 1 || count > vbx::kMaxBatch) return fail(VBX_ERR_INVALID_ARG, "count must lie in [1, %d]", vbx::kMaxBatch);
  if (max_queries < 0 || max_queries > (int64_t(1) << 26)) return fail(VBX_ERR_INVALID_ARG, "max_queries out of range");
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  for (int i = 0; i < count; ++i) {
    if (!maps[i]) return fail(VBX_ERR_INVALID_ARG, "slot %d: map is NULL", i);
    if (maps[i]->device != device) return fail(VBX_ERR_INVALID_ARG, "slot %d: map lives on another device", i);
    if (maps[i]->opt.euclidean) return fail(VBX_ERR_INVALID_ARG, "slot %d: Euclidean maps are updated one at a time", i);
    for (int j = 0; j < i; ++j)
      if (maps[j] == maps[i]) return fail(VBX_ERR_INVALID_ARG, "a map is bound to two slots");
  }
  vbx_batch_s* b = new vbx_batch_s();
  b->count = count;
  b->device = device;
  b->num_sms = maps[0]->num_sms;
  b->max_queries = max_queries;
  b->maps.assign(maps, maps + count);
  uint64_t cap_sum = 0;
  for (int i = 0; i < count; ++i) {
    b->max_B = std::max(b->max_B, maps[i]->B);
    cap_sum += (uint64_t)maps[i]->d.cap_blocks << maps[i]->d.tile_shift;
  }
  b->block_bytes = (size_t)count * (sizeof(vbx::DevMap) + sizeof(vbx::ScanDesc) + sizeof(vbx::QueryDesc));
  auto dalloc = [&](void** p, size_t bytes) -> cudaError_t {
    cudaError_t r = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (r == cudaSuccess) {
      b->dev_allocs.push_back(*p);
      r = cudaMemset(*p, 0, std::max<size_t>(bytes, 16));
    }
    return r;
  };
  vbx::EsdfCtl ctl{};
  ctl.cap = (unsigned)std::min<uint64_t>(cap_sum, UINT32_MAX);
  const uint64_t ring = lower_ring_slots(cap_sum, b->num_sms);
  ctl.rcap = (unsigned)std::min<uint64_t>(ring, UINT32_MAX);
  if ((e = dalloc((void**)&b->dev_block, b->block_bytes)) != cudaSuccess ||
      (e = dalloc((void**)&ctl.lring, ring * sizeof(uint2))) != cudaSuccess ||
      (e = dalloc((void**)&ctl.ltag, ring * sizeof(unsigned long long))) != cudaSuccess ||
      (e = dalloc((void**)&b->ctl_dev, sizeof(vbx::EsdfCtl))) != cudaSuccess ||
      (e = dalloc((void**)&ctl.ract0, cap_sum * sizeof(uint2))) != cudaSuccess ||
      (e = dalloc((void**)&ctl.ract1, cap_sum * sizeof(uint2))) != cudaSuccess ||
      (e = dalloc((void**)&ctl.lact0, cap_sum * sizeof(uint2))) != cudaSuccess ||
      (e = dalloc((void**)&ctl.lact1, cap_sum * sizeof(uint2))) != cudaSuccess ||
      (e = cudaMemcpy(b->ctl_dev, &ctl, sizeof(ctl), cudaMemcpyHostToDevice)) != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch buffers");
  }
  b->ctl_cap = ctl.cap;
  for (int k = 0; k < vbx_batch_s::kStages; ++k) {
    if ((e = cudaMallocHost((void**)&b->staging[k], b->block_bytes)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->staged[k], cudaEventDisableTiming)) != cudaSuccess) {
      delete b;
      return cuda_fail(e, "batch staging");
    }
  }
  if ((e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    delete b;
    return cuda_fail(e, "capture stream");
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
    delete b;
    return cuda_fail(e, "batch create sync");
  }
  *out = b;
  return VBX_OK;
}

vbx_status vbx_batch_bind(vbx_batch_t b, int slot, vbx_map_t map) {
  if (!b || !map) return fail(VBX_ERR_INVALID_ARG, "batch or map is NULL");
  if (slot < 0 || slot >= b->count) return fail(VBX_ERR_INVALID_ARG, "slot out of range");
  if (map->device != b->device) return fail(VBX_ERR_INVALID_ARG, "map lives on another device");
  if (map->opt.euclidean) return fail(VBX_ERR_INVALID_ARG, "Euclidean maps are updated one at a time");
  for (int j = 0; j < b->count; ++j)
    if (j != slot && b->maps[j] == map) return fail(VBX_ERR_INVALID_ARG, "map already bound to slot %d", j);
  // the ESDF active lists were sized for the bound maps' pools
  uint64_t cap_sum = 0;
  for (int j = 0; j < b->count; ++j) {
    const vbx_map_t mj = j == slot ? map : b->maps[j];
    cap_sum += (uint64_t)mj->d.cap_blocks << mj->d.tile_shift;
  }
  const bool grow_lists = cap_sum > b->ctl_cap;
  const bool new_shape = map->B > b->max_B;  // the ESDF launch's shared-memory tile must fit the largest block
  if (!grow_lists && !new_shape) {
    // steps read the slot's map from the descriptors they stage, so in-flight steps keep the
    // map they were issued with and the next step takes the new one: no synchronisation
    b->maps[slot] = map;
    return VBX_OK;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "bind sync");
  if (new_shape) {
    b->max_B = map->B;
    b->drop_graphs();
  }
  if (grow_lists) {
    vbx::EsdfCtl ctl{};
    if ((e = cudaMemcpy(&ctl, b->ctl_dev, sizeof(ctl), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return cuda_fail(e, "esdf control");
    // grow geometrically: a server binding maps one by one reallocates a few times, not per map
    const uint64_t cap = std::min<uint64_t>(std::max<uint64_t>(cap_sum, 2 * b->ctl_cap), UINT32_MAX);
    const uint64_t ring = lower_ring_slots(cap, b->num_sms);
    const size_t bytes[6] = {cap * sizeof(uint2), cap * sizeof(uint2), cap * sizeof(uint2),
                             cap * sizeof(uint2), ring * sizeof(uint2), ring * sizeof(unsigned long long)};
    void* lists[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 6; ++i) {
      if ((e = cudaMalloc(&lists[i], bytes[i])) != cudaSuccess ||
          (e = cudaMemset(lists[i], 0, bytes[i])) != cudaSuccess) {
        for (int j = 0; j <= i; ++j) cudaFree(lists[j]);
        return cuda_fail(e, "esdf lists");
      }
    }
    for (int i = 0; i < 6; ++i) b->dev_allocs.push_back(lists[i]);
    ctl.ract0 = (uint2*)lists[0];
    ctl.ract1 = (uint2*)lists[1];
    ctl.lact0 = (uint2*)lists[2];
    ctl.lact1 = (uint2*)lists[3];
    ctl.lring = (uint2*)lists[4];
    ctl.ltag = (unsigned long long*)lists[5];
    ctl.rcap = (unsigned)std::min<uint64_t>(ring, UINT32_MAX);
    ctl.cap = (unsigned)cap;
    if ((e = cudaMemcpy(b->ctl_dev, &ctl, sizeof(ctl), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cuda_fail(e, "esdf control");
    b->ctl_cap = ctl.cap;
  }
  b->maps[slot] = map;
  return VBX_OK;
}

vbx_status vbx_batch_step(vbx_batch_t b, const vbx_scan_in* scans, const vbx_query_io* queries, int flags, void* stream) {
  if (!b) return fail(VBX_ERR_INVALID_ARG, "batch is NULL");
  return batch_run(b, scans, queries, flags, (cudaStream_t)stream);
}

vbx_status vbx_batch_autotune(vbx_batch_t b, const vbx_scan_in* scans, const vbx_query_io* queries, int flags, void* stream,
                              char* report, int report_len) {
  if (!b) return fail(VBX_ERR_INVALID_ARG, "batch is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  const int f = flags & 7;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int trials = 0;
  auto time_step = [&](float* ms) -> vbx_status {
    ++trials;
    cudaEventRecord(e0, s);
    vbx_status st = batch_run(b, scans, queries, f, s);
    if (st != VBX_OK) return st;
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune sync");
    cudaEventElapsedTime(ms, e0, e1);
    return VBX_OK;
  };
  vbx::Tuning best = b->tune;
  float best_ms = 1e30f;
  vbx_status st = VBX_OK;
  // one untimed step first: the first step on fresh maps builds them from scratch, the later
  // ones (the same scans again) see comparable work
  {
    float ms = 0.0f;
    if ((st = time_step(&ms)) != VBX_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return st;
    }
  }
  // a candidate's time is the better of two steps; a later candidate replaces the best only
  // when it is clearly faster (the trial steps repeat the same scans, so their ESDF work is
  // small and differences within a few per cent are noise; the candidates are listed with the
  // usual winner first)
  constexpr float kMargin = 0.97f;
  auto time_candidate = [&](float* ms) -> vbx_status {
    float a = 0.0f, c = 0.0f;
    vbx_status s2 = time_step(&a);
    if (s2 == VBX_OK) s2 = time_step(&c);
    *ms = std::min(a, c);
    return s2;
  };
  // coordinate search: traversal grid first, then the cooperative ESDF grid
  const int rays_opts[3] = {8, 16, 32};
  for (int r : rays_opts) {
    b->tune = best;
    b->tune.rays_ctas_per_sm = r;
    float ms = 0.0f;
    if ((st = time_candidate(&ms)) != VBX_OK) break;
    if (ms < best_ms * kMargin) {
      best_ms = ms;
      best = b->tune;
    }
  }
  if (st == VBX_OK && (f & VBX_STEP_ESDF)) {
    best_ms = 1e30f;
    // (threads per CTA, CTAs per SM) of the cooperative ESDF grid; the grid is clamped to the
    // kernel's occupancy
    const int esdf_opts[5][2] = {{128, 12}, {128, 8}, {256, 6}, {256, 4}, {512, 2}};
    for (const auto& o : esdf_opts) {
      b->tune = best;
      b->tune.esdf_threads = o[0];
      b->tune.esdf_ctas_per_sm = o[1];
      float ms = 0.0f;
      if ((st = time_candidate(&ms)) != VBX_OK) break;
      if (ms < best_ms * kMargin) {
        best_ms = ms;
        best = b->tune;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tune = best;
  b->drop_graphs();  // launch shapes changed
  if (report && report_len > 0)
    snprintf(report, (size_t)report_len, "rays_ctas_per_sm=%d esdf_ctas_per_sm=%d esdf_threads=%d bin_ctas_per_sm=%d apply_ctas_per_sm=%d best_step_ms=%.4f trial_steps=%d",
             best.rays_ctas_per_sm, best.esdf_ctas_per_sm, best.esdf_threads, best.bin_ctas_per_sm, best.apply_ctas_per_sm, best_ms, trials);
  return st;
}

vbx_status vbx_batch_set_profiling(vbx_batch_t b, int enable) {
  if (!b) return fail(VBX_ERR_INVALID_ARG, "batch is NULL");
  b->hook.profile = enable != 0;
  return VBX_OK;
}

vbx_status vbx_batch_kernel_times(vbx_batch_t b, const char** names, double* ms, int64_t* launches, int cap, int* n_out,
                                  void* stream) {
  if (!b || !n_out) return fail(VBX_ERR_INVALID_ARG, "batch or n_out is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "sync");
  b->hook.collect();
  *n_out = vbx::kNumKernels;
  for (int i = 0; i < vbx::kNumKernels && i < cap; ++i) {
    if (names) names[i] = vbx::kKernelNames[i];
    if (ms) ms[i] = b->hook.ms[i];
    if (launches) launches[i] = b->hook.count[i];
  }
  return VBX_OK;
}

vbx_status vbx_batch_sync(vbx_batch_t b, void* stream) {
  if (!b) return fail(VBX_ERR_INVALID_ARG, "batch is NULL");
  vbx_status first = VBX_OK;
  for (int i = 0; i < b->count; ++i) {
    vbx_status st = read_error(b->maps[i], (cudaStream_t)stream);
    if (st != VBX_OK && first == VBX_OK) first = st;
  }
  return first;
}

vbx_status vbx_batch_destroy(vbx_batch_t b) {
  delete b;
  return VBX_OK;
}

vbx_status vbx_map_bytes(int B, const vbx_map_options* opt_in, int64_t* out) {
  if (!out) return fail(VBX_ERR_INVALID_ARG, "bytes_out is NULL");
  if (B != 4 && B != 8 && B != 16) return fail(VBX_ERR_INVALID_ARG, "voxels_per_block must be 4, 8 or 16");
  vbx_map_options opt;
  vbx_default_options(&opt);
  if (opt_in) opt = *opt_in;
  const uint64_t B3 = (uint64_t)B * B * B;
  const uint64_t cap = opt.block_capacity > 0 ? (uint64_t)opt.block_capacity : (uint64_t(1) << 25) / B3;
  const uint64_t V = cap * B3;
  const uint64_t tiles = cap << (B == 16 ? 3 : 0);
  const uint64_t H = next_pow2(cap * 2);
  const uint64_t pts = next_pow2((uint64_t)std::max<int64_t>(opt.max_points > 0 ? opt.max_points : (int64_t(1) << 20), 1024));
  const uint64_t entries = next_pow2(pts * 2);
  const uint64_t scr = opt.scratch_blocks > 0 ? std::min<uint64_t>((uint64_t)opt.scratch_blocks, cap) : cap;
  uint64_t bytes = 0;
  bytes += H * (8 + 4 + 4);                               // block hash, scratch claims
  bytes += cap * (12 + 27 * 4 + 8 + 4 + 1 + 4);           // block coords, links, scratch index/epoch, new list,
                                                          // mesh marks and list
  bytes += V * (8 + 8 + 1 + 4 + 4);                       // tsdf, esdf, flags, updated and dirty lists
  bytes += scr * (4 + 4 + 27 * 4) + scr * B3 * (32 + 1);  // scratch blocks: lists, neighbour links, sums, touch flags
  bytes += 5 * (V / 32) * 4;                              // frontier and pull bitmasks
  bytes += tiles * (2 * 4 + 4 * 8);                       // tile stamps, active lists
  {
    int dev = 0, sms = 152;  // lower-wave queue ring (this device's SM count, else 152)
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      sms = 152;
    }
    bytes += lower_ring_slots(tiles, sms) * (8 + 8);
  }
  bytes += entries * sizeof(vbx::GroupEntry) + pts * (4 + 16);  // per-scan scratch
  *out = (int64_t)bytes;
  return VBX_OK;
}

vbx_status vbx_map_device_bytes(vbx_map_t m, int64_t* out) {
  if (!m || !out) return fail(VBX_ERR_INVALID_ARG, "map or bytes_out is NULL");
  size_t total = 0;
  for (size_t b : m->alloc_bytes) total += b;
  *out = (int64_t)total;
  return VBX_OK;
}

vbx_status vbx_reset_map(vbx_map_t m, void* stream) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  cudaError_t e = vbx::launch_reset_map(m->d, m->cfg(stream));
  if (e != cudaSuccess) return cuda_fail(e, "reset");
  m->last_points_in = 0;
  return VBX_OK;
}

int64_t vbx_total_launches(void) { return g_total_launches.load(); }

const char* vbx_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
