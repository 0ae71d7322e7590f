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
const char* const kKernelNames[kNumKernels] = {"bin_points",  "group_rays",   "link_blocks", "integrate_rays",
                                               "apply",       "esdf",         "query",       "import_alloc",
                                               "import_set",  "init_groups"};
}  // namespace vbx

namespace {

thread_local std::string g_last_error;
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
  std::vector<void*> allocs;
  MapHook hook;

  vbx::LaunchCfg cfg(void* stream) const { return vbx::LaunchCfg{num_sms, (cudaStream_t)stream}; }

  template <typename T>
  cudaError_t alloc(T** p, size_t count, int fill_byte) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 16));
    if (e != cudaSuccess) return e;
    allocs.push_back(q);
    e = cudaMemset(q, fill_byte, std::max<size_t>(count * sizeof(T), 16));
    *p = (T*)q;
    return e;
  }
  void release(void* p) {
    if (!p) return;
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (it != allocs.end()) allocs.erase(it);
    cudaFree(p);
  }
  ~vbx_map_s() {
    for (void* p : allocs) cudaFree(p);
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
  d.weighting = opt.weighting;
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
  VBX_ALLOC(d.hkeys, H, 0xff);
  VBX_ALLOC(d.hvals, H, 0xff);
  VBX_ALLOC(d.bcoord, (size_t)cap, 0);
  VBX_ALLOC(d.nbr, (size_t)cap * 27, 0xff);
  VBX_ALLOC(d.tsdf, V, 0);
  VBX_ALLOC(d.acc, 4 * V, 0);
  VBX_ALLOC(d.touch, V, 0);
  VBX_ALLOC(d.btouch, (size_t)cap, 0);
  VBX_ALLOC(d.esdf, V, 0);
  VBX_ALLOC(d.vflags, V, 0);
  VBX_ALLOC(d.rbits0, V / 32, 0);
  VBX_ALLOC(d.rbits1, V / 32, 0);
  VBX_ALLOC(d.lbits0, V / 32, 0);
  VBX_ALLOC(d.lbits1, V / 32, 0);
  VBX_ALLOC(d.bstamp_r, (size_t)cap, 0);
  VBX_ALLOC(d.bstamp_l, (size_t)cap, 0);
  VBX_ALLOC(d.updated, V, 0);
  VBX_ALLOC(d.dirty, V, 0);
  VBX_ALLOC(d.newblk, (size_t)cap, 0);
  VBX_ALLOC(d.ctr, 1, 0);
  VBX_ALLOC(m->d_dev, 1, 0);
  VBX_ALLOC(m->ctl_dev, 1, 0);
  {
    vbx::EsdfCtl ctl{};
    ctl.cap = (unsigned)cap;
    VBX_ALLOC(ctl.ract0, (size_t)cap, 0);
    VBX_ALLOC(ctl.ract1, (size_t)cap, 0);
    VBX_ALLOC(ctl.lact0, (size_t)cap, 0);
    VBX_ALLOC(ctl.lact1, (size_t)cap, 0);
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
  e = vbx::launch_integrate(m->d, points_dev, (int)n, pose, m->cfg(stream), &m->hook);
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
  e = vbx::launch_integrate_noalloc(m->d, scratch, points_dev, (int)n, pose, m->cfg(stream), &m->hook);
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
  e = vbx::launch_esdf(m->d_dev, 1, m->B, m->ctl_dev, m->cfg(stream), &m->hook);
  if (e != cudaSuccess) return cuda_fail(e, "esdf cooperative launch");
  return VBX_OK;
}

vbx_status vbx_query_distance_gradient(vbx_map_t m, const float* q_dev, int64_t n, float* dist_dev, float* grad_dev,
                                       uint8_t* status_dev, void* stream) {
  if (!m) return fail(VBX_ERR_INVALID_ARG, "map is NULL");
  if (n < 0 || n > (int64_t(1) << 30)) return fail(VBX_ERR_INVALID_ARG, "n must lie in [0, 2^30]");
  if (n > 0 && (!q_dev || !dist_dev || !grad_dev || !status_dev))
    return fail(VBX_ERR_INVALID_ARG, "query buffers must not be NULL");
  cudaError_t e = vbx::launch_query(m->d, q_dev, (int)n, dist_dev, grad_dev, status_dev, m->cfg(stream), &m->hook);
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

int64_t vbx_total_launches(void) { return g_total_launches.load(); }

const char* vbx_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
