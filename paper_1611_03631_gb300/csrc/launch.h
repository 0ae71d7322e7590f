// launch.h -- host-side launchers of the map-update kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "vbx_internal.cuh"

namespace vbx {

struct Pose {
  float T[16];  // row-major T_world_sensor
};

constexpr int kMaxBatch = 256;  // maps per batched launch (one prefix entry per thread of a CTA)

// One map's scan and query batch inside a batched launch.
struct ScanDesc {
  const float* pts;  // n x 3 float32, sensor frame (device)
  unsigned n;
  unsigned epoch;  // scan epoch of the map (> 0, increases by one per integrated scan)
  float T[16];  // row-major T_world_sensor
};

struct QueryDesc {
  const float* q;  // n x 3 (device)
  float* dist;
  float* grad;
  unsigned char* status;
  unsigned n;
  unsigned pad;
};

// Kernel parameter of every map-update kernel: either a device array of nmaps maps with their
// scan / query descriptors, or (maps == nullptr) the single map `one` with `one_scan` and
// `one_query` passed by value.
struct Batch {
  const DevMap* maps;
  const ScanDesc* scans;
  const QueryDesc* queries;
  int nmaps;
  DevMap one;
  ScanDesc one_scan;
  QueryDesc one_query;
};

// Launch shape knobs (chosen by the batch autotuner).
struct Tuning {
  int rays_ctas_per_sm;  // CTAs per SM of the voxel-traversal kernel
  int bin_ctas_per_sm;   // CTAs per SM of the point and group kernels
  int apply_ctas_per_sm;
  int esdf_ctas_per_sm;  // resident CTAs per SM of the cooperative ESDF grid
  int esdf_threads;      // threads per ESDF CTA (128 to 1024): one CTA relaxes one tile at a time
};
// Start point of the batch autotuner (the ESDF grid is clamped to the kernel's occupancy).
constexpr Tuning kDefaultTuning = {16, 16, 16, 8, 256};
// Calls on one map: the ESDF waves run as work queues. A wave advances as fast as a tile's local
// relaxation (wide CTAs shorten it) while several tiles along its front are in flight (more
// CTAs): updates of a few hundred thousand voxels (a room frame) are paced by the wave's
// critical path and run best as 512 x 2 per SM; updates of millions of voxels (a LiDAR scan)
// have tiles to spare, and every extra CTA per SM helps them (LiDAR ESDF 1.70 ms at 512 x 3,
// 1.54 at 256 x 4, 1.36 at 256 x 6, 1.30 at 256 x 8; room 0.31 ms at 512 x 2, 0.46 at 256 x 6).
#ifndef VBX_MAP_ESDF_THREADS
#define VBX_MAP_ESDF_THREADS 512
#endif
#ifndef VBX_MAP_ESDF_CTAS
#define VBX_MAP_ESDF_CTAS 2
#endif
constexpr Tuning kMapTuning = {16, 16, 16, VBX_MAP_ESDF_CTAS, VBX_MAP_ESDF_THREADS};
#ifndef VBX_MAP_LARGE_THREADS
#define VBX_MAP_LARGE_THREADS 256
#endif
#ifndef VBX_MAP_LARGE_CTAS
#define VBX_MAP_LARGE_CTAS 8
#endif
constexpr Tuning kMapTuningLarge = {16, 16, 16, VBX_MAP_LARGE_CTAS, VBX_MAP_LARGE_THREADS};
// Dirty voxels at or above which a map's update uses kMapTuningLarge (the previous update's
// count is the predictor: consecutive scans of a sequence update similar amounts).
constexpr unsigned kMapLargeUpdate = 1u << 19;

struct LaunchCfg {
  int num_sms;
  cudaStream_t stream;
  Tuning tune;
};

// Records one launch (for profiling and launch counting). Implemented by the API layer.
struct LaunchHook {
  virtual void begin(int kernel_id, cudaStream_t s) = 0;
  virtual void end(int kernel_id, cudaStream_t s) = 0;
  virtual ~LaunchHook() {}
};

enum KernelId {
  kKReset = 0,
  kKBin,
  kKGroupRays,
  kKLink,
  kKIntegrateRays,
  kKApply,
  kKEsdf,
  kKQuery,
  kKImportAlloc,
  kKImportSet,
  kKInitGroups,
  kKMeshSelect,
  kKMeshBlocks,
  kKMeshClear,
  kKScratchLinks,
  kNumKernels
};

extern const char* const kKernelNames[kNumKernels];

// integrate.cu
cudaError_t launch_init_groups(GroupEntry* tab, uint32_t entries, cudaStream_t s, LaunchHook* hook);
cudaError_t launch_integrate(const Batch& b, const LaunchCfg& cfg, LaunchHook* hook);
// zeroes the per-scan and per-ESDF counters of every map of a device array of maps
cudaError_t launch_reset_counters(const Batch& b, const LaunchCfg& cfg, LaunchHook* hook);
// Largest scan accepted by the allocation-free integration entry point.
constexpr int kNoAllocMaxPoints = 1 << 16;
cudaError_t noalloc_scratch_setup(int device, void** ptr);
cudaError_t launch_integrate_noalloc(const DevMap& m, void* scratch, const float* pts, int n, const Pose& T,
                                     unsigned epoch, const LaunchCfg& cfg, LaunchHook* hook);
Batch single_batch(const DevMap& m, const float* pts, int n, const Pose& T, unsigned epoch = 0);
cudaError_t launch_import(const DevMap& m, const int* vox, const float* D, const float* W, int n,
                          const LaunchCfg& cfg, LaunchHook* hook);
// empties the map on cfg.stream (no host synchronisation)
cudaError_t launch_reset_map(const DevMap& m, const LaunchCfg& cfg);

// esdf.cu: one cooperative launch updates the ESDF of nmaps maps (device array of DevMap)
size_t esdf_smem_bytes(int max_B);
// be: the block edge of a single map whose waves run as work queues (0: the batch kernel)
int esdf_grid(int num_sms, int max_B, int ctas_per_sm, int threads, int be = 0);
// allow_async: the raise and lower waves may run as asynchronous work queues instead of rounds
// (the kernel takes them when few maps of the launch have work)
// Full Euclidean ESDF update of one map (the map's device descriptor, block edge B).
cudaError_t launch_esdf_euclid(const DevMap* map_dev, int B, EsdfCtl* ctl, const LaunchCfg& cfg, LaunchHook* hook);
cudaError_t launch_esdf(const DevMap* maps_dev, int nmaps, int max_B, EsdfCtl* ctl, const LaunchCfg& cfg,
                        LaunchHook* hook, bool allow_async);

// mesh.cu: triangles of the TSDF iso-surface, per block
struct MeshBlockRec {  // same layout as vbx_mesh_block
  int32_t key[3];
  uint32_t ntri;
  long long first;
};
struct MeshOut {
  int4* cells;  // [tri_cap] cell minimum-corner voxel x, y, z and index in the cell
  float* verts;  // [tri_cap][3][3]
  unsigned long long tri_cap;
  MeshBlockRec* blocks;  // [block_cap]
  unsigned long long block_cap;
};
// Lists the blocks to mesh (all, or those with a stale cell) and writes their triangles; the
// sizes needed are left in the map's counters (mesh_tris, mesh_blocks), cleared beforehand by
// the caller.
cudaError_t launch_mesh(const DevMap& m, bool all, const MeshOut& o, const LaunchCfg& cfg, LaunchHook* hook);
// Drops the stale marks of the blocks the last launch_mesh listed.
cudaError_t launch_mesh_clear(const DevMap& m, const LaunchCfg& cfg, LaunchHook* hook);

// query.cu: b.queries (or b.one_query) give each map's query points and outputs
cudaError_t launch_query(const Batch& b, unsigned max_total, const LaunchCfg& cfg, LaunchHook* hook);

}  // namespace vbx
