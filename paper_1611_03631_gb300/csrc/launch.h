// launch.h -- host-side launchers of the map-update kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "vbx_internal.cuh"

namespace vbx {

struct Pose {
  float T[16];  // row-major T_world_sensor
};

struct LaunchCfg {
  int num_sms;
  cudaStream_t stream;
};

// Records one launch (for profiling and launch counting). Implemented by the API layer.
struct LaunchHook {
  virtual void begin(int kernel_id, cudaStream_t s) = 0;
  virtual void end(int kernel_id, cudaStream_t s) = 0;
  virtual ~LaunchHook() {}
};

enum KernelId {
  kKBin = 0,
  kKGroupRays,
  kKLink,
  kKIntegrateRays,
  kKApply,
  kKEsdf,
  kKQuery,
  kKImportAlloc,
  kKImportSet,
  kKInitGroups,
  kNumKernels
};

extern const char* const kKernelNames[kNumKernels];

// integrate.cu
cudaError_t launch_init_groups(GroupEntry* tab, uint32_t entries, cudaStream_t s, LaunchHook* hook);
cudaError_t launch_integrate(const DevMap& m, const float* pts, int n, const Pose& T, const LaunchCfg& cfg,
                             LaunchHook* hook);
// Largest scan accepted by the allocation-free integration entry point.
constexpr int kNoAllocMaxPoints = 1 << 16;
cudaError_t noalloc_scratch_setup(int device, void** ptr);
cudaError_t launch_integrate_noalloc(const DevMap& m, void* scratch, const float* pts, int n, const Pose& T,
                                     const LaunchCfg& cfg, LaunchHook* hook);
cudaError_t launch_import(const DevMap& m, const int* vox, const float* D, const float* W, int n,
                          const LaunchCfg& cfg, LaunchHook* hook);

// esdf.cu: one cooperative launch updates the ESDF of nmaps maps (device array of DevMap)
constexpr int kMaxBatch = 256;  // maps per ESDF launch (one prefix entry per thread)
size_t esdf_smem_bytes(int max_B);
int esdf_grid(int num_sms, int max_B);
cudaError_t launch_esdf(const DevMap* maps_dev, int nmaps, int max_B, EsdfCtl* ctl, const LaunchCfg& cfg,
                        LaunchHook* hook);

// query.cu
cudaError_t launch_query(const DevMap& m, const float* q, int n, float* dist, float* grad, unsigned char* status,
                         const LaunchCfg& cfg, LaunchHook* hook);

}  // namespace vbx
