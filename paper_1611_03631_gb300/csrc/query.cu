// query.cu -- distance and gradient queries on the ESDF (A9): trilinear interpolation of the
// 8 voxel centres around each query point (the evaluation used in Sec. VI-A of Oleynikova et
// al. 2017) and the analytic gradient of that interpolant, which the trajectory optimiser of
// Sec. VII consumes. A query is "unknown" if any of the 8 voxels is unobserved.
#include <cuda_runtime.h>

#include "launch.h"
#include "vbx_internal.cuh"

namespace vbx {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_query(DevMap m, const float* __restrict__ q, int n, float* __restrict__ dist,
                                                   float* __restrict__ grad, unsigned char* __restrict__ status) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int i0[3];
  float f[3];
  for (int a = 0; a < 3; ++a) {
    // corner selection in float32: t = fl(fl(q / v) - 1/2), i0 = floor(t), f = t - i0
    const float t = __fsub_rn(__fdiv_rn(__ldg(&q[3 * (size_t)i + a]), m.v), 0.5f);
    const float fl = floorf(t);
    i0[a] = (int)fl;
    f[a] = t - fl;
  }
  float c[8];
  bool ok = true;
  int last_b[3] = {0x7fffffff, 0, 0};
  uint32_t slot = kInvalid;
  const int B = m.B, blog = m.blog;
  for (int j = 0; j < 8 && ok; ++j) {
    const int x = i0[0] + (j >> 2), y = i0[1] + ((j >> 1) & 1), z = i0[2] + (j & 1);
    const int bx = x >> blog, by = y >> blog, bz = z >> blog;
    if (bx != last_b[0] || by != last_b[1] || bz != last_b[2]) {
      slot = block_lookup(m, bx, by, bz);
      last_b[0] = bx;
      last_b[1] = by;
      last_b[2] = bz;
    }
    if (slot == kInvalid) {
      ok = false;
      break;
    }
    const uint32_t vid = (slot << m.b3log) | (uint32_t)((((z & (B - 1)) << blog | (y & (B - 1))) << blog) | (x & (B - 1)));
    const unsigned long long w = __ldg(&m.esdf[vid]);
    if (!(ew_flags(w) & kObserved)) {
      ok = false;
      break;
    }
    c[j] = ew_d(w);
  }
  if (!ok) {
    const float nan = __int_as_float(0x7fc00000);
    dist[i] = nan;
    grad[3 * (size_t)i] = nan;
    grad[3 * (size_t)i + 1] = nan;
    grad[3 * (size_t)i + 2] = nan;
    status[i] = 1;
    return;
  }
  // c[j] with j = 4*bx + 2*by + bz
  const float fx = f[0], fy = f[1], fz = f[2];
  const float gx0 = 1.0f - fx, gy0 = 1.0f - fy, gz0 = 1.0f - fz;
  // interpolate along z, then y, then x
  const float c00 = c[0] * gz0 + c[1] * fz;  // bx=0, by=0
  const float c01 = c[2] * gz0 + c[3] * fz;  // bx=0, by=1
  const float c10 = c[4] * gz0 + c[5] * fz;  // bx=1, by=0
  const float c11 = c[6] * gz0 + c[7] * fz;  // bx=1, by=1
  const float c0 = c00 * gy0 + c01 * fy;
  const float c1 = c10 * gy0 + c11 * fy;
  const float d = c0 * gx0 + c1 * fx;
  const float ddx = c1 - c0;
  const float ddy = (c01 - c00) * gx0 + (c11 - c10) * fx;
  const float e00 = c[1] - c[0], e01 = c[3] - c[2], e10 = c[5] - c[4], e11 = c[7] - c[6];
  const float ddz = (e00 * gy0 + e01 * fy) * gx0 + (e10 * gy0 + e11 * fy) * fx;
  const float inv_v = 1.0f / m.v;
  dist[i] = d;
  grad[3 * (size_t)i] = ddx * inv_v;
  grad[3 * (size_t)i + 1] = ddy * inv_v;
  grad[3 * (size_t)i + 2] = ddz * inv_v;
  status[i] = 0;
}

}  // namespace

cudaError_t launch_query(const DevMap& m, const float* q, int n, float* dist, float* grad, unsigned char* status,
                         const LaunchCfg& cfg, LaunchHook* hook) {
  if (n <= 0) return cudaSuccess;
  hook->begin(kKQuery, cfg.stream);
  k_query<<<(n + kThreads - 1) / kThreads, kThreads, 0, cfg.stream>>>(m, q, n, dist, grad, status);
  hook->end(kKQuery, cfg.stream);
  return cudaGetLastError();
}

}  // namespace vbx
