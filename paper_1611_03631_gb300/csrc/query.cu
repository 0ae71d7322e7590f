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

__device__ __forceinline__ const DevMap& qmap_of(const Batch& b, unsigned mi) { return b.maps ? b.maps[mi] : b.one; }
__device__ __forceinline__ const QueryDesc& qdesc_of(const Batch& b, unsigned mi) { return b.queries ? b.queries[mi] : b.one_query; }

__global__ void __launch_bounds__(kThreads) k_query(Batch b) {
  __shared__ unsigned pfx[kMaxBatch + 1];
  const int nm = b.maps ? b.nmaps : 1;
  const int t = threadIdx.x;
  // exclusive prefix of the maps' query counts
  pfx[t + 1] = t < nm ? qdesc_of(b, t).n : 0u;
  if (t == 0) pfx[0] = 0u;
  __syncthreads();
  for (int off = 1; off < kMaxBatch && off < nm; off <<= 1) {
    const unsigned add = t >= off ? pfx[t + 1 - off] : 0u;
    __syncthreads();
    pfx[t + 1] += add;
    __syncthreads();
  }
  const unsigned total = pfx[nm];
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int lo = 0, hi = nm - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pfx[mid] <= i)
        lo = mid;
      else
        hi = mid - 1;
    }
    const DevMap& m = qmap_of(b, lo);
    const QueryDesc& qd = qdesc_of(b, lo);
    const unsigned j = i - pfx[lo];
    int i0[3];
    float f[3];
    for (int a = 0; a < 3; ++a) {
      // corner selection in float32: t = fl(fl(q / v) - 1/2), i0 = floor(t), f = t - i0
      const float tq = __fsub_rn(__fdiv_rn(__ldg(&qd.q[3 * (size_t)j + a]), m.v), 0.5f);
      const float fl = floorf(tq);
      i0[a] = (int)fl;
      f[a] = tq - fl;
    }
    float c[8];
    bool ok = true;
    int last_b[3] = {0x7fffffff, 0, 0};
    uint32_t slot = kInvalid;
    const int B = m.B, blog = m.blog;
    for (int k = 0; k < 8 && ok; ++k) {
      const int x = i0[0] + (k >> 2), y = i0[1] + ((k >> 1) & 1), z = i0[2] + (k & 1);
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
      const unsigned long long w = __ldcg(&m.esdf[vid]);
      if (!(ew_flags(w) & kObserved)) {
        ok = false;
        break;
      }
      c[k] = ew_d(w);
    }
    if (!ok) {
      const float nan = __int_as_float(0x7fc00000);
      qd.dist[j] = nan;
      qd.grad[3 * (size_t)j] = nan;
      qd.grad[3 * (size_t)j + 1] = nan;
      qd.grad[3 * (size_t)j + 2] = nan;
      qd.status[j] = 1;
      continue;
    }
    // c[k] with k = 4*bx + 2*by + bz; interpolate along z, then y, then x
    const float fx = f[0], fy = f[1], fz = f[2];
    const float gx0 = 1.0f - fx, gy0 = 1.0f - fy, gz0 = 1.0f - fz;
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
    qd.dist[j] = d;
    qd.grad[3 * (size_t)j] = ddx * inv_v;
    qd.grad[3 * (size_t)j + 1] = ddy * inv_v;
    qd.grad[3 * (size_t)j + 2] = ddz * inv_v;
    qd.status[j] = 0;
  }
}

}  // namespace

cudaError_t launch_query(const Batch& b, unsigned max_total, const LaunchCfg& cfg, LaunchHook* hook) {
  if (max_total == 0) return cudaSuccess;
  long long g = ((long long)max_total + kThreads - 1) / kThreads;
  const long long cap = (long long)cfg.num_sms * 16;
  if (g > cap) g = cap;
  hook->begin(kKQuery, cfg.stream);
  k_query<<<(int)g, kThreads, 0, cfg.stream>>>(b);
  hook->end(kKQuery, cfg.stream);
  return cudaGetLastError();
}

}  // namespace vbx
