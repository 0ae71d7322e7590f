// Host check of the ray-segment seek of the traversal (DdaSeg in vbx_internal.cuh): for random
// rays, the state that seek() computes for each segment start must equal the state that plain
// stepping reaches at that cut, and the segments' cells must cover the ray's cells exactly once.
// Prints "ok <rays> <segments>" or the first mismatch; exit status 0 on success.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "vbx_internal.cuh"

using vbx::Dda;
using vbx::DdaSeg;

static unsigned long long rng_state = 0x9e3779b97f4a7c15ull;
static unsigned long long next_u64() {  // splitmix64
  unsigned long long z = (rng_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static long long uniform(long long lo, long long hi) { return lo + (long long)(next_u64() % (unsigned long long)(hi - lo + 1)); }

static bool same(const Dda& a, const Dda& b) {
  return a.cx == b.cx && a.cy == b.cy && a.cz == b.cz && a.rx == b.rx && a.ry == b.ry && a.rz == b.rz && a.cxy == b.cxy &&
         a.cxz == b.cxz && a.cyz == b.cyz;
}

int main() {
  const int Ks[] = {1, 2, 3, 4, 16};
  long long nseg_total = 0;
  int nrays = 0;
  for (int trial = 0; trial < 20000; ++trial) {
    const int log2F = (trial & 1) ? 16 : 19;  // voxel cells, 8-voxel block cells
    long long S[3], E[3];
    const int kind = trial % 5;
    for (int a = 0; a < 3; ++a) {
      S[a] = uniform(-(1ll << 36), 1ll << 36);
      // ray lengths up to 2^14 voxels per axis (the traversal's range bound)
      long long span = kind == 0 ? 40 : (kind == 1 ? 1000 : 16384);
      long long dlt = uniform(-span * 65536, span * 65536);
      if (kind == 3 && a != 0) dlt = 0;                       // axis-aligned rays
      if (kind == 4) dlt = (a == 0 ? 1 : (a == 1 ? -1 : 1)) * uniform(0, 300) * 65536;  // exact diagonals: ties
      if (kind == 4) S[a] = (S[a] >> 16) << 16;
      E[a] = S[a] + dlt;
    }
    DdaSeg sg;
    sg.init(S, E, log2F);
    // plain stepping: state at every step index, and the axis of each step
    std::vector<Dda> states;
    std::vector<int> axes;
    Dda q = sg.q0;
    states.push_back(q);
    for (int left = q.steps(); left > 0; --left) {
      axes.push_back(q.step());
      states.push_back(q);
    }
    const int N = (int)axes.size();
    for (int K : Ks) {
      // cut positions: the step index after the (s*K)-th crossing of the dominant axis
      std::vector<int> cut = {0};
      int dc = 0;
      for (int m = 0; m < N; ++m)
        if (axes[m] == sg.d && ++dc % K == 0) cut.push_back(m + 1);
      const int segs = sg.segments(K);
      if ((int)cut.size() != segs) {
        printf("segment count mismatch trial %d K %d: %d vs %d\n", trial, K, (int)cut.size(), segs);
        return 1;
      }
      int covered = 0;
      for (int s = 0; s < segs; ++s) {
        int left = 0;
        Dda z = sg.seek(s, K, &left);
        if (!same(z, states[cut[s]]) || left != N - cut[s]) {
          printf("seek mismatch trial %d K %d segment %d (log2F %d)\n", trial, K, s, log2F);
          return 1;
        }
        // walk the segment as the kernels do
        int cells = 1, dk = 0;
        while (left > 0) {
          const int ax = z.step();
          --left;
          if (ax == sg.d && ++dk == K) break;
          ++cells;
        }
        covered += cells;
      }
      if (covered != N + 1) {
        printf("coverage mismatch trial %d K %d: %d cells of %d\n", trial, K, covered, N + 1);
        return 1;
      }
      nseg_total += segs;
    }
    ++nrays;
  }
  printf("ok %d %lld\n", nrays, nseg_total);
  return 0;
}
