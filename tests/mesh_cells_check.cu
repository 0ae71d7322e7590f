// Host check of the per-cell mesh code of the CUDA library (mesh_cells.cuh), compiled with nvcc
// as host code. Reads cells from stdin -- a count, then per cell its minimum-corner voxel
// (3 ints), the voxel size and its 8 corner values (float32 bit patterns in hex) -- and prints
// each cell's triangles as "cell index_in_cell" followed by the 9 vertex coordinates as float32
// bit patterns in hex.
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "mesh_cells.cuh"

static float from_bits(unsigned u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
static unsigned to_bits(float f) {
  unsigned u;
  std::memcpy(&u, &f, 4);
  return u;
}

int main() {
  long n = 0;
  if (std::scanf("%ld", &n) != 1) return 2;
  for (long i = 0; i < n; ++i) {
    int g[3];
    unsigned vb, db[8];
    if (std::scanf("%d %d %d %x", &g[0], &g[1], &g[2], &vb) != 4) return 2;
    for (int c = 0; c < 8; ++c)
      if (std::scanf("%x", &db[c]) != 1) return 2;
    const float v = from_bits(vb);
    float Dc[8];
    unsigned pattern = 0;
    for (int c = 0; c < 8; ++c) {
      Dc[c] = from_bits(db[c]);
      if (Dc[c] < 0.0f) pattern |= 1u << c;
    }
    const vbx::McLoops L = vbx::mc_cell_loops(pattern);
    auto D = [&](int c) { return Dc[c]; };
    auto P = [&](int c, int q) { return vbx::mc_mul(vbx::mc_add((float)(g[q] + ((c >> q) & 1)), 0.5f), v); };
    float tri[12][9];
    int emitted = 0;
    auto out = [&](int idx, int slot, const float* w) {
      for (int q = 0; q < 3; ++q) tri[idx][3 * slot + q] = w[q];
      if (idx + 1 > emitted) emitted = idx + 1;
    };
    vbx::mc_emit(L, D, P, out);
    for (int t = 0; t < emitted; ++t) {
      std::printf("%ld %d", i, t);
      for (int q = 0; q < 9; ++q) std::printf(" %08x", to_bits(tri[t][q]));
      std::printf("\n");
    }
    if (emitted != vbx::mc_triangles(L.meta)) {
      std::printf("count mismatch cell %ld: %d emitted, %d in table\n", i, emitted, vbx::mc_triangles(L.meta));
      return 1;
    }
  }
  return 0;
}
