// vbx_oracle.cpp -- plain, slow, single-threaded CPU oracle of the Voxblox per-scan map
// update (Oleynikova et al., "Voxblox: Incremental 3D Euclidean Signed Distance Fields for
// On-Board MAV Planning", arXiv 1611.03631).
//
// TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark's CPU
// baseline leg load this library. The product path (the CUDA library) shares no code,
// header, table or helper with this file, and never calls it.
//
// What it computes, in the paper's order:
//   * Sec. IV-A, Eq. (1)-(4): projective distance d, constant / quadratic weight with the
//     linear drop-off behind the surface, and the weighted running-average merge of D, W.
//   * Sec. IV-B: raycasting from the sensor origin to truncation distance delta behind each
//     point, either per point (plain raycasting) or once per group of points that fall into
//     the same voxel (grouped raycasting, weighted mean position, summed weight).
//   * Sec. III: a map of fixed-size voxel blocks indexed by integer block position through a
//     hash table (std::unordered_map here).
//   * Sec. V-A, Algorithm 1: incremental ESDF update from the updated TSDF voxels with a fixed
//     band |D| < gamma, a raise wavefront and a lower wavefront over 26-connected neighbours
//     with quasi-Euclidean step lengths v, v*sqrt(2), v*sqrt(3); the open set is processed
//     either by a priority queue keyed by |d| or by a FIFO queue (both are in Sec. V-A).
//   * A full (batch) recompute of the same distance field by multi-source Dijkstra, the
//     comparison point of Sec. VI-B; used as an invariant: incremental == batch.
//   * Trilinear interpolation of the distance field and its analytic gradient, the query
//     the paper's trajectory optimiser consumes (Sec. VI-A uses trilinear interpolation).
//
// Readings where the paper is silent or its Algorithm 1 is inconsistent (each is listed in
// the design notes of the repository):
//   R1 grouping arithmetic: key = floor(p/v) per axis from the float32 quotient q = p/v; the
//      sub-voxel offset o = rint((q - floor(q)) * 65536) clamped to 65535; per-point weight
//      w_q = rint(w * 2^20) as an integer (1 for constant weight); the group mean offset is
//      (sum w_q o + floor(sum w_q / 2)) div sum w_q, exact in integers; the group position is
//      fl(fl(key + m * 2^-16) * v); the group weight is the point count (constant weight) or
//      fl(sum w_q) * 2^-20 (quadratic weight).
//   R2 ray extent: from the sensor origin s to e = pbar + delta * u, u = (pbar - s)/|pbar - s|;
//      both ends quantised to 1/65536 voxel: llrint(fl(x / v) * 65536).
//   R3 voxel traversal: exact integer 3-D DDA (6-connected); at equal crossing parameters the
//      x step is taken first, then y, then z; a coordinate exactly on a face belongs to the
//      voxel on its + side (floor).
//   R4 allocation: every block containing a traversed voxel is allocated.
//   R5 per-voxel update: x = voxel centre fl(fl(i + 0.5) * v); d per Eq. (1) in float32 with
//      sign(0) = +1, clamped to [-delta, delta]; w per Eq. (2) or Eq. (4), where d <= -delta
//      gives w = 0 and the record is dropped; sums over one scan in float64; the merge of
//      Eq. (3) is applied once per scan per voxel with the summed weight (order-independent);
//      W is capped at W_max; a voxel is "updated" by a scan iff it received a record.
//   R6 ESDF classification (Algorithm 1, first loop): isFixed is evaluated on the TSDF voxel,
//      fixed iff |fl32(D)| < gamma; its comparison of the ESDF and TSDF distances is read as a
//      magnitude comparison in the same sign; the "fixed" flag is set in the fixed branch and
//      cleared where the voxel
//      leaves the band; a non-fixed observed voxel whose TSDF sign flipped is raised like a
//      voxel leaving the band.
//   R7 raise: only non-fixed voxels are reset; a neighbour is a child iff its parent
//      direction points at the popped voxel; only observed voxels are ever queued.
//   R8 lower: only observed, non-fixed neighbours of the same sign are relaxed, by magnitude:
//      cand = |d_v| + L_k, accepted iff cand < |d_n|; values never exceed d_max.
//   R9 query: the 8 voxel centres around q are selected in float32 (t = fl(fl(q/v) - 0.5),
//      i0 = floor(t), f = t - i0); any unobserved corner gives status "unknown".
//   R10 the one-voxel fixed band that Sec. VI-B and VIII recommend has no stated value:
//      gamma = v unless given; the half-truncation band of Sec. VI-B is |D| < delta / 2.
//   R11 Sec. VI-B compares the fixed band with an occupancy ESDF that treats negative TSDF
//      voxels as occupied at distance 0: in that mode (esdf_mode = 1) the seeds are the
//      observed voxels with fl32(D) < 0, fixed at +0, and every other observed voxel is
//      positive, so the field is the unsigned quasi-Euclidean distance to occupied voxels.
//   R12 mesh layer (Sec. III names meshes as a layer built from the TSDF, for display, but
//      gives no algorithm): marching cells over each cube of 8 observed voxel centres, inside
//      iff fl32(D) < 0, float32 edge interpolation, ambiguous faces resolved by cutting off
//      each inside corner, loops longer than 3 fanned around their centroid, normals towards
//      positive D; triangles keyed by (cell min corner, index in cell). See mesh_cell.
//   R13 full Euclidean variant (Sec. V-A says only that the parent then holds the full offset):
//      a voxel keeps the offset to its site (a fixed voxel); a site offers |d_s| + v * ||n - s||;
//      a fixed voxel whose value changes, or that leaves the band, is raised, and a voxel is its
//      child iff it is measured to it. See update_esdf_euclidean.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <deque>
#include <functional>
#include <queue>
#include <unordered_map>
#include <vector>

namespace {

constexpr int kNoParent = 255;
constexpr int64_t kSub = 65536;  // fixed-point sub-voxel resolution of R1 / R2

struct Key3 {
  int32_t x, y, z;
  bool operator==(const Key3& o) const { return x == o.x && y == o.y && z == o.z; }
  bool operator<(const Key3& o) const {
    if (x != o.x) return x < o.x;
    if (y != o.y) return y < o.y;
    return z < o.z;
  }
};

struct Key3Hash {
  size_t operator()(const Key3& k) const {
    uint64_t h = (uint64_t)(uint32_t)k.x * 73856093ull;
    h ^= (uint64_t)(uint32_t)k.y * 19349669ull;
    h ^= (uint64_t)(uint32_t)k.z * 83492791ull;
    return (size_t)h;
  }
};

int32_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return (int32_t)q;
}

struct TsdfVoxel {
  double D = 0.0;
  double W = 0.0;
};

struct EsdfVoxel {
  double d = 0.0;
  int parent = kNoParent;
  bool observed = false;
  bool fixed = false;
  // Euclidean variant (R13): the fixed voxel ("site") this voxel's distance is measured to
  bool has_site = false;
  int32_t site[3] = {0, 0, 0};
};

struct Block {
  std::vector<TsdfVoxel> tsdf;
  std::vector<EsdfVoxel> esdf;
};

struct Params {
  float v;
  int B;
  float delta;
  float dmax;
  int weighting;  // 0 constant (Eq. 2), 1 quadratic with drop-off (Eq. 4)
  float eps;
  float gamma;
  float wmax;
  float max_range;
  int grouped;
  int esdf_fp32;  // 1: ESDF values computed in float32 (bit-exact mode), 0: float64
  int esdf_mode;  // 0: fixed band |D| < gamma (Sec. V-A); 1: occupancy (R11, Sec. VI-B)
  int euclidean;  // 1: full Euclidean distance through stored sites (Sec. V-A, R13)
};

// 26-neighbourhood; index k = (dx+1)*9 + (dy+1)*3 + (dz+1); 13 is the voxel itself, and the
// opposite direction of k is 26 - k.
struct Nbr {
  int dx, dy, dz;
};

Nbr nbr(int k) { return Nbr{k / 9 - 1, (k / 3) % 3 - 1, k % 3 - 1}; }

struct Stats {
  int64_t points_in = 0, points_valid = 0, groups = 0, records = 0, updated = 0, new_blocks = 0;
  int64_t esdf_updated_in = 0, seeds = 0, raise_pops = 0, lower_pops = 0, lower_improve = 0;
};

struct Map {
  Params p;
  std::unordered_map<Key3, Block, Key3Hash> blocks;
  std::vector<Key3> last_updated;  // voxels updated by the last scan
  std::vector<Key3> dirty;         // voxels updated since the last ESDF update
  std::unordered_map<Key3, char, Key3Hash> dirty_set;
  // Euclidean variant: the voxels that took each site (entries of voxels that later took another
  // site are stale and skipped where the list is read)
  std::unordered_map<Key3, std::vector<Key3>, Key3Hash> site_takers;
  Stats st;

  int B3() const { return p.B * p.B * p.B; }

  Block& block_for(const Key3& bk, bool* created) {
    auto it = blocks.find(bk);
    if (it != blocks.end()) {
      if (created) *created = false;
      return it->second;
    }
    Block b;
    b.tsdf.assign(B3(), TsdfVoxel{});
    b.esdf.assign(B3(), EsdfVoxel{});
    if (created) *created = true;
    return blocks.emplace(bk, std::move(b)).first->second;
  }

  Key3 block_of(const Key3& c) const {
    return Key3{floor_div(c.x, p.B), floor_div(c.y, p.B), floor_div(c.z, p.B)};
  }
  int local_of(const Key3& c) const {
    int lx = c.x - floor_div(c.x, p.B) * p.B;
    int ly = c.y - floor_div(c.y, p.B) * p.B;
    int lz = c.z - floor_div(c.z, p.B) * p.B;
    return (lz * p.B + ly) * p.B + lx;
  }
  TsdfVoxel* tsdf_at(const Key3& c) {
    auto it = blocks.find(block_of(c));
    if (it == blocks.end()) return nullptr;
    return &it->second.tsdf[local_of(c)];
  }
  EsdfVoxel* esdf_at(const Key3& c) {
    auto it = blocks.find(block_of(c));
    if (it == blocks.end()) return nullptr;
    return &it->second.esdf[local_of(c)];
  }
};

// ------------------------------------------------------------------------------------------
// Sec. IV-B / R3: the voxels a segment from S to E (fixed point, kSub units per voxel) passes.
// At every step the axis whose next face crossing has the smallest parameter t is stepped;
// t of axis a is num_a / den_a and the comparison is done on cross products (exact).
void traverse(const int64_t S[3], const int64_t E[3], std::vector<Key3>* out) {
  int32_t c[3], end[3];
  int64_t den[3];
  int step[3];
  int64_t remaining[3];
  for (int a = 0; a < 3; ++a) {
    c[a] = floor_div(S[a], kSub);
    end[a] = floor_div(E[a], kSub);
    den[a] = E[a] >= S[a] ? E[a] - S[a] : S[a] - E[a];
    step[a] = E[a] >= S[a] ? 1 : -1;
    remaining[a] = end[a] >= c[a] ? (int64_t)end[a] - c[a] : (int64_t)c[a] - end[a];
  }
  out->push_back(Key3{c[0], c[1], c[2]});
  while (remaining[0] + remaining[1] + remaining[2] > 0) {
    int best = -1;
    __int128 best_num = 0, best_den = 1;
    for (int a = 0; a < 3; ++a) {
      if (remaining[a] == 0) continue;
      int64_t num = step[a] > 0 ? (int64_t)(c[a] + 1) * kSub - S[a] : S[a] - (int64_t)c[a] * kSub;
      // t_a = num / den[a]; pick strictly smaller t, so ties keep the earlier axis (x, y, z).
      if (best < 0 || (__int128)num * best_den < best_num * (__int128)den[a]) {
        best = a;
        best_num = num;
        best_den = den[a];
      }
    }
    c[best] += step[best];
    remaining[best] -= 1;
    out->push_back(Key3{c[0], c[1], c[2]});
  }
}

struct Group {
  int64_t n = 0;
  int64_t sw = 0;          // sum of integer weights w_q
  __int128 swo[3] = {0, 0, 0};  // sum of w_q * o_q per axis
};

struct Ray {
  float pbar[3];
  float Wg;
};

// Eq. (1) with R5: the projective distance of voxel centre x for a ray s -> pbar, clamped.
float projective_distance(const float pbar[3], const float s[3], const Key3& c, float v, float delta) {
  float x[3] = {((float)c.x + 0.5f) * v, ((float)c.y + 0.5f) * v, ((float)c.z + 0.5f) * v};
  float dx = pbar[0] - x[0], dy = pbar[1] - x[1], dz = pbar[2] - x[2];
  float gx = pbar[0] - s[0], gy = pbar[1] - s[1], gz = pbar[2] - s[2];
  float dist = std::sqrt((dx * dx + dy * dy) + dz * dz);
  float dot = (dx * gx + dy * gy) + dz * gz;
  float d = dot >= 0.0f ? dist : -dist;
  if (d > delta) d = delta;
  if (d < -delta) d = -delta;
  return d;
}

// Eq. (2) / Eq. (4): the weight of one record; W_g already carries the 1/z^2 factor.
float record_weight(const Params& p, float Wg, float d) {
  if (p.weighting == 0) return Wg;
  if (d <= -p.delta) return 0.0f;
  if (d < -p.eps) return Wg * ((d + p.delta) / (p.delta - p.eps));
  return Wg;
}

// A1: sensor-to-world transform of one point in float32, fixed operation order.
void transform_point(const float T[16], const float ps[3], float pw[3]) {
  for (int r = 0; r < 3; ++r) pw[r] = ((T[4 * r + 0] * ps[0] + T[4 * r + 1] * ps[1]) + T[4 * r + 2] * ps[2]) + T[4 * r + 3];
}

// A1 filter + per-point weight (R1). Returns false when the point is dropped.
bool accept_point(const Params& p, const float ps[3], float* w) {
  if (!std::isfinite(ps[0]) || !std::isfinite(ps[1]) || !std::isfinite(ps[2])) return false;
  float r2 = (ps[0] * ps[0] + ps[1] * ps[1]) + ps[2] * ps[2];
  if (!(r2 > 0.0f)) return false;
  // R1: points farther than 2^14 voxels from the sensor are dropped (bounds the ray length).
  const float lim = 16384.0f * p.v;
  if (!(r2 < lim * lim)) return false;
  if (std::isfinite(p.max_range) && p.max_range > 0.0f && r2 > p.max_range * p.max_range) return false;
  if (p.weighting == 1) {
    // Eq. (4): 1/z^2 with z the depth of the measurement in the sensor frame.
    if (!(ps[2] > 0.0f)) return false;
    float wi = 1.0f / (ps[2] * ps[2]);
    if (!(wi <= 1024.0f)) return false;
    *w = wi;
  } else {
    *w = 1.0f;
  }
  return true;
}

// A1 + A2 (R1): the rays of one scan. Grouped raycasting (Sec. IV-B) gives one ray per voxel
// that holds accepted points, at the weighted mean of its points with the summed weight;
// plain raycasting gives one ray per accepted point. Each ray comes with the voxel key of its
// group and the group's point count (per point: the point's own key, count 1). Returns the
// number of accepted points. Both integrate() and the grouping pin entry use this function.
struct ScanRay {
  Key3 key;
  Ray ray;
  int64_t count;
};

int64_t scan_rays(const Params& p, const float* pts, int64_t n, const float T[16], std::vector<ScanRay>* out) {
  int64_t valid = 0;
  std::unordered_map<Key3, Group, Key3Hash> groups;
  for (int64_t i = 0; i < n; ++i) {
    float w;
    if (!accept_point(p, pts + 3 * i, &w)) continue;
    float pw[3];
    transform_point(T, pts + 3 * i, pw);
    float q[3];
    bool in_range = true;
    for (int a = 0; a < 3; ++a) {
      q[a] = pw[a] / p.v;
      if (!(std::fabs(q[a]) < 1048576.0f)) in_range = false;  // |key| < 2^20
    }
    if (!in_range) continue;
    valid++;
    Key3 key{(int32_t)std::floor(q[0]), (int32_t)std::floor(q[1]), (int32_t)std::floor(q[2])};
    if (!p.grouped) {
      ScanRay r;
      r.key = key;
      for (int a = 0; a < 3; ++a) r.ray.pbar[a] = pw[a];
      r.ray.Wg = w;
      r.count = 1;
      out->push_back(r);
      continue;
    }
    int64_t wq = p.weighting == 0 ? 1 : (int64_t)std::llrint((double)w * 1048576.0);
    Group& g = groups[key];
    g.n += 1;
    g.sw += wq;
    for (int a = 0; a < 3; ++a) {
      float frac = q[a] - std::floor(q[a]);
      int64_t o = (int64_t)std::llrint(frac * 65536.0f);
      if (o > 65535) o = 65535;
      g.swo[a] += (__int128)wq * o;
    }
  }
  for (auto& kv : groups) {
    const Key3& key = kv.first;
    const Group& g = kv.second;
    ScanRay r;
    r.key = key;
    const int32_t kk[3] = {key.x, key.y, key.z};
    for (int a = 0; a < 3; ++a) {
      __int128 mnum = g.swo[a] + (__int128)(g.sw / 2);
      int64_t mo = (int64_t)(mnum / (__int128)g.sw);
      r.ray.pbar[a] = ((float)kk[a] + (float)mo * (1.0f / 65536.0f)) * p.v;
    }
    r.ray.Wg = p.weighting == 0 ? (float)g.n : (float)g.sw * (1.0f / 1048576.0f);
    r.count = g.n;
    out->push_back(r);
  }
  return valid;
}

void integrate(Map& m, const float* pts, int64_t n, const float T[16]) {
  const Params& p = m.p;
  m.st = Stats{};
  m.st.points_in = n;
  const float s[3] = {T[3], T[7], T[11]};

  // Rays: grouped (one per voxel containing points) or one per point.
  std::vector<ScanRay> srays;
  m.st.points_valid = scan_rays(p, pts, n, T, &srays);
  std::vector<Ray> rays;
  rays.reserve(srays.size());
  for (const ScanRay& r : srays) rays.push_back(r.ray);
  m.st.groups = (int64_t)rays.size();

  // Raycasting (Sec. IV-B) and per-voxel accumulation (Eq. 3 summed over the scan).
  struct Acc {
    double sw = 0.0, swd = 0.0;
  };
  std::unordered_map<Key3, Acc, Key3Hash> acc;
  std::vector<Key3> visited;
  for (const Ray& r : rays) {
    float g[3] = {r.pbar[0] - s[0], r.pbar[1] - s[1], r.pbar[2] - s[2]};
    float len = std::sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
    if (!(len > 0.0f)) continue;
    int64_t S[3], E[3];
    for (int a = 0; a < 3; ++a) {
      float u = g[a] / len;
      float e = r.pbar[a] + p.delta * u;
      S[a] = (int64_t)std::llrint((s[a] / p.v) * 65536.0f);
      E[a] = (int64_t)std::llrint((e / p.v) * 65536.0f);
    }
    visited.clear();
    traverse(S, E, &visited);
    for (const Key3& c : visited) {
      bool created = false;
      m.block_for(m.block_of(c), &created);
      if (created) m.st.new_blocks++;
      float d = projective_distance(r.pbar, s, c, p.v, p.delta);
      float w = record_weight(p, r.Wg, d);
      if (!(w > 0.0f)) continue;
      m.st.records++;
      Acc& a = acc[c];
      a.sw += (double)w;
      a.swd += (double)w * (double)d;
    }
  }

  // Eq. (3): merge, once per voxel per scan.
  m.last_updated.clear();
  for (auto& kv : acc) {
    TsdfVoxel* t = m.tsdf_at(kv.first);
    double W = t->W, D = t->D;
    t->D = (W * D + kv.second.swd) / (W + kv.second.sw);
    t->W = std::min(W + kv.second.sw, (double)p.wmax);
    m.last_updated.push_back(kv.first);
    if (!m.dirty_set.count(kv.first)) {
      m.dirty_set[kv.first] = 1;
      m.dirty.push_back(kv.first);
    }
  }
  std::sort(m.last_updated.begin(), m.last_updated.end());
  m.st.updated = (int64_t)m.last_updated.size();
}

// ------------------------------------------------------------------------------------------
// Sec. V-A, Algorithm 1 with readings R6-R8.

struct LowerItem {
  double key;
  uint64_t seq;
  Key3 c;
  bool operator>(const LowerItem& o) const { return key != o.key ? key > o.key : seq > o.seq; }
};

double sgn(double d) { return d >= 0.0 ? 1.0 : -1.0; }

double step_len(const Params& p, int k) {
  Nbr o = nbr(k);
  int n1 = (o.dx != 0) + (o.dy != 0) + (o.dz != 0);
  if (p.esdf_fp32) {
    const float L1 = p.v, L2 = p.v * 1.41421356237309515f, L3 = p.v * 1.73205080756887719f;
    return n1 == 1 ? L1 : (n1 == 2 ? L2 : L3);
  }
  const double v = p.v;
  return n1 == 1 ? v : (n1 == 2 ? v * std::sqrt(2.0) : v * std::sqrt(3.0));
}

double add_len(const Params& p, double a, double L) {
  if (p.esdf_fp32) return (double)((float)a + (float)L);
  return a + L;
}

// Seed value of a fixed voxel: the TSDF distance (float32 in the bit-exact mode).
double seed_value(const Params& p, double D) {
  float Df = (float)D;
  if (Df == 0.0f) Df = 0.0f;  // sign(0) = +1
  if (p.esdf_fp32) return (double)Df;
  if (Df == 0.0f) return 0.0;
  return D;
}

void update_esdf_euclidean(Map& m, int fifo);

void update_esdf(Map& m, int fifo) {
  if (m.p.euclidean) {
    update_esdf_euclidean(m, fifo);
    return;
  }
  const Params& p = m.p;
  const double dmax = p.esdf_fp32 ? (double)p.dmax : (double)p.dmax;
  std::deque<Key3> raise;
  std::priority_queue<LowerItem, std::vector<LowerItem>, std::greater<LowerItem>> lower_pq;
  std::deque<Key3> lower_fifo;
  uint64_t seq = 0;
  auto push_lower = [&](const Key3& c, double d) {
    if (fifo)
      lower_fifo.push_back(c);
    else
      lower_pq.push(LowerItem{std::fabs(d), seq++, c});
  };
  m.st.esdf_updated_in = (int64_t)m.dirty.size();
  m.st.seeds = m.st.raise_pops = m.st.lower_pops = m.st.lower_improve = 0;

  // First loop of Algorithm 1 over the TSDF voxels updated since the last call.
  std::vector<Key3> work = m.dirty;
  std::sort(work.begin(), work.end());
  for (const Key3& c : work) {
    TsdfVoxel* t = m.tsdf_at(c);
    EsdfVoxel* e = m.esdf_at(c);
    if (!t || !e || !(t->W > 0.0)) continue;
    float Df = (float)t->D;
    const bool occ = p.esdf_mode == 1;  // R11
    double sT = occ ? 1.0 : (Df >= 0.0f ? 1.0 : -1.0);
    bool fixed_now = occ ? Df < 0.0f : std::fabs(Df) < p.gamma;  // R6: isFixed on the TSDF voxel
    if (fixed_now) {
      m.st.seeds++;
      double val = occ ? 0.0 : seed_value(p, t->D);
      bool lower_only = !e->observed || (sgn(e->d) == sT && std::fabs(val) <= std::fabs(e->d));
      e->observed = true;
      e->fixed = true;
      e->d = val;
      e->parent = kNoParent;
      if (!lower_only) raise.push_back(c);
      push_lower(c, val);
    } else if (e->fixed) {  // leaves the band
      e->observed = true;
      e->fixed = false;
      e->d = sT * dmax;
      e->parent = kNoParent;
      raise.push_back(c);
    } else if (!e->observed) {  // new voxel: neighbours go to the lower queue
      e->observed = true;
      e->d = sT * dmax;
      e->parent = kNoParent;
      for (int k = 0; k < 27; ++k) {
        if (k == 13) continue;
        Nbr o = nbr(k);
        Key3 n{c.x + o.dx, c.y + o.dy, c.z + o.dz};
        EsdfVoxel* en = m.esdf_at(n);
        if (en && en->observed) push_lower(n, en->d);
      }
    } else if (sgn(e->d) != sT) {  // R6: sign flip of a non-fixed observed voxel
      e->d = sT * dmax;
      e->parent = kNoParent;
      raise.push_back(c);
    }
  }
  m.dirty.clear();
  m.dirty_set.clear();

  // Raise wavefront (R7).
  while (!raise.empty()) {
    Key3 c = raise.front();
    raise.pop_front();
    EsdfVoxel* e = m.esdf_at(c);
    m.st.raise_pops++;
    if (!e->fixed) {
      e->d = sgn(e->d) * dmax;
      e->parent = kNoParent;
    }
    for (int k = 0; k < 27; ++k) {
      if (k == 13) continue;
      Nbr o = nbr(k);
      Key3 n{c.x + o.dx, c.y + o.dy, c.z + o.dz};
      EsdfVoxel* en = m.esdf_at(n);
      if (!en || !en->observed) continue;
      // n's parent direction points from n back to c, i.e. the opposite of k.
      if (!en->fixed && en->parent == 26 - k)
        raise.push_back(n);
      else
        push_lower(n, en->d);
    }
  }

  // Lower wavefront (R8).
  while (fifo ? !lower_fifo.empty() : !lower_pq.empty()) {
    Key3 c;
    if (fifo) {
      c = lower_fifo.front();
      lower_fifo.pop_front();
    } else {
      c = lower_pq.top().c;
      lower_pq.pop();
    }
    EsdfVoxel* e = m.esdf_at(c);
    if (!e || !e->observed) continue;
    m.st.lower_pops++;
    double sv = sgn(e->d);
    double av = std::fabs(e->d);
    for (int k = 0; k < 27; ++k) {
      if (k == 13) continue;
      Nbr o = nbr(k);
      Key3 n{c.x + o.dx, c.y + o.dy, c.z + o.dz};
      EsdfVoxel* en = m.esdf_at(n);
      if (!en || !en->observed || en->fixed || sgn(en->d) != sv) continue;
      double cand = add_len(p, av, step_len(p, k));
      if (cand < std::fabs(en->d)) {
        en->d = sv * cand;
        en->parent = 26 - k;  // direction from n back to c
        m.st.lower_improve++;
        push_lower(n, en->d);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------
// Sec. V-A, full Euclidean variant: a voxel keeps the full offset to its site, the fixed voxel
// its distance is measured to, instead of the direction of the neighbour that lowered it. Reading
// R13 (the paper states only that the parent then holds the full offset):
//  * the distance a site s offers voxel n is |d_s| + v * ||n - s|| (float32 in the bit-exact
//    mode: |d_s| + fl(v * sqrt(fl(dx^2 + dy^2 + dz^2))), each operation rounded once);
//  * classification follows Algorithm 1 (R6), except that a fixed voxel whose value changes at
//    all is raised (voxels measured to it would otherwise keep a value computed from its old
//    value);
//  * raise: a voxel is a child of a raised site iff it is measured to that site (found here
//    through the list of voxels that took the site, each re-checked); children are reset to
//    +-d_max without a site, and the observed neighbours of every reset voxel and raised site
//    join the lower wave (this also reaches voxels whose chain of neighbours back to the site
//    was broken by later improvements along it);
//  * lower: the popped voxel offers its site (itself if fixed) to its observed, non-fixed,
//    same-sign neighbours; a neighbour takes it iff the offered distance is smaller than its own.

double euclid_offer(const Params& p, double dsite, const int32_t s[3], const Key3& n) {
  const int64_t dx = (int64_t)n.x - s[0], dy = (int64_t)n.y - s[1], dz = (int64_t)n.z - s[2];
  const int64_t q = dx * dx + dy * dy + dz * dz;
  if (p.esdf_fp32) {
    const float len = p.v * std::sqrt((float)q);
    return (double)(std::fabs((float)dsite) + len);
  }
  return std::fabs(dsite) + (double)p.v * std::sqrt((double)q);
}

void update_esdf_euclidean(Map& m, int fifo) {
  const Params& p = m.p;
  const double dmax = (double)p.dmax;
  std::vector<Key3> raised;  // sites whose value changed or that left the band
  std::priority_queue<LowerItem, std::vector<LowerItem>, std::greater<LowerItem>> lower_pq;
  std::deque<Key3> lower_fifo;
  uint64_t seq = 0;
  auto push_lower = [&](const Key3& c, double d) {
    if (fifo)
      lower_fifo.push_back(c);
    else
      lower_pq.push(LowerItem{std::fabs(d), seq++, c});
  };
  auto push_observed_neighbours = [&](const Key3& c) {
    for (int k = 0; k < 27; ++k) {
      if (k == 13) continue;
      Nbr o = nbr(k);
      Key3 n{c.x + o.dx, c.y + o.dy, c.z + o.dz};
      EsdfVoxel* en = m.esdf_at(n);
      if (en && en->observed) push_lower(n, en->d);
    }
  };
  m.st.esdf_updated_in = (int64_t)m.dirty.size();
  m.st.seeds = m.st.raise_pops = m.st.lower_pops = m.st.lower_improve = 0;

  // Classification (first loop of Algorithm 1, R6 and R13).
  std::vector<Key3> work = m.dirty;
  std::sort(work.begin(), work.end());
  for (const Key3& c : work) {
    TsdfVoxel* t = m.tsdf_at(c);
    EsdfVoxel* e = m.esdf_at(c);
    if (!t || !e || !(t->W > 0.0)) continue;
    float Df = (float)t->D;
    const bool occ = p.esdf_mode == 1;
    double sT = occ ? 1.0 : (Df >= 0.0f ? 1.0 : -1.0);
    bool fixed_now = occ ? Df < 0.0f : std::fabs(Df) < p.gamma;
    if (fixed_now) {
      m.st.seeds++;
      double val = occ ? 0.0 : seed_value(p, t->D);
      if (e->observed && e->fixed && e->d != val) raised.push_back(c);
      e->observed = true;
      e->fixed = true;
      e->d = val;
      e->has_site = false;
      push_lower(c, val);
    } else if (e->fixed) {  // leaves the band: its dependants are raised
      e->fixed = false;
      e->d = sT * dmax;
      e->has_site = false;
      raised.push_back(c);
    } else if (!e->observed) {  // new voxel: its observed neighbours offer their sites
      e->observed = true;
      e->d = sT * dmax;
      e->has_site = false;
      push_observed_neighbours(c);
    } else if (sgn(e->d) != sT) {  // sign flip of a non-fixed voxel (nothing is measured to it)
      e->d = sT * dmax;
      e->has_site = false;
      push_observed_neighbours(c);
    }
  }
  m.dirty.clear();
  m.dirty_set.clear();

  // Raise (R13): reset every voxel measured to a raised site.
  for (const Key3& r : raised) {
    m.st.raise_pops++;
    push_observed_neighbours(r);
    auto it = m.site_takers.find(r);
    if (it == m.site_takers.end()) continue;
    for (const Key3& n : it->second) {
      EsdfVoxel* en = m.esdf_at(n);
      if (!en || !en->observed || en->fixed || !en->has_site) continue;
      if (en->site[0] != r.x || en->site[1] != r.y || en->site[2] != r.z) continue;
      en->d = sgn(en->d) * dmax;
      en->has_site = false;
      m.st.raise_pops++;
      push_observed_neighbours(n);
    }
    m.site_takers.erase(it);
  }

  // Lower (R8 with R13): sites travel through observed, non-fixed, same-sign neighbours.
  while (fifo ? !lower_fifo.empty() : !lower_pq.empty()) {
    Key3 c;
    if (fifo) {
      c = lower_fifo.front();
      lower_fifo.pop_front();
    } else {
      c = lower_pq.top().c;
      lower_pq.pop();
    }
    EsdfVoxel* e = m.esdf_at(c);
    if (!e || !e->observed) continue;
    int32_t s[3];
    double dsite;
    if (e->fixed) {
      s[0] = c.x;
      s[1] = c.y;
      s[2] = c.z;
      dsite = e->d;
    } else if (e->has_site) {
      std::memcpy(s, e->site, sizeof(s));
      dsite = m.esdf_at(Key3{s[0], s[1], s[2]})->d;
    } else {
      continue;  // at d_max without a site: nothing to offer
    }
    m.st.lower_pops++;
    double sv = sgn(e->d);
    for (int k = 0; k < 27; ++k) {
      if (k == 13) continue;
      Nbr o = nbr(k);
      Key3 n{c.x + o.dx, c.y + o.dy, c.z + o.dz};
      EsdfVoxel* en = m.esdf_at(n);
      if (!en || !en->observed || en->fixed || sgn(en->d) != sv) continue;
      double cand = euclid_offer(p, dsite, s, n);
      if (cand < std::fabs(en->d)) {
        en->d = sv * cand;
        en->has_site = true;
        std::memcpy(en->site, s, sizeof(s));
        m.site_takers[Key3{s[0], s[1], s[2]}].push_back(n);
        m.st.lower_improve++;
        push_lower(n, en->d);
      }
    }
  }
}

// Batch recompute: multi-source Dijkstra over observed voxels (the invariant
// incremental == batch). Values of non-observed voxels are NaN.
void full_esdf(Map& m, std::vector<Key3>* keys_sorted, std::vector<double>* out) {
  const Params& p = m.p;
  const int B3 = m.B3();
  keys_sorted->clear();
  for (auto& kv : m.blocks) keys_sorted->push_back(kv.first);
  std::sort(keys_sorted->begin(), keys_sorted->end());
  std::unordered_map<Key3, size_t, Key3Hash> index;
  for (size_t i = 0; i < keys_sorted->size(); ++i) index[(*keys_sorted)[i]] = i;
  out->assign(keys_sorted->size() * (size_t)B3, std::nan(""));
  std::vector<double> dist(out->size(), (double)p.dmax);
  std::vector<signed char> sign(out->size(), 0);
  std::vector<char> fixed(out->size(), 0), observed(out->size(), 0), done(out->size(), 0);
  auto flat = [&](const Key3& c, size_t* f) -> bool {
    auto it = index.find(m.block_of(c));
    if (it == index.end()) return false;
    *f = it->second * (size_t)B3 + (size_t)m.local_of(c);
    return true;
  };
  std::priority_queue<std::pair<double, size_t>, std::vector<std::pair<double, size_t>>, std::greater<>> pq;
  std::vector<Key3> coord(out->size());
  for (size_t b = 0; b < keys_sorted->size(); ++b) {
    const Key3& bk = (*keys_sorted)[b];
    const Block& blk = m.blocks[bk];
    for (int l = 0; l < B3; ++l) {
      size_t f = b * (size_t)B3 + l;
      int lx = l % p.B, ly = (l / p.B) % p.B, lz = l / (p.B * p.B);
      coord[f] = Key3{bk.x * p.B + lx, bk.y * p.B + ly, bk.z * p.B + lz};
      const TsdfVoxel& t = blk.tsdf[l];
      if (!(t.W > 0.0)) continue;
      observed[f] = 1;
      float Df = (float)t.D;
      const bool occ = p.esdf_mode == 1;  // R11
      sign[f] = occ || Df >= 0.0f ? 1 : -1;
      if (occ ? Df < 0.0f : std::fabs(Df) < p.gamma) {
        fixed[f] = 1;
        dist[f] = occ ? 0.0 : std::fabs(seed_value(p, t.D));
        pq.push({dist[f], f});
      }
    }
  }
  while (!pq.empty()) {
    auto top = pq.top();
    pq.pop();
    size_t f = top.second;
    if (done[f] || top.first != dist[f]) continue;
    done[f] = 1;
    const Key3& c = coord[f];
    for (int k = 0; k < 27; ++k) {
      if (k == 13) continue;
      Nbr o = nbr(k);
      size_t g;
      if (!flat(Key3{c.x + o.dx, c.y + o.dy, c.z + o.dz}, &g)) continue;
      if (!observed[g] || fixed[g] || sign[g] != sign[f]) continue;
      double cand = add_len(p, dist[f], step_len(p, k));
      if (cand < dist[g]) {
        dist[g] = cand;
        pq.push({cand, g});
      }
    }
  }
  for (size_t f = 0; f < out->size(); ++f)
    if (observed[f]) (*out)[f] = (double)sign[f] * dist[f];
}

// R9: trilinear interpolation of the distance field and its gradient.
void query(Map& m, const float* q, int64_t n, double* dist, double* grad, uint8_t* status) {
  const Params& p = m.p;
  for (int64_t i = 0; i < n; ++i) {
    int32_t i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
      float t = q[3 * i + a] / p.v - 0.5f;
      float fl = std::floor(t);
      i0[a] = (int32_t)fl;
      f[a] = (double)(t - fl);
    }
    double c[2][2][2];
    bool ok = true;
    for (int bx = 0; bx < 2 && ok; ++bx)
      for (int by = 0; by < 2 && ok; ++by)
        for (int bz = 0; bz < 2 && ok; ++bz) {
          EsdfVoxel* e = m.esdf_at(Key3{i0[0] + bx, i0[1] + by, i0[2] + bz});
          if (!e || !e->observed) {
            ok = false;
            break;
          }
          c[bx][by][bz] = e->d;
        }
    if (!ok) {
      status[i] = 1;
      dist[i] = std::nan("");
      for (int a = 0; a < 3; ++a) grad[3 * i + a] = std::nan("");
      continue;
    }
    status[i] = 0;
    double d = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int bx = 0; bx < 2; ++bx)
      for (int by = 0; by < 2; ++by)
        for (int bz = 0; bz < 2; ++bz) {
          double wx = bx ? f[0] : 1.0 - f[0];
          double wy = by ? f[1] : 1.0 - f[1];
          double wz = bz ? f[2] : 1.0 - f[2];
          double val = c[bx][by][bz];
          d += wx * wy * wz * val;
          gx += (bx ? 1.0 : -1.0) * wy * wz * val;
          gy += (by ? 1.0 : -1.0) * wx * wz * val;
          gz += (bz ? 1.0 : -1.0) * wx * wy * val;
        }
    dist[i] = d;
    grad[3 * i + 0] = gx / p.v;
    grad[3 * i + 1] = gy / p.v;
    grad[3 * i + 2] = gz / p.v;
  }
}

}  // namespace

// ------------------------------------------------------------------------------------------
// Iso-surface of the TSDF (the mesh layer of Sec. III), reading R12: marching cells over every
// cube of 8 observed voxel centres, a corner being inside iff fl32(D) < 0. Each edge with a
// sign change carries the vertex pa + t (pb - pa), t = Da / (Da - Db) (float32). On each face
// (corners counter-clockwise seen from outside the cube) the edge crossings are joined by
// directed segments, each with the inside corners on its left: from the edge where the
// counter-clockwise walk leaves the inside to the edge where it enters it; a face with four
// crossings cuts off each inside corner by its own segment. Two cells sharing a face see it
// from opposite sides, so they make the same segments in opposite directions, and the surface
// is closed and consistently oriented. The segments chain into loops, each starting at its
// smallest edge, and each loop is emitted against its direction, so that triangle normals
// (b - a) x (c - a) point towards positive D. A loop of three vertices is one triangle, a
// longer one a fan of triangles
// around the float32 mean of its vertices (a fan from a loop vertex could put a triangle inside
// a cube face, where the neighbouring cell would put its mirror image).

// cube corners c = x + 2 y + 4 z; edges 0-3 along x, 4-7 along y, 8-11 along z
const int kCubeEdge[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
// faces x = 0, x = 1, y = 0, y = 1, z = 0, z = 1: corners counter-clockwise seen from outside
const int kCubeFace[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};

int edge_of(int a, int b) {
  for (int e = 0; e < 12; ++e)
    if ((kCubeEdge[e][0] == a && kCubeEdge[e][1] == b) || (kCubeEdge[e][0] == b && kCubeEdge[e][1] == a)) return e;
  return -1;
}

struct MeshTri {
  int32_t cell[4];  // min-corner voxel of the cell, triangle index within the cell
  float v[9];
};

// Triangles of one cell (corner values Dc, corner positions pc[8][3]); appends to out.
void mesh_cell(const float Dc[8], const float pc[8][3], const int32_t cell[3], std::vector<MeshTri>& out) {
  bool in[8];
  for (int c = 0; c < 8; ++c) in[c] = Dc[c] < 0.0f;
  float vx[12][3];
  bool cross[12];
  for (int e = 0; e < 12; ++e) {
    const int a = kCubeEdge[e][0], b = kCubeEdge[e][1];
    cross[e] = in[a] != in[b];
    if (cross[e]) {
      const float t = Dc[a] / (Dc[a] - Dc[b]);
      for (int k = 0; k < 3; ++k) vx[e][k] = pc[a][k] + t * (pc[b][k] - pc[a][k]);
    }
  }
  // directed segments: next[e] = the edge the surface boundary goes to from crossing edge e
  int next[12];
  for (int e = 0; e < 12; ++e) next[e] = -1;
  for (int f = 0; f < 6; ++f) {
    int fe[4];  // fe[i]: edge from corner i to corner i + 1 of the face
    for (int i = 0; i < 4; ++i) fe[i] = edge_of(kCubeFace[f][i], kCubeFace[f][(i + 1) % 4]);
    int n = 0;
    for (int i = 0; i < 4; ++i) n += cross[fe[i]] ? 1 : 0;
    for (int i = 0; i < 4; ++i) {
      const bool in_i = in[kCubeFace[f][i]], in_n = in[kCubeFace[f][(i + 1) % 4]];
      if (n == 4) {
        if (in_i) next[fe[i]] = fe[(i + 3) % 4];  // cut off inside corner i
      } else if (n == 2 && in_i && !in_n) {  // the walk leaves the inside at fe[i] ...
        int j = (i + 1) % 4;  // ... and enters it again at the next crossing
        while (!cross[fe[j]]) j = (j + 1) % 4;
        next[fe[i]] = fe[j];
      }
    }
  }
  bool used[12] = {false};
  int tri_in_cell = 0;
  auto emit = [&](const float* a, const float* b, const float* c) {
    MeshTri t;
    t.cell[0] = cell[0], t.cell[1] = cell[1], t.cell[2] = cell[2], t.cell[3] = tri_in_cell++;
    for (int q = 0; q < 3; ++q) t.v[q] = a[q], t.v[3 + q] = b[q], t.v[6 + q] = c[q];
    out.push_back(t);
  };
  for (int e0 = 0; e0 < 12; ++e0) {
    if (!cross[e0] || used[e0]) continue;
    int loop[12], k = 0;
    for (int e = e0; k < 12 && !used[e]; e = next[e]) {
      loop[k++] = e;
      used[e] = true;
    }
    if (k == 3) {
      emit(vx[loop[0]], vx[loop[2]], vx[loop[1]]);
    } else {  // a fan around the loop's centroid, which lies inside the cube
      float cen[3] = {0.0f, 0.0f, 0.0f};
      for (int i = 0; i < k; ++i)
        for (int a = 0; a < 3; ++a) cen[a] += vx[loop[i]][a];
      for (int a = 0; a < 3; ++a) cen[a] = cen[a] / (float)k;
      for (int i = 0; i < k; ++i) emit(cen, vx[loop[(i + 1) % k]], vx[loop[i]]);
    }
  }
}

std::vector<MeshTri> extract_mesh(Map& m) {
  const Params& p = m.p;
  std::vector<Key3> keys;
  for (auto& kv : m.blocks) keys.push_back(kv.first);
  std::sort(keys.begin(), keys.end());
  std::vector<MeshTri> out;
  const float v = p.v;
  for (const Key3& bk : keys) {
    for (int l = 0; l < m.B3(); ++l) {
      const Key3 c0{bk.x * p.B + l % p.B, bk.y * p.B + (l / p.B) % p.B, bk.z * p.B + l / (p.B * p.B)};
      float Dc[8], pc[8][3];
      bool ok = true;
      for (int c = 0; c < 8 && ok; ++c) {
        const Key3 q{c0.x + (c & 1), c0.y + ((c >> 1) & 1), c0.z + ((c >> 2) & 1)};
        TsdfVoxel* t = m.tsdf_at(q);
        if (!t || !(t->W > 0.0)) {
          ok = false;
          break;
        }
        Dc[c] = (float)t->D;
        const int32_t qi[3] = {q.x, q.y, q.z};
        for (int a = 0; a < 3; ++a) pc[c][a] = ((float)qi[a] + 0.5f) * v;  // voxel centre
      }
      if (!ok) continue;
      const int32_t cell[3] = {c0.x, c0.y, c0.z};
      mesh_cell(Dc, pc, cell, out);
    }
  }
  std::sort(out.begin(), out.end(), [](const MeshTri& a, const MeshTri& b) {
    return std::lexicographical_compare(a.cell, a.cell + 4, b.cell, b.cell + 4);
  });
  return out;
}

// ------------------------------------------------------------------------------------------
// C interface used by the tests (ctypes).

extern "C" {

struct orc_params {
  float voxel_size;
  int voxels_per_block;
  float truncation;
  float max_esdf_dist;
  int weighting;
  float eps;
  float fixed_band;
  float w_max;
  float max_range;
  int grouped;
  int esdf_fp32;
  int esdf_mode;
  int euclidean;
};

void* orc_create(const orc_params* op) {
  Map* m = new Map();
  m->p = Params{op->voxel_size, op->voxels_per_block, op->truncation, op->max_esdf_dist, op->weighting,
                op->eps,        op->fixed_band,       op->w_max,      op->max_range,     op->grouped,
                op->esdf_fp32,  op->esdf_mode,        op->euclidean};
  return m;
}

void orc_destroy(void* h) { delete (Map*)h; }

void orc_integrate(void* h, const float* pts, int64_t n, const float* T16) { integrate(*(Map*)h, pts, n, T16); }

void orc_update_esdf(void* h, int fifo) { update_esdf(*(Map*)h, fifo); }

// stats: points_in, points_valid, groups, records, updated, new_blocks, esdf_updated_in,
// seeds, raise_pops, lower_pops, lower_improve
void orc_stats(void* h, int64_t* out11) {
  const Stats& s = ((Map*)h)->st;
  int64_t v[11] = {s.points_in, s.points_valid, s.groups,     s.records,    s.updated,      s.new_blocks,
                   s.esdf_updated_in, s.seeds,  s.raise_pops, s.lower_pops, s.lower_improve};
  std::memcpy(out11, v, sizeof(v));
}

int64_t orc_num_blocks(void* h) { return (int64_t)((Map*)h)->blocks.size(); }

// Blocks sorted by key; per voxel (local index (lz*B+ly)*B+lx): D, W, d, parent, flags
// (bit0 observed, bit1 fixed).
void orc_export(void* h, int32_t* keys, double* D, double* W, double* d, uint8_t* parent, uint8_t* flags) {
  Map& m = *(Map*)h;
  std::vector<Key3> ks;
  for (auto& kv : m.blocks) ks.push_back(kv.first);
  std::sort(ks.begin(), ks.end());
  const int B3 = m.B3();
  for (size_t b = 0; b < ks.size(); ++b) {
    keys[3 * b + 0] = ks[b].x;
    keys[3 * b + 1] = ks[b].y;
    keys[3 * b + 2] = ks[b].z;
    const Block& blk = m.blocks[ks[b]];
    for (int l = 0; l < B3; ++l) {
      size_t f = b * (size_t)B3 + l;
      if (D) D[f] = blk.tsdf[l].D;
      if (W) W[f] = blk.tsdf[l].W;
      if (d) d[f] = blk.esdf[l].d;
      if (parent) parent[f] = (uint8_t)blk.esdf[l].parent;
      if (flags) flags[f] = (uint8_t)((blk.esdf[l].observed ? 1 : 0) | (blk.esdf[l].fixed ? 2 : 0));
    }
  }
}

int64_t orc_num_last_updated(void* h) { return (int64_t)((Map*)h)->last_updated.size(); }

void orc_last_updated(void* h, int32_t* out) {
  Map& m = *(Map*)h;
  for (size_t i = 0; i < m.last_updated.size(); ++i) {
    out[3 * i + 0] = m.last_updated[i].x;
    out[3 * i + 1] = m.last_updated[i].y;
    out[3 * i + 2] = m.last_updated[i].z;
  }
}

// Sites of the Euclidean variant in the block order of orc_export: offsets (site - voxel) as
// nb x B^3 x 3 int32 and a has-site flag per voxel.
void orc_export_sites(void* h, int32_t* offsets, uint8_t* has_site) {
  Map& m = *(Map*)h;
  std::vector<Key3> ks;
  for (auto& kv : m.blocks) ks.push_back(kv.first);
  std::sort(ks.begin(), ks.end());
  const int B = m.p.B, B3 = m.B3();
  for (size_t b = 0; b < ks.size(); ++b) {
    const Block& blk = m.blocks.at(ks[b]);
    for (int l = 0; l < B3; ++l) {
      const int x = ks[b].x * B + l % B, y = ks[b].y * B + (l / B) % B, z = ks[b].z * B + l / (B * B);
      const EsdfVoxel& e = blk.esdf[l];
      has_site[b * B3 + l] = e.has_site ? 1 : 0;
      int32_t* o = offsets + 3 * (b * B3 + l);
      o[0] = e.has_site ? e.site[0] - x : 0;
      o[1] = e.has_site ? e.site[1] - y : 0;
      o[2] = e.has_site ? e.site[2] - z : 0;
    }
  }
}

// Full recompute in the block order of orc_export.
void orc_full_esdf(void* h, double* out) {
  std::vector<Key3> ks;
  std::vector<double> d;
  full_esdf(*(Map*)h, &ks, &d);
  std::memcpy(out, d.data(), d.size() * sizeof(double));
}

void orc_query(void* h, const float* q, int64_t n, double* dist, double* grad, uint8_t* status) {
  query(*(Map*)h, q, n, dist, grad, status);
}

// Set TSDF voxels directly (voxel coordinates, D, W) and mark them updated, as if a scan
// had produced these values. Blocks are allocated as needed.
void orc_set_tsdf(void* h, const int32_t* vox, const double* D, const double* W, int64_t n) {
  Map& m = *(Map*)h;
  m.last_updated.clear();
  for (int64_t i = 0; i < n; ++i) {
    Key3 c{vox[3 * i], vox[3 * i + 1], vox[3 * i + 2]};
    m.block_for(m.block_of(c), nullptr);
    TsdfVoxel* t = m.tsdf_at(c);
    t->D = D[i];
    t->W = W[i];
    m.last_updated.push_back(c);
    if (!m.dirty_set.count(c)) {
      m.dirty_set[c] = 1;
      m.dirty.push_back(c);
    }
  }
}

// Set ESDF voxels directly (for query tests): value, observed flag; the block is allocated.
void orc_set_esdf(void* h, const int32_t* vox, const double* d, const uint8_t* observed, int64_t n) {
  Map& m = *(Map*)h;
  for (int64_t i = 0; i < n; ++i) {
    Key3 c{vox[3 * i], vox[3 * i + 1], vox[3 * i + 2]};
    m.block_for(m.block_of(c), nullptr);
    EsdfVoxel* e = m.esdf_at(c);
    e->d = d[i];
    e->observed = observed[i] != 0;
  }
}

// Primitive entry points for the pins.
int64_t orc_traverse(const int64_t* S, const int64_t* E, int32_t* out, int64_t cap) {
  std::vector<Key3> v;
  traverse(S, E, &v);
  int64_t k = std::min<int64_t>(cap, (int64_t)v.size());
  for (int64_t i = 0; i < k; ++i) {
    out[3 * i] = v[i].x;
    out[3 * i + 1] = v[i].y;
    out[3 * i + 2] = v[i].z;
  }
  return (int64_t)v.size();
}

float orc_projective_distance(const float* pbar, const float* s, const int32_t* c, float v, float delta) {
  return projective_distance(pbar, s, Key3{c[0], c[1], c[2]}, v, delta);
}

float orc_record_weight(const orc_params* op, float Wg, float d) {
  Params p{op->voxel_size, op->voxels_per_block, op->truncation, op->max_esdf_dist, op->weighting, op->eps,
           op->fixed_band, op->w_max,            op->max_range,  op->grouped,       op->esdf_fp32, op->esdf_mode, op->euclidean};
  return record_weight(p, Wg, d);
}

// Grouping only (Sec. IV-B): returns the number of groups; writes key, pbar, W_g, count
// sorted by key. The groups come from scan_rays, the function integrate() casts its rays from.
int64_t orc_group(const orc_params* op, const float* pts, int64_t n, const float* T16, int32_t* keys, float* pbar,
                  float* Wg, int64_t* count, int64_t cap) {
  Params p{op->voxel_size, op->voxels_per_block, op->truncation, op->max_esdf_dist, op->weighting, op->eps,
           op->fixed_band, op->w_max,            op->max_range,  1,                 op->esdf_fp32, op->esdf_mode, op->euclidean};
  std::vector<ScanRay> gs;
  scan_rays(p, pts, n, T16, &gs);
  std::sort(gs.begin(), gs.end(), [](const ScanRay& a, const ScanRay& b) { return a.key < b.key; });
  int64_t k = std::min<int64_t>(cap, (int64_t)gs.size());
  for (int64_t i = 0; i < k; ++i) {
    keys[3 * i] = gs[i].key.x;
    keys[3 * i + 1] = gs[i].key.y;
    keys[3 * i + 2] = gs[i].key.z;
    for (int a = 0; a < 3; ++a) pbar[3 * i + a] = gs[i].ray.pbar[a];
    Wg[i] = gs[i].ray.Wg;
    count[i] = gs[i].count;
  }
  return (int64_t)gs.size();
}

// Mesh of the TSDF (R12): writes min(n, cap) triangles sorted by (cell, index in cell):
// cells cap x 4 int32 (cell min corner, index), verts cap x 9 float32; returns n.
int64_t orc_extract_mesh(void* h, int32_t* cells, float* verts, int64_t cap) {
  std::vector<MeshTri> tris = extract_mesh(*(Map*)h);
  const int64_t n = (int64_t)tris.size();
  for (int64_t i = 0; i < n && i < cap; ++i) {
    std::memcpy(cells + 4 * i, tris[i].cell, sizeof(tris[i].cell));
    std::memcpy(verts + 9 * i, tris[i].v, sizeof(tris[i].v));
  }
  return n;
}

}  // extern "C"
