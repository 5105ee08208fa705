// CPU oracle for hash-blocked TSDF fusion. TEST INFRASTRUCTURE ONLY.
//
// Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
// this library. It shares no code, header, constant or helper with the CUDA
// path. It is deliberately plain, single threaded and slow: it computes the
// *definition* of a fused frame, not the hashed/probed/atomic algorithm.
//
// What it computes (paper Section 2, "The workload"):
//   * The volume is a set of 8^3-voxel blocks (Section 2.1) holding, per voxel,
//     a truncated signed distance, a weight and three colour channels, stored as
//     weighted SUMS; the mean is recovered on read-out (Section 2.2, "sums rather
//     than running means").
//   * Integration walks the truncation band along each depth point's view ray
//     (Section 2 intro and Section 2.2 "Allocate"/"Update") and adds one
//     contribution per distinct voxel the walk selects, after the occlusion test
//     that both passes share (Section 2.2, last paragraph).
//   * The signed distance is evaluated at the voxel CENTRE, not at the ray sample
//     that selected the voxel (Section 4.1, the half-voxel bias).
//   * Blocks are created for every block a contribution lands in; the hash table,
//     probing and compare-exchange of Listing 1 only decide *where* a block lives,
//     never *whether*, so the oracle uses an ordered map keyed by block
//     coordinate instead. Pool exhaustion is reported, never silent (Section 3.4,
//     "pool-exhaustion reporting"; Section 7.2 on silent loss).
//
// Readings where the paper is silent (each is also listed in the design notes):
//   R1 band walk: 2M+1 samples at range offsets t_k = (k-M) v, M = lrintf(tau/v),
//      along the unit view ray; each distinct voxel counted once per point.
//   R2 signed distance: sdf = d - z_c, the point's depth minus the camera-frame
//      depth of the voxel centre (projective distance, KinectFusion convention);
//      stored value tsdf = clamp(sdf / tau, -1, 1); weight 1 per contribution.
//   R3 occlusion test: the voxel centre must lie in front of the camera, project
//      (nearest pixel) inside the image onto a valid depth d', and be no more
//      than tau behind it: d' - z_c >= -tau.
//   R4 colour: the point's own pixel, 8-bit per channel, accumulated as c/255.
//   R5 single-precision decision arithmetic with a fixed operation order and
//      explicit fused multiply-adds (fmaf), so that every integer the geometry
//      decides (voxel index, pixel index, accept/reject) is reproducible
//      bit-for-bit by any IEEE-754 implementation of the same steps. The ray
//      is taken to the world frame once per point (P = R p + t, D = R d) and
//      sample k is P + t_k D; the voxel centre reaches the camera frame by one
//      per-frame affine map of the integer voxel, c = A g + b with A = v R^T
//      and b = R^T (v/2 - t).
//   R6 block coordinates must fit the 21-bit biased key (|b| < 2^20); voxels
//      outside are rejected and counted.
// Sums of tsdf and colour are accumulated in double (the reference value);
// weights are integers.
//
// Build: g++ -O2 -ffp-contract=off -fno-fast-math -std=c++17 -shared -fPIC
// (contraction must be off: the order of every rounding is part of R5).

#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>

namespace {

constexpr int kEdge = 8;            // Section 2.1: blocks of 8^3 voxels
constexpr int kVox = kEdge * kEdge * kEdge;

enum OracleStatus {
  OR_OK = 0,
  OR_INVALID_ARG = 1,
  OR_POOL_FULL = 3,
  OR_TABLE_FULL = 4,
  OR_POISONED = 7,
};

struct BlockData {
  std::array<double, kVox> tsdf_sum{};
  std::array<double, kVox> r_sum{}, g_sum{}, b_sum{};
  std::array<uint32_t, kVox> weight{};
};

struct Coord {
  int32_t x, y, z;
  bool operator<(const Coord& o) const {
    if (x != o.x) return x < o.x;
    if (y != o.y) return y < o.y;
    return z < o.z;
  }
  bool operator==(const Coord& o) const { return x == o.x && y == o.y && z == o.z; }
};

struct Volume {
  float voxel;
  float trunc;
  uint32_t slots;
  uint32_t pool;
  bool poisoned = false;
  uint64_t claimed = 0;  // distinct blocks ever requested (may exceed pool)
  std::map<Coord, BlockData> blocks;
};

// floor division by 8 for negative coordinates too
int32_t floor_div8(int32_t g) { return (g >= 0) ? g / kEdge : -((-g + kEdge - 1) / kEdge); }
int32_t floor_mod8(int32_t g) { return g - floor_div8(g) * kEdge; }

}  // namespace

extern "C" {

// Statistics of the last fused frame, in this order:
//  [0] valid points P            [1] walk samples taken
//  [2] accepted (point, voxel) contributions
//  [3] distinct voxels touched   [4] distinct blocks touched
//  [5] blocks created this frame [6] voxels rejected by the key range (R6)
//  [7] blocks requested beyond the pool this frame
static const int kStats = 8;

void* oracle_create(float voxel, float trunc, uint32_t slots, uint32_t pool) {
  if (!(voxel > 0.0f) || !(trunc >= voxel) || slots == 0 || (slots & (slots - 1)) != 0 ||
      pool == 0 || pool > slots)
    return nullptr;
  Volume* v = new Volume();
  v->voxel = voxel;
  v->trunc = trunc;
  v->slots = slots;
  v->pool = pool;
  return v;
}

void oracle_destroy(void* h) { delete static_cast<Volume*>(h); }

void oracle_reset(void* h) {
  Volume* v = static_cast<Volume*>(h);
  v->blocks.clear();
  v->claimed = 0;
  v->poisoned = false;
}

uint32_t oracle_block_count(void* h) {
  Volume* v = static_cast<Volume*>(h);
  return static_cast<uint32_t>(v->claimed < v->pool ? v->claimed : v->pool);
}

// Fuse one frame. depth: H*W float32 row-major; rgb: H*W*3 uint8 or null;
// intr = {fx, fy, cx, cy}; pose = row-major 4x4 camera-to-world.
int oracle_fuse(void* h, const float* depth, int W, int H, const float* intr,
                const float* pose, const uint8_t* rgb, uint64_t* stats) {
  Volume* V = static_cast<Volume*>(h);
  uint64_t st[kStats] = {0};
  if (V->poisoned) {
    if (stats) std::memcpy(stats, st, sizeof(st));
    return OR_POISONED;
  }
  if (W <= 0 || H <= 0 || depth == nullptr || intr == nullptr || pose == nullptr)
    return OR_INVALID_ARG;

  const float v = V->voxel;
  const float tau = V->trunc;
  const float inv_v = 1.0f / v;
  const int M = static_cast<int>(lrintf(tau / v));
  const float fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
  // R = pose[0..2][0..2] (row-major), t = pose[0..2][3]
  float R[3][3], t[3];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) R[i][j] = pose[4 * i + j];
    t[i] = pose[4 * i + 3];
  }
  // R5: the voxel centre in the camera frame, R^T ((g + 1/2) v - t), as one
  // affine map of the integer voxel g: c = A g + b, A = v R^T,
  // b = R^T (v/2 - t), each constant computed once per frame.
  float A[3][3], bc[3], half_minus_t[3];
  for (int i = 0; i < 3; ++i) half_minus_t[i] = std::fmaf(0.5f, v, -t[i]);
  for (int j = 0; j < 3; ++j) {
    for (int i = 0; i < 3; ++i) A[j][i] = v * R[i][j];
    bc[j] = std::fmaf(R[2][j], half_minus_t[2],
                      std::fmaf(R[1][j], half_minus_t[1], R[0][j] * half_minus_t[0]));
  }

  // Per-frame bookkeeping for the statistics.
  std::map<Coord, std::array<uint8_t, kVox>> touched;
  std::map<Coord, bool> is_new;
  std::vector<std::array<int32_t, 3>> walk;
  walk.reserve(2 * M + 1);

  for (int pv = 0; pv < H; ++pv) {
    for (int pu = 0; pu < W; ++pu) {
      const float d = depth[pv * W + pu];
      if (!std::isfinite(d) || !(d > 0.0f)) continue;
      st[0]++;

      // Back-projection and unit view ray (camera frame), then both in the
      // world frame once per point (R5): P = R p + t, D = R d.
      const float rx = (static_cast<float>(pu) - cx) / fx;
      const float ry = (static_cast<float>(pv) - cy) / fy;
      const float pcx = rx * d, pcy = ry * d, pcz = d;
      const float n = std::sqrt(std::fmaf(rx, rx, std::fmaf(ry, ry, 1.0f)));
      const float dx = rx / n, dy = ry / n, dz = 1.0f / n;
      float Pw[3], Dw[3];
      for (int i = 0; i < 3; ++i) {
        Pw[i] = std::fmaf(R[i][2], pcz, std::fmaf(R[i][1], pcy, std::fmaf(R[i][0], pcx, t[i])));
        Dw[i] = std::fmaf(R[i][2], dz, std::fmaf(R[i][1], dy, R[i][0] * dx));
      }

      float col[3] = {0.0f, 0.0f, 0.0f};
      if (rgb) {
        for (int c = 0; c < 3; ++c) col[c] = static_cast<float>(rgb[(pv * W + pu) * 3 + c]);
      }

      walk.clear();
      bool have_last = false;
      Coord last_coord{0, 0, 0};
      BlockData* last_block = nullptr;
      std::array<uint8_t, kVox>* last_touched = nullptr;
      for (int k = 0; k <= 2 * M; ++k) {
        st[1]++;
        const float tk = static_cast<float>(k - M) * v;
        int32_t g[3];
        bool in_range = true;
        for (int i = 0; i < 3; ++i) {
          const float sw = std::fmaf(tk, Dw[i], Pw[i]);  // the sample, world frame
          const float fg = std::floor(sw * inv_v);
          // R6: block coordinate must lie in [-2^20, 2^20), voxel in [-2^23, 2^23)
          if (!(fg >= -8388608.0f && fg < 8388608.0f)) {
            in_range = false;
            g[i] = 0;
          } else {
            g[i] = static_cast<int32_t>(fg);
          }
        }
        if (!in_range) {
          st[6]++;
          continue;
        }
        // Each distinct voxel at most once per point (R1).
        bool seen = false;
        for (const auto& w : walk)
          if (w[0] == g[0] && w[1] == g[1] && w[2] == g[2]) seen = true;
        if (seen) continue;
        walk.push_back({g[0], g[1], g[2]});

        // Voxel centre in the camera frame: c = A g + b.
        float cc[3];
        for (int j = 0; j < 3; ++j)
          cc[j] = std::fmaf(A[j][2], static_cast<float>(g[2]),
                            std::fmaf(A[j][1], static_cast<float>(g[1]),
                                      std::fmaf(A[j][0], static_cast<float>(g[0]), bc[j])));

        // Occlusion test (R3).
        if (!(cc[2] > 0.0f)) continue;
        const float iz = 1.0f / cc[2];
        const float qu = std::floor(std::fmaf(fx, cc[0] * iz, cx) + 0.5f);
        const float qv = std::floor(std::fmaf(fy, cc[1] * iz, cy) + 0.5f);
        if (!(qu >= 0.0f && qu < static_cast<float>(W))) continue;
        if (!(qv >= 0.0f && qv < static_cast<float>(H))) continue;
        const float d2 = depth[static_cast<int>(qv) * W + static_cast<int>(qu)];
        if (!std::isfinite(d2) || !(d2 > 0.0f)) continue;
        if (!((d2 - cc[2]) >= -tau)) continue;

        // Signed distance at the voxel centre (R2).
        const float sdf = d - cc[2];
        const float tsdf = std::fmin(1.0f, std::fmax(-1.0f, sdf / tau));

        const Coord b{floor_div8(g[0]), floor_div8(g[1]), floor_div8(g[2])};
        const int l = floor_mod8(g[0]) + kEdge * floor_mod8(g[1]) + kEdge * kEdge * floor_mod8(g[2]);

        // One-entry cache of the last block this point touched (a plain lookup
        // shortcut; consecutive samples of a ray mostly share a block).
        if (!(have_last && last_coord == b)) {
          auto it0 = V->blocks.find(b);
          last_block = (it0 == V->blocks.end()) ? nullptr : &it0->second;
          last_touched = (it0 == V->blocks.end()) ? nullptr : &touched[b];
          last_coord = b;
          have_last = true;
        }
        auto it = V->blocks.end();
        if (last_block == nullptr) {
          // A block first requested in this frame.
          auto nw = is_new.find(b);
          if (nw == is_new.end()) {
            V->claimed++;
            const bool fits = V->claimed <= V->pool;
            is_new[b] = fits;
            if (!fits) st[7]++;
            if (fits) {
              it = V->blocks.emplace(b, BlockData()).first;
              st[5]++;
            }
          }
          if (it == V->blocks.end()) continue;  // over the pool: dropped, reported below
          last_block = &it->second;
          last_touched = &touched[b];
        }
        st[2]++;
        BlockData& B = *last_block;
        B.tsdf_sum[l] += static_cast<double>(tsdf);
        B.weight[l] += 1u;
        B.r_sum[l] += static_cast<double>(col[0]) / 255.0;
        B.g_sum[l] += static_cast<double>(col[1]) / 255.0;
        B.b_sum[l] += static_cast<double>(col[2]) / 255.0;
        (*last_touched)[l] = 1;
      }
    }
  }

  for (const auto& kv : touched) {
    st[4]++;
    for (int l = 0; l < kVox; ++l) st[3] += kv.second[l];
  }
  if (stats) std::memcpy(stats, st, sizeof(st));
  if (V->claimed > V->pool) {
    // Overflow is reported, never silent (Section 3.4). Each distinct block
    // needs its own table slot and pool entry. With pool < slots the pool runs
    // out first; with pool == slots the table does.
    V->poisoned = true;
    return V->pool < V->slots ? OR_POOL_FULL : OR_TABLE_FULL;
  }
  return OR_OK;
}

// Export every allocated block, ordered by coordinate. coords: n*3 int32;
// vox: n*5*512 float32 as [block][channel][voxel] with channels
// {tsdf mean, weight, red mean, green mean, blue mean}; vox64 (nullable) the
// same in double. Means are sum / weight where weight > 0, else 0.
// Returns the number of blocks (written only if <= cap).
uint32_t oracle_export(void* h, int32_t* coords, float* vox, double* vox64, uint32_t cap) {
  Volume* V = static_cast<Volume*>(h);
  const uint32_t n = static_cast<uint32_t>(V->blocks.size());
  if (n > cap) return n;
  uint32_t i = 0;
  for (const auto& kv : V->blocks) {
    coords[3 * i + 0] = kv.first.x;
    coords[3 * i + 1] = kv.first.y;
    coords[3 * i + 2] = kv.first.z;
    const BlockData& B = kv.second;
    for (int l = 0; l < kVox; ++l) {
      const double w = static_cast<double>(B.weight[l]);
      double ch[5] = {0.0, w, 0.0, 0.0, 0.0};
      if (B.weight[l] > 0) {
        ch[0] = B.tsdf_sum[l] / w;
        ch[2] = B.r_sum[l] / w;
        ch[3] = B.g_sum[l] / w;
        ch[4] = B.b_sum[l] / w;
      }
      for (int c = 0; c < 5; ++c) {
        const size_t o = (static_cast<size_t>(i) * 5 + c) * kVox + l;
        if (vox) vox[o] = static_cast<float>(ch[c]);
        if (vox64) vox64[o] = ch[c];
      }
    }
    ++i;
  }
  return n;
}

// Export the blocks at the given coordinates (n x 3 int32), in that order, as
// n x 5 x 512 doubles (same channels as oracle_export). found[i] = 1 if the
// block is allocated, else 0 and its values are zero. A plain read-out.
void oracle_export_some(void* h, const int32_t* coords, uint32_t n, double* vox64,
                        uint8_t* found) {
  Volume* V = static_cast<Volume*>(h);
  for (uint32_t i = 0; i < n; ++i) {
    const Coord c{coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]};
    auto it = V->blocks.find(c);
    found[i] = it != V->blocks.end();
    for (int l = 0; l < kVox; ++l) {
      double ch[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
      if (it != V->blocks.end() && it->second.weight[l] > 0) {
        const BlockData& B = it->second;
        const double w = static_cast<double>(B.weight[l]);
        ch[0] = B.tsdf_sum[l] / w;
        ch[1] = w;
        ch[2] = B.r_sum[l] / w;
        ch[3] = B.g_sum[l] / w;
        ch[4] = B.b_sum[l] / w;
      }
      for (int c5 = 0; c5 < 5; ++c5) vox64[(static_cast<size_t>(i) * 5 + c5) * kVox + l] = ch[c5];
    }
  }
}

// ---------------------------------------------------------------------------
// Surface extraction: marching tetrahedra (the extraction stage of Section 2,
// which the paper runs once, in CUDA C++, and excludes from its comparison).
// The paper names the method and nothing more; the definition below is this
// project's reading (E1-E4), written out plainly:
//   E1 The grid points are voxel centres (g + 1/2) v. Every voxel g whose 8
//      corners g + {0,1}^3 all have weight > 0 spans one cube; cubes with a
//      corner of weight 0 (unobserved, or in no allocated block) are skipped.
//      A corner's value is its mean tsdf, sum / weight.
//   E2 Each cube is split into the 6 tetrahedra that share its diagonal from
//      corner 0 to corner 7 (corner c = g + (c&1, c>>1&1, c>>2&1)); each is a
//      monotone path 0 -> one axis -> two axes -> 7, so neighbouring cubes
//      split shared faces the same way.
//   E3 A corner is inside when its value is < 0 (behind the surface). Every
//      tetrahedron edge whose ends differ holds one vertex at the linear zero
//      crossing, parameterised from the edge's lower corner (the one with
//      fewer offset bits): p = p_lo + t (p_hi - p_lo), t = v_lo / (v_lo - v_hi).
//   E4 One inside (or one outside) corner gives one triangle, two give two;
//      triangles are wound so that their normals point towards positive values
//      (free space).
// Output: each triangle as 9 coordinates (x, y, z of its three vertices) and
// a cell record {gx, gy, gz, 2*tet + sub} naming the cube, the tetrahedron and
// which of its triangles it is. Computed in double.

namespace {

// corner of the cube, by index, as an offset
inline void corner_offset(int c, int& dx, int& dy, int& dz) {
  dx = c & 1;
  dy = (c >> 1) & 1;
  dz = (c >> 2) & 1;
}

// The six tetrahedra, each listed in positive orientation
// (det[p1 - p0, p2 - p0, p3 - p0] > 0).
const int kTets[6][4] = {{0, 1, 3, 7}, {0, 1, 7, 5}, {0, 2, 7, 3},
                         {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 7, 6}};

inline int popcount4(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }

struct Mesher {
  const Volume* V;
  std::vector<double>* tris;
  std::vector<int32_t>* cells;

  // value at voxel g: false if unobserved
  bool value(int32_t gx, int32_t gy, int32_t gz, double& out) const {
    const Coord b{floor_div8(gx), floor_div8(gy), floor_div8(gz)};
    auto it = V->blocks.find(b);
    if (it == V->blocks.end()) return false;
    const int l = floor_mod8(gx) + kEdge * floor_mod8(gy) + kEdge * kEdge * floor_mod8(gz);
    const uint32_t w = it->second.weight[l];
    if (w == 0) return false;
    out = it->second.tsdf_sum[l] / static_cast<double>(w);
    return true;
  }

  // vertex on the edge between corners a and b of the cube at g
  void vertex(const int32_t g[3], const double val[8], int a, int b, double p[3]) const {
    // the lower corner is the one whose offset bits are a subset of the other's
    const int lo = ((a & b) == a) ? a : b;
    const int hi = lo == a ? b : a;
    const double t = val[lo] / (val[lo] - val[hi]);
    int o_lo[3], o_hi[3];
    corner_offset(lo, o_lo[0], o_lo[1], o_lo[2]);
    corner_offset(hi, o_hi[0], o_hi[1], o_hi[2]);
    const double v = static_cast<double>(V->voxel);
    for (int k = 0; k < 3; ++k) {
      const double plo = (static_cast<double>(g[k] + o_lo[k]) + 0.5) * v;
      const double phi = (static_cast<double>(g[k] + o_hi[k]) + 0.5) * v;
      p[k] = plo + t * (phi - plo);
    }
  }

  void emit(const int32_t g[3], const double val[8], int tet, int sub, const int e[3][2]) {
    for (int k = 0; k < 3; ++k) {
      double p[3];
      vertex(g, val, e[k][0], e[k][1], p);
      tris->push_back(p[0]);
      tris->push_back(p[1]);
      tris->push_back(p[2]);
    }
    cells->push_back(g[0]);
    cells->push_back(g[1]);
    cells->push_back(g[2]);
    cells->push_back(2 * tet + sub);
  }

  void cube(int32_t gx, int32_t gy, int32_t gz) {
    double val[8];
    for (int c = 0; c < 8; ++c) {
      int dx, dy, dz;
      corner_offset(c, dx, dy, dz);
      if (!value(gx + dx, gy + dy, gz + dz, val[c])) return;  // E1
    }
    const int32_t g[3] = {gx, gy, gz};
    for (int t = 0; t < 6; ++t) {
      const int* T = kTets[t];
      int m = 0;  // which of the tetrahedron's corners are inside
      for (int k = 0; k < 4; ++k)
        if (val[T[k]] < 0.0) m |= 1 << k;
      const int n_in = popcount4(m);
      if (n_in == 0 || n_in == 4) continue;
      if (n_in == 1 || n_in == 3) {
        // the corner on its own side, first in a positive ordering of the four
        const int lone = (n_in == 1) ? m : (~m & 15);
        static const int kLone[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 0, 1, 3}, {3, 0, 2, 1}};
        const int i = lone == 1 ? 0 : lone == 2 ? 1 : lone == 4 ? 2 : 3;
        const int a = T[kLone[i][0]], b = T[kLone[i][1]], c = T[kLone[i][2]], d = T[kLone[i][3]];
        if (n_in == 1) {
          const int e[3][2] = {{a, b}, {a, c}, {a, d}};  // normal away from the inside corner
          emit(g, val, t, 0, e);
        } else {
          const int e[3][2] = {{a, b}, {a, d}, {a, c}};  // normal towards the outside corner
          emit(g, val, t, 0, e);
        }
      } else {
        // two inside (a, b) and two outside (c, d), (a, b, c, d) positively ordered
        static const int kPair[6][5] = {
            // mask, then the ordering
            {0x3, 0, 1, 2, 3}, {0x5, 0, 2, 3, 1}, {0x9, 0, 3, 1, 2},
            {0x6, 1, 2, 0, 3}, {0xA, 1, 3, 2, 0}, {0xC, 2, 3, 0, 1}};
        int r = 0;
        while (kPair[r][0] != m) ++r;
        const int a = T[kPair[r][1]], b = T[kPair[r][2]], c = T[kPair[r][3]], d = T[kPair[r][4]];
        const int e0[3][2] = {{a, c}, {a, d}, {b, d}};
        const int e1[3][2] = {{a, c}, {b, d}, {b, c}};
        emit(g, val, t, 0, e0);
        emit(g, val, t, 1, e1);
      }
    }
  }
};

}  // namespace

// Marching tetrahedra over every observed voxel (E1-E4 above), blocks in
// coordinate order, voxels in local-index order. tris: n*9 doubles, cells:
// n*4 int32 (either may be null). Returns n; writes only if n <= cap.
uint32_t oracle_extract(void* h, double* tris, int32_t* cells, uint32_t cap) {
  const Volume* V = static_cast<const Volume*>(h);
  std::vector<double> t;
  std::vector<int32_t> c;
  Mesher M{V, &t, &c};
  for (const auto& kv : V->blocks) {
    const BlockData& B = kv.second;
    for (int l = 0; l < kVox; ++l) {
      if (B.weight[l] == 0) continue;
      M.cube(kv.first.x * kEdge + (l % kEdge), kv.first.y * kEdge + (l / kEdge) % kEdge,
             kv.first.z * kEdge + l / (kEdge * kEdge));
    }
  }
  const uint32_t n = static_cast<uint32_t>(c.size() / 4);
  if (n <= cap) {
    if (tris) std::memcpy(tris, t.data(), t.size() * sizeof(double));
    if (cells) std::memcpy(cells, c.data(), c.size() * sizeof(int32_t));
  }
  return n;
}

// Set one voxel's tsdf sum and weight directly (creating its block): for
// extraction tests on hand-built grids. Returns 0, or 1 if the block would
// exceed the pool.
int oracle_set_voxel(void* h, int32_t gx, int32_t gy, int32_t gz, double tsdf_sum,
                     uint32_t weight) {
  Volume* V = static_cast<Volume*>(h);
  const Coord b{floor_div8(gx), floor_div8(gy), floor_div8(gz)};
  auto it = V->blocks.find(b);
  if (it == V->blocks.end()) {
    if (V->claimed >= V->pool) return 1;
    it = V->blocks.emplace(b, BlockData{}).first;
    ++V->claimed;
  }
  const int l = floor_mod8(gx) + kEdge * floor_mod8(gy) + kEdge * kEdge * floor_mod8(gz);
  it->second.tsdf_sum[l] = tsdf_sum;
  it->second.weight[l] = weight;
  return 0;
}

}  // extern "C"
