// Kernels of hash-blocked TSDF fusion (paper Section 2.2, "Two passes").
//
// tile_fused_kernel (the default path, one launch per frame): one CTA per
// 16x16 pixel tile --
//   1. every thread walks its point's band once (unrolled when the half band
//      M is compiled), keeps each accepted sample as one packed word and its
//      tsdf value, and the tile's distinct blocks are collected in a
//      shared-memory set and list (a per-warp __match_any_sync dedupe first);
//   2. the list is inserted warp-cooperatively (Listing 1 probe and
//      compare-exchange, counter increments aggregated per warp) and every
//      block's pool index obtained into shared memory;
//   3. every accepted voxel's five sums are added with two fire-and-forget
//      reductions (a 16-byte vector and a scalar), the index taken from the
//      tile's list: no second walk, no table probe.
// The two-pass path of the paper is kept as separate stage A and stage B
// kernels, each with several strategies:
//   stage A: allocate_kernel (Listing 1 per sample after a warp dedupe,
//     waiting for publication on a hit: the paper's protocol),
//     tile_allocate_kernel (phases 1 and 2 above, without waiting),
//     warp_kernel<Allocate> (per warp, no shared memory);
//   stage B: integrate_scatter_kernel (per-thread lookups, the paper's
//     update), warp_kernel<Integrate> (warp-deduped lookups), the tile kernel
//     with phase 2 looking the tile's keys up warp-cooperatively;
//   warp_kernel<Fused>: a barrier-free fused kernel, one warp per 8x4 patch.
// Batched persistent variants serve many frames, each into its own volume,
// per launch. Read-out, reset and diagnostics: export_kernel (means from
// sums), slot_list_kernel, clear_used_kernel / clear_slots_kernel,
// table_stats_kernel, weight_sum_kernel; surface extraction: extract_kernel.
// The tile machinery and the tile kernels are in tsdf_tile.cuh; the fused
// tile kernels with a point's walk split over several threads, and the tile
// kernel of stage B (tile_fused_kernel<..., kOpIntegrate>), are compiled in
// tsdf_kernels_split.cu.

#include <algorithm>
#include <climits>
#include <cstdint>

#include "tsdf_device.cuh"
#include "tsdf_launch.h"
#include "tsdf_tile.cuh"

namespace tsdf {

// ----------------------------------------------------------------------------
// stage B, scatter: five atomic additions per accepted voxel (Section 2.2)
// ----------------------------------------------------------------------------
__device__ __forceinline__ void scatter_add(const FrameArgs& f, const VolumeArgs& vol,
                                            BlockCacheT& bc, const Ray& r, int gx, int gy, int gz,
                                            float zc, bool colour, float cr, float cg,
                                            float cb) {
  const int bx = gx >> 3, by = gy >> 3, bz = gz >> 3;
  const unsigned long long key = pack_key(bx, by, bz);
  if (key != bc.key) {
    bc.key = key;
    bc.idx = resolve_for_update(vol, lookup_block(vol, key, bx, by, bz));
  }
  if (bc.idx < 0) return;
  add_contribution(vol, static_cast<size_t>(bc.idx) * kBlockVoxels + local_index(gx, gy, gz),
                   tsdf_value(f, r.d, zc), colour, cr, cg, cb);
}

// Stage B, the paper's update, for the 256 points of one tile (each thread
// alone; no barrier).
template <int M>
__device__ __forceinline__ void scatter_body(const FrameArgs& f, const VolumeArgs& vol, int tile,
                                             int tiles_x) {
  if (load_err_volatile(vol.hdr)) return;  // poisoned volume: do nothing
  int u, v;
  tile_pixel(tile, tiles_x, u, v);
  if (u >= f.W || v >= f.H) return;
  Ray r;
  if (!make_ray(f, u, v, load_depth(f, static_cast<long long>(v) * f.W + u), r)) return;
  float cr = 0.0f, cg = 0.0f, cb = 0.0f;
  const bool colour = f.rgb != nullptr;
  if (colour) {
    load_colour(f, u, v, cr, cg, cb);
  }
  if constexpr (M > 0) {
    unsigned smp[2 * M + 1];
    float tv[2 * M + 1];
    int bx0 = 0, by0 = 0, bz0 = 0;
    walk_point_packed<M>(f, r, smp, tv, bx0, by0, bz0);
    unsigned last = 0u;  // block offset bits of the looked-up block (0: none yet)
    int idx = -1;
#pragma unroll
    for (int k = 0; k < 2 * M + 1; ++k) {
      const unsigned q = smp[k];
      if (!(q & kSampleValid)) continue;
      const unsigned blk = q & kSampleBlockBits;
      if (blk != last) {
        last = blk;
        const int bx = bx0 + static_cast<int>((q >> 9) & 15u) - 8;
        const int by = by0 + static_cast<int>((q >> 13) & 15u) - 8;
        const int bz = bz0 + static_cast<int>((q >> 17) & 15u) - 8;
        idx = resolve_for_update(vol, lookup_block(vol, pack_key(bx, by, bz), bx, by, bz));
      }
      if (idx >= 0)
        add_contribution(vol, static_cast<size_t>(idx) * kBlockVoxels + (q & 511u),
                         tv[k], colour, cr, cg, cb);
    }
  } else {
    BlockCacheT bc;
    WalkDedupe walk;
    for (int k = 0; k <= 2 * f.M; ++k) {
      int gx, gy, gz;
      float zc;
      if (!sample_voxel(f, r, k, gx, gy, gz) || walk.seen_then_push(gx, gy, gz) ||
          !voxel_test(f, gx, gy, gz, zc))
        continue;
      scatter_add(f, vol, bc, r, gx, gy, gz, zc, colour, cr, cg, cb);
    }
  }
}

template <int M>
__global__ void __launch_bounds__(kThreads, 4)
    integrate_scatter_kernel(const __grid_constant__ FrameArgs f,
                             const __grid_constant__ VolumeArgs vol, int tiles_x) {
  scatter_body<M>(f, vol, blockIdx.x, tiles_x);
}

// ----------------------------------------------------------------------------
// read-out and reset
// ----------------------------------------------------------------------------
// Means of n blocks (Section 2.2: the pool holds sums). Output block j is pool
// block list[j], or pool block j when list is null.
__global__ void export_kernel(const __grid_constant__ VolumeArgs vol, float* __restrict__ out,
                              unsigned int n, const unsigned int* __restrict__ list) {
  const size_t total = static_cast<size_t>(n) * kBlockVoxels;
  for (size_t j = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; j < total;
       j += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t blk = j / kBlockVoxels;
    const size_t l = j % kBlockVoxels;
    const size_t i = (list ? static_cast<size_t>(list[blk]) : blk) * kBlockVoxels + l;
    if (!index_ok(i, static_cast<unsigned long long>(vol.pool) * kBlockVoxels, &vol.hdr->err))
      continue;
    const float4 s = vol.twrg[i];
    const float w = s.y;
    float* o = out + blk * 5 * kBlockVoxels + l;
    const bool any = w > 0.0f;
    const float w255 = w * 255.0f;  // exact while w < 65793
    o[0] = any ? __fdiv_rn(s.x, w) : 0.0f;
    o[kBlockVoxels] = w;
    o[2 * kBlockVoxels] = any ? __fdiv_rn(s.z, w255) : 0.0f;
    o[3 * kBlockVoxels] = any ? __fdiv_rn(s.w, w255) : 0.0f;
    o[4 * kBlockVoxels] = any ? __fdiv_rn(vol.blue[i], w255) : 0.0f;
  }
}

// Slot-index volumes: the occupied slots in slot order, and their block
// coordinates (from the key), by one CTA of 1024 threads scanning the table
// 1024 slots at a time with a block-wide prefix sum. Writes at most cap
// entries; *found receives the number of occupied slots.
constexpr int kListThreads = 1024;
__global__ void __launch_bounds__(kListThreads)
    slot_list_kernel(const __grid_constant__ VolumeArgs vol, unsigned int* __restrict__ list,
                     int32_t* __restrict__ coords, unsigned int cap,
                     unsigned int* __restrict__ found) {
  __shared__ unsigned int warp_count[kListThreads / 32];
  __shared__ unsigned int warp_excl[kListThreads / 32];
  __shared__ unsigned int s_total;
  __shared__ unsigned int base;
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) base = 0;
  for (unsigned int start = 0; start < vol.slots; start += kListThreads) {
    const unsigned int slot = start + threadIdx.x;
    const unsigned long long key = slot < vol.slots ? vol.table[slot].key : kEmptyKey;
    const bool occ = key != kEmptyKey;
    const unsigned m = __ballot_sync(0xffffffffu, occ);
    if (lane == 0) warp_count[w] = __popc(m);
    __syncthreads();
    if (w == 0) {
      const unsigned c = warp_count[lane];
      unsigned incl = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= static_cast<unsigned>(o)) incl += t;
      }
      warp_excl[lane] = incl - c;
      if (lane == 31) s_total = incl;
    }
    __syncthreads();
    if (occ) {
      const unsigned int p = base + warp_excl[w] + __popc(m & ((1u << lane) - 1u));
      if (p < cap) {
        int bx, by, bz;
        unpack_key(key, bx, by, bz);
        list[p] = slot;
        coords[3 * static_cast<size_t>(p)] = bx;
        coords[3 * static_cast<size_t>(p) + 1] = by;
        coords[3 * static_cast<size_t>(p) + 2] = bz;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) base += s_total;
  }
  if (threadIdx.x == 0) *found = base;
}

// Zero the used prefix [0, min(count, pool)) of the pool's sums; reads the
// count on the device so the host needs no round trip.
__global__ void clear_used_kernel(const __grid_constant__ VolumeArgs vol) {
  const unsigned int c = *reinterpret_cast<volatile unsigned int*>(&vol.hdr->count);
  const unsigned int n = c < vol.pool ? c : vol.pool;
  // one 16-byte store per thread and step, consecutive threads on
  // consecutive addresses: the records first, then the blue sums
  const size_t records = static_cast<size_t>(n) * kBlockVoxels;
  const size_t quads = records + records / 4;
  const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < quads;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    if (i < records)
      vol.twrg[i] = z;
    else
      reinterpret_cast<float4*>(vol.blue)[i - records] = z;
  }
}

// Slot-index volumes: zero the pool block of every occupied slot (one warp per
// slot; the used blocks are scattered over the whole pool). Runs before the
// table is cleared.
__global__ void clear_slots_kernel(const __grid_constant__ VolumeArgs vol) {
  const unsigned lane = threadIdx.x & 31u;
  const size_t nwarps = (static_cast<size_t>(gridDim.x) * blockDim.x) >> 5;
  const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (size_t slot = (blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x) >> 5;
       slot < vol.slots; slot += nwarps) {
    if (vol.table[slot].key == kEmptyKey) continue;
    float4* t = vol.twrg + slot * kBlockVoxels;
#pragma unroll
    for (int j = 0; j < kBlockVoxels / 32; ++j) t[lane + 32 * j] = z;
    float4* q = reinterpret_cast<float4*>(vol.blue) + slot * (kBlockVoxels / 4);
#pragma unroll
    for (int j = 0; j < kBlockVoxels / 4 / 32; ++j) q[lane + 32 * j] = z;
  }
}

// Occupancy and probe lengths of the table, and the total weight in the pool
// (= contributions received): a diagnostic read-out, not part of fusion.
__global__ void table_stats_kernel(const __grid_constant__ VolumeArgs vol,
                                   TableStatsDev* __restrict__ out) {
  unsigned long long occ = 0, psum = 0;
  unsigned int pmax = 0;
  for (size_t slot = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
       slot < vol.slots; slot += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const unsigned long long key = vol.table[slot].key;
    if (key == kEmptyKey) continue;
    int bx, by, bz;
    unpack_key(key, bx, by, bz);
    const unsigned int home = hash_block(bx, by, bz) & vol.mask;
    const unsigned int len = ((static_cast<unsigned int>(slot) - home) & vol.mask) + 1u;
    occ += 1;
    psum += len;
    pmax = len > pmax ? len : pmax;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    occ += __shfl_xor_sync(0xffffffffu, occ, o);
    psum += __shfl_xor_sync(0xffffffffu, psum, o);
    const unsigned int t = __shfl_xor_sync(0xffffffffu, pmax, o);
    pmax = t > pmax ? t : pmax;
  }
  if ((threadIdx.x & 31u) == 0 && occ) {
    atomicAdd(&out->occupied, occ);
    atomicAdd(&out->probe_sum, psum);
    atomicMax(&out->probe_max, pmax);
  }
}

// Sum of all voxel weights of the used blocks (weights are integer counts
// held exactly in float32; summed as integers). One warp per block.
__global__ void weight_sum_kernel(const __grid_constant__ VolumeArgs vol,
                                  TableStatsDev* __restrict__ out) {
  const unsigned lane = threadIdx.x & 31u;
  const size_t nwarps = (static_cast<size_t>(gridDim.x) * blockDim.x) >> 5;
  const unsigned int c = *reinterpret_cast<volatile unsigned int*>(&vol.hdr->count);
  const size_t nb = vol.slot_index ? vol.slots : (c < vol.pool ? c : vol.pool);
  unsigned long long sum = 0;
  for (size_t b = (blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x) >> 5; b < nb;
       b += nwarps) {
    if (vol.slot_index && vol.table[b].key == kEmptyKey) continue;
    const float4* q = vol.twrg + b * kBlockVoxels;
#pragma unroll
    for (int j = 0; j < kBlockVoxels / 32; ++j)
      sum += static_cast<unsigned long long>(q[lane + 32 * j].y);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  if (lane == 0 && sum) atomicAdd(&out->weight_sum, sum);
}

// ----------------------------------------------------------------------------
// surface extraction: marching tetrahedra over the allocated blocks
// ----------------------------------------------------------------------------
// The grid points are voxel centres; every voxel whose 8 corners g + {0,1}^3
// are all observed (weight > 0) spans a cube, split into the 6 tetrahedra
// around its 0-7 diagonal; a corner is inside when its mean tsdf is < 0; each
// tetrahedron edge with ends on both sides holds a vertex at the linear zero
// crossing, measured from its lower corner; triangles are wound with normals
// towards positive values.
//
// One WARP per allocated block, with no CTA-wide barrier: lanes 0-7 look up
// the block's 7 upper neighbours, the warp stages the 9x9x9 tile of means in
// its own shared memory (NaN where unobserved), each lane takes 16 of the
// 512 cubes, the warp reserves its output with one atomicAdd, and the
// triangles go through a per-warp shared staging area so that they leave in
// coalesced stores. Many warps per SM, each on its own block, hide the
// latency of the lookups and loads.
constexpr int kExtractWarps = 4;     // warps (blocks in flight) per CTA
constexpr int kExtractStage = 64;    // triangles per output window of a warp
constexpr int kTileVals = 9 * 9 * 9;

// Tetrahedra of a cube, positively oriented; corner c = g + (c&1, c>>1&1, c>>2&1).
__constant__ unsigned char c_tets[6][4] = {{0, 1, 3, 7}, {0, 1, 7, 5}, {0, 2, 7, 3},
                                           {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 7, 6}};
// For a lone corner at position i: an even reordering of the four that puts it first.
__constant__ unsigned char c_lone[4][4] = {{0, 1, 2, 3}, {1, 0, 3, 2}, {2, 0, 1, 3}, {3, 0, 2, 1}};
// For an inside pair, indexed by its 4-bit mask: an even reordering that puts
// the pair first (unused masks hold zeros).
__constant__ unsigned char c_pair[16][4] = {
    {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 1, 2, 3}, {0, 0, 0, 0}, {0, 2, 3, 1},
    {1, 2, 0, 3}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 3, 1, 2}, {1, 3, 2, 0}, {0, 0, 0, 0},
    {2, 3, 0, 1}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}};

// Offset of cube corner c in the staged 9x9x9 tile.
__device__ __forceinline__ int corner_offset(int c) {
  return (c & 1) + ((c >> 1) & 1) * 9 + ((c >> 2) & 1) * 81;
}

// The 4-bit inside mask of tetrahedron t from the cube's 8-bit inside mask.
__device__ __forceinline__ unsigned tet_bits(unsigned inside, int t) {
  unsigned m = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) m |= ((inside >> c_tets[t][k]) & 1u) << k;
  return m;
}

// Triangles of a cube with inside mask `inside` (0..12).
__device__ __forceinline__ int cube_triangle_count(unsigned inside) {
  int n = 0;
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int k = __popc(tet_bits(inside, t));
    n += (k == 0 || k == 4) ? 0 : (k == 2 ? 2 : 1);
  }
  return n;
}

// A cube of the staged tile: its base voxel, the tile position of corner 0,
// and its 8-bit inside mask (0 when a corner is unobserved or none differs).
struct Cube {
  int gx, gy, gz;
  int at;
  unsigned inside;
};

__device__ __forceinline__ Cube load_cube(const float* val, int c, int bx, int by, int bz) {
  Cube C;
  const int lx = c & 7, ly = (c >> 3) & 7, lz = c >> 6;
  C.gx = bx * kBlockEdge + lx;
  C.gy = by * kBlockEdge + ly;
  C.gz = bz * kBlockEdge + lz;
  C.at = lz * 81 + ly * 9 + lx;
  bool ok = true;
  unsigned inside = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float x = val[C.at + corner_offset(k)];
    ok = ok && !isnan(x);
    inside |= (x < 0.0f) ? (1u << k) : 0u;
  }
  C.inside = (ok && inside != 0xFFu) ? inside : 0u;
  return C;
}

// The k-th triangle (in tetrahedron order) of a cube with inside mask
// `inside`: its name tag 2*tetrahedron + sub and its three edges as corner
// pairs, wound with the normal towards positive values.
__device__ __forceinline__ void cube_triangle(unsigned inside, int k, int& tag, int e[6]) {
  int t = 0;
  unsigned m = 0;
  int n_in = 0;
  for (; t < 6; ++t) {
    m = tet_bits(inside, t);
    n_in = __popc(m);
    const int c = (n_in == 0 || n_in == 4) ? 0 : (n_in == 2 ? 2 : 1);
    if (k < c) break;
    k -= c;
  }
  if (t == 6) t = 5;  // unreachable: k is below the cube's count
  const unsigned char* T = c_tets[t];
  if (n_in == 2) {
    const unsigned char* o = c_pair[m];
    const int a = T[o[0]], b = T[o[1]], c = T[o[2]], d = T[o[3]];
    // two inside (a, b), two outside (c, d): the quad a-c, a-d, b-d, b-c
    const int q0[6] = {a, c, a, d, b, d}, q1[6] = {a, c, b, d, b, c};
#pragma unroll
    for (int i = 0; i < 6; ++i) e[i] = k == 0 ? q0[i] : q1[i];
    tag = 2 * t + k;
  } else {
    const unsigned lone = n_in == 1 ? m : (~m & 15u);
    const unsigned char* o = c_lone[__ffs(lone) - 1];
    const int a = T[o[0]], b = T[o[1]], c = T[o[2]], d = T[o[3]];
    // a lone inside corner: normal away from it; a lone outside corner: towards it
    e[0] = a;
    e[1] = b;
    e[2] = a;
    e[3] = n_in == 1 ? c : d;
    e[4] = a;
    e[5] = n_in == 1 ? d : c;
    tag = 2 * t;
  }
}

// Vertex on the edge between corners a and b of cube `cube` of the staged
// tile, measured from the lower corner (the one whose offset bits are a
// subset of the other's).
__device__ __forceinline__ void tile_edge_vertex(const float* val, int cube, int bx, int by,
                                                 int bz, float v, int a, int b, float* out) {
  const int lo = ((a & b) == a) ? a : b;
  const int hi = lo ^ a ^ b;
  const int lx = cube & 7, ly = (cube >> 3) & 7, lz = cube >> 6;
  const int at = lz * 81 + ly * 9 + lx;
  const float vlo = val[at + corner_offset(lo)];
  const float vhi = val[at + corner_offset(hi)];
  const float t = __fdiv_rn(vlo, __fsub_rn(vlo, vhi));
  const int g[3] = {bx * kBlockEdge + lx, by * kBlockEdge + ly, bz * kBlockEdge + lz};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float plo = __fmul_rn(__fadd_rn(static_cast<float>(g[k] + ((lo >> k) & 1)), 0.5f), v);
    const float phi = __fmul_rn(__fadd_rn(static_cast<float>(g[k] + ((hi >> k) & 1)), 0.5f), v);
    out[k] = __fadd_rn(plo, __fmul_rn(t, __fsub_rn(phi, plo)));
  }
}

constexpr int kHalo = kTileVals - kBlockVoxels;  // 217 tile points in the 7 upper neighbours

__device__ __forceinline__ float mean_or_nan(float2 s) {
  return s.y > 0.0f ? __fdiv_rn(s.x, s.y) : __int_as_float(0x7fc00000);  // NaN: unobserved
}

// Stage the 9x9x9 tile of means of a block: its own 512 voxels (contiguous
// records, coalesced loads) and the 217 voxels of the faces, edges and corner
// of its upper neighbours (listed in `halo` as tile position << 12 |
// neighbour << 9 | local index). Loads are issued in batches of 8 before any
// is used, so a warp waits for three round trips.
__device__ __forceinline__ void stage_tile(const VolumeArgs& vol, const int* nb,
                                           const unsigned* halo, float* val, unsigned lane) {
  const float4* own = vol.twrg + static_cast<size_t>(nb[0]) * kBlockVoxels;
#pragma unroll
  for (int b0 = 0; b0 < kBlockVoxels / 32; b0 += 8) {
    float2 sum[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      sum[j] = __ldg(reinterpret_cast<const float2*>(own + lane + 32 * (b0 + j)));
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int l = static_cast<int>(lane) + 32 * (b0 + j);
      val[(l >> 6) * 81 + ((l >> 3) & 7) * 9 + (l & 7)] = mean_or_nan(sum[j]);
    }
  }
  constexpr int kPer = (kHalo + 31) / 32;  // 7
  float2 sum[kPer];
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int h = static_cast<int>(lane) + 32 * j;
    sum[j] = make_float2(0.0f, 0.0f);
    if (h < kHalo) {
      const unsigned e = halo[h];
      const int idx = nb[(e >> 9) & 7u];
      if (idx >= 0 && index_ok(idx, vol.pool, &vol.hdr->err))
        sum[j] = __ldg(reinterpret_cast<const float2*>(
            vol.twrg + static_cast<size_t>(idx) * kBlockVoxels + (e & 511u)));
    }
  }
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    const int h = static_cast<int>(lane) + 32 * j;
    if (h < kHalo) val[halo[h] >> 12] = mean_or_nan(sum[j]);
  }
}

__global__ void __launch_bounds__(32 * kExtractWarps, 8)
    extract_kernel(const __grid_constant__ VolumeArgs vol, float v, float* __restrict__ tris,
                   int32_t* __restrict__ cells, unsigned int capacity,
                   unsigned int* __restrict__ counter) {
  __shared__ float s_val[kExtractWarps][kTileVals];
  __shared__ int s_nb[kExtractWarps][8];
  __shared__ float s_stage[kExtractWarps][9 * kExtractStage];
  __shared__ unsigned s_busy[kExtractWarps][kBlockVoxels];
  __shared__ unsigned short s_before[kExtractWarps][kBlockVoxels];
  __shared__ unsigned s_halo[kHalo];
  // the halo points of a tile, in tile order
  if (threadIdx.x == 0) {
    int h = 0;
    for (int i = 0; i < kTileVals; ++i) {
      const int x = i % 9, y = (i / 9) % 9, z = i / 81;
      const int d = (x >> 3) | ((y >> 3) << 1) | ((z >> 3) << 2);
      if (d)
        s_halo[h++] = (static_cast<unsigned>(i) << 12) | (static_cast<unsigned>(d) << 9) |
                      static_cast<unsigned>(local_index(x & 7, y & 7, z & 7));
    }
  }
  __syncthreads();
  const unsigned lane = threadIdx.x & 31u;
  const int warp = threadIdx.x >> 5;
  float* val = s_val[warp];
  int* nb = s_nb[warp];
  float* stage = s_stage[warp];
  unsigned* busy = s_busy[warp];
  unsigned short* before = s_before[warp];
  const unsigned int c = *reinterpret_cast<volatile unsigned int*>(&vol.hdr->count);
  const unsigned int units = vol.slot_index ? vol.slots : (c < vol.pool ? c : vol.pool);
  for (unsigned int unit = blockIdx.x * kExtractWarps + warp; unit < units;
       unit += gridDim.x * kExtractWarps) {
    int bx = 0, by = 0, bz = 0;
    if (vol.slot_index) {
      const unsigned long long key = vol.table[unit].key;   // same address in every lane
      if (key == kEmptyKey) continue;                        // uniform across the warp
      unpack_key(key, bx, by, bz);
    } else {
      bx = vol.coords[3 * static_cast<size_t>(unit)];
      by = vol.coords[3 * static_cast<size_t>(unit) + 1];
      bz = vol.coords[3 * static_cast<size_t>(unit) + 2];
    }
    if (lane < 8) {
      const int d = static_cast<int>(lane);
      int idx = static_cast<int>(unit);
      if (d) {
        const int nx = bx + (d & 1), ny = by + ((d >> 1) & 1), nz = bz + ((d >> 2) & 1);
        // neighbours beyond the key range are absent
        const bool in_range = nx < kKeyBias && ny < kKeyBias && nz < kKeyBias;
        idx = in_range ? lookup_block(vol, pack_key(nx, ny, nz), nx, ny, nz) : kAbsent;
      }
      nb[d] = idx >= 0 ? idx : -1;
    }
    __syncwarp();
    stage_tile(vol, nb, s_halo, val, lane);
    __syncwarp();
    // the cubes that make triangles, listed warp-wide with their inside
    // masks (cube | mask << 9) and the running count of triangles before each
    unsigned nbusy = 0;
    int total = 0;
    for (int j = 0; j < kBlockVoxels / 32; ++j) {
      const int cube = static_cast<int>(lane) + 32 * j;
      const Cube C = load_cube(val, cube, bx, by, bz);
      const int cnt = C.inside ? cube_triangle_count(C.inside) : 0;
      const unsigned m = __ballot_sync(0xffffffffu, cnt > 0);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (static_cast<int>(lane) >= o) incl += y;
      }
      if (cnt > 0) {
        const unsigned at = nbusy + __popc(m & ((1u << lane) - 1u));
        busy[at] = static_cast<unsigned>(cube) | (C.inside << 9);
        before[at] = static_cast<unsigned short>(total + incl - cnt);
      }
      nbusy += __popc(m);
      total += __shfl_sync(0xffffffffu, incl, 31);
    }
    unsigned base = 0;
    if (lane == 0 && total) base = atomicAdd(counter, static_cast<unsigned>(total));
    base = __shfl_sync(0xffffffffu, base, 0);
    __syncwarp();
    if (total && (tris || cells)) {
      // one triangle per lane: find its cube by binary search over the
      // running counts, then its tetrahedron; windows of kExtractStage
      // triangles are staged and stored in coalesced words
      for (unsigned w0 = 0; w0 < static_cast<unsigned>(total); w0 += kExtractStage) {
        const unsigned n = min(static_cast<unsigned>(kExtractStage), total - w0);
        for (unsigned q = lane; q < n; q += 32) {
          const unsigned tri = w0 + q;
          unsigned lo = 0, hi = nbusy;  // last entry with before <= tri
          while (hi - lo > 1) {
            const unsigned mid = (lo + hi) >> 1;
            if (before[mid] <= tri) lo = mid; else hi = mid;
          }
          const unsigned e0 = busy[lo];
          const int cube = static_cast<int>(e0 & 511u);
          int tag, e[6];
          cube_triangle(e0 >> 9, static_cast<int>(tri - before[lo]), tag, e);
          const unsigned pos = base + tri;
          if (tris) {
            float* o = stage + 9 * q;
            tile_edge_vertex(val, cube, bx, by, bz, v, e[0], e[1], o);
            tile_edge_vertex(val, cube, bx, by, bz, v, e[2], e[3], o + 3);
            tile_edge_vertex(val, cube, bx, by, bz, v, e[4], e[5], o + 6);
          }
          if (cells && pos < capacity)
            reinterpret_cast<int4*>(cells)[pos] =
                make_int4(bx * kBlockEdge + (cube & 7), by * kBlockEdge + ((cube >> 3) & 7),
                          bz * kBlockEdge + (cube >> 6), tag);
        }
        __syncwarp();
        if (tris) {
          const size_t o0 = 9 * (static_cast<size_t>(base) + w0);
          const size_t ocap = 9 * static_cast<size_t>(capacity);
          for (unsigned w = lane; w < 9 * n; w += 32)
            if (o0 + w < ocap) tris[o0 + w] = stage[w];
        }
        __syncwarp();
      }
    }
    __syncwarp();  // the tile, neighbour list and staging are reused
  }
}

// ----------------------------------------------------------------------------
// warp kernels: barrier-free stage A / stage B / fused
// ----------------------------------------------------------------------------
// Each warp covers an 8x4 pixel patch and works alone: its lanes walk their
// bands, the warp dedupes the first three distinct blocks of every point with
// __match_any_sync, compacts the leaders' keys of all three rounds into lanes
// 0..n-1, resolves them in one warp-cooperative pass (insert without waiting,
// look up, or insert and obtain the index), and shuffles the indices back to
// every lane that needs them. Stage B and the fused kernel then add five sums
// per accepted voxel straight to the pool. No shared memory, no barriers:
// occupancy is bounded by registers alone, and every warp overlaps its global
// round trips with other warps' walks.
template <int Op, int P>
__device__ __forceinline__ int warp_resolve(const VolumeArgs& vol, unsigned long long key,
                                            bool has) {
  if (Op == kOpAllocate) {
    warp_insert_nowait<P>(vol, key, has);
    return -1;
  }
  if (Op == kOpFused) return warp_insert_get<P>(vol, key, has);
  if (!has) return -1;
  int bx, by, bz;
  unpack_key(key, bx, by, bz);
  return resolve_for_update(vol, lookup_block(vol, key, bx, by, bz));
}

// A point's accepted voxel after phase 1, packed: local index (9 bits), which
// of the point's first three blocks it lies in (2 bits), valid flag.
constexpr unsigned kPackValid = 1u << 11;

// A fourth or later block of one point (rare): handled by its own thread at
// once -- inserted (stage A), or resolved and its voxel added (stage B, fused).
template <int Op, int P>
__device__ __noinline__ void extra_block_voxel(const FrameArgs& f, const VolumeArgs& vol,
                                               unsigned long long key, int l, float t,
                                               int pu, int pv) {
  const int idx = resolve_single<Op, P>(vol, key);
  if (Op == kOpAllocate) return;
  const bool colour = f.rgb != nullptr;
  float cr = 0.0f, cg = 0.0f, cb = 0.0f;
  if (colour) load_colour(f, pu, pv, cr, cg, cb);
  add_voxel_direct(vol, idx, l, t, colour, cr, cg, cb);
}

template <int Op, int P, int M>
__device__ __forceinline__ void warp_body(const FrameArgs& f, const VolumeArgs& vol, int tile,
                                          int tiles_x) {
  if (load_err_volatile(vol.hdr)) return;  // poisoned volume: do nothing
  const unsigned lane = threadIdx.x & 31u;
  int u, v;
  tile_pixel(tile, tiles_x, u, v);
  Ray r;
  const bool valid =
      u < f.W && v < f.H && make_ray(f, u, v, load_depth(f, static_cast<long long>(v) * f.W + u), r);

  // phase 1: walk; the point's first three distinct accepted blocks; every
  // accepted voxel packed as (local index, block slot) with its tsdf value
  constexpr int K = M > 0 ? 2 * M + 1 : 1;
  unsigned pack[K];
  float tv[K];
  unsigned long long key[3] = {kEmptyKey, kEmptyKey, kEmptyKey};
  unsigned long long last = kEmptyKey;
  int nk = 0;
  auto take = [&](unsigned long long kk, int l, float t) -> unsigned {
    if (kk != last) {
      last = kk;
      if (nk == 0)
        key[0] = kk;
      else if (nk == 1)
        key[1] = kk;
      else if (nk == 2)
        key[2] = kk;
      ++nk;
    }
    if (kk == key[0]) return kPackValid | static_cast<unsigned>(l);
    if (kk == key[1]) return kPackValid | (1u << 9) | static_cast<unsigned>(l);
    if (kk == key[2]) return kPackValid | (2u << 9) | static_cast<unsigned>(l);
    extra_block_voxel<Op, P>(f, vol, kk, l, t, u, v);
    return 0u;
  };
  if constexpr (M > 0) {
    if (valid) {
      Walk<M> w;
      const unsigned acc = walk_point<M>(f, r, w);
#pragma unroll
      for (int k = 0; k < K; ++k) {
        pack[k] = 0u;
        tv[k] = 0.0f;
        if ((acc >> k) & 1u) {
          tv[k] = tsdf_value(f, r.d, w.zc[k]);
          pack[k] = take(block_key_of(w.gx[k], w.gy[k], w.gz[k]),
                         local_index(w.gx[k], w.gy[k], w.gz[k]), tv[k]);
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        pack[k] = 0u;
        tv[k] = 0.0f;
      }
    }
  } else if (valid) {
    // generic half band: keys only here, voxels are re-walked in phase 3
    WalkDedupe walk;
    for (int k = 0; k <= 2 * f.M; ++k) {
      int gx, gy, gz;
      float zc;
      if (!sample_voxel(f, r, k, gx, gy, gz)) continue;
      const unsigned long long kk = block_key_of(gx, gy, gz);
      if (Op == kOpAllocate) {
        if (kk == last) continue;
      } else if (walk.seen_then_push(gx, gy, gz)) {
        continue;
      }
      if (!voxel_test(f, gx, gy, gz, zc)) continue;
      if (kk == last) continue;
      last = kk;
      if (nk == 0)
        key[0] = kk;
      else if (nk == 1)
        key[1] = kk;
      else if (nk == 2)
        key[2] = kk;
      else if (Op == kOpAllocate)
        resolve_single<kOpAllocate, P>(vol, kk);
      ++nk;
    }
  }

  // phase 2: warp dedupe of each round, compaction of the leaders, one
  // cooperative resolution, indices back to every lane
  unsigned leaders[3], leader_of[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const bool has = nk > j;
    const unsigned m = __ballot_sync(0xffffffffu, has);
    unsigned peers = 0;
    if (has) peers = __match_any_sync(m, key[j]);
    leader_of[j] = has ? static_cast<unsigned>(__ffs(peers) - 1) : 0u;
    leaders[j] = __ballot_sync(0xffffffffu, has && leader_of[j] == lane);
  }
  const int n0 = __popc(leaders[0]), n1 = __popc(leaders[1]), n2 = __popc(leaders[2]);
  const int n = n0 + n1 + n2;
  int idx[3] = {-1, -1, -1};
  int c_of[3];  // compact index of the entry that resolves this lane's key j
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const int base = j == 0 ? 0 : (j == 1 ? n0 : n0 + n1);
    c_of[j] = base + __popc(leaders[j] & ((1u << leader_of[j]) - 1u));
  }
  for (int chunk = 0; chunk < n; chunk += 32) {
    const int c = chunk + static_cast<int>(lane);
    const bool has = c < n;
    int j = 2, rank = c - n0 - n1;
    if (c < n0) {
      j = 0;
      rank = c;
    } else if (c < n0 + n1) {
      j = 1;
      rank = c - n0;
    }
    const unsigned src0 = __fns(leaders[0], 0, (j == 0 && has ? rank : 0) + 1);
    const unsigned src1 = __fns(leaders[1], 0, (j == 1 && has ? rank : 0) + 1);
    const unsigned src2 = __fns(leaders[2], 0, (j == 2 && has ? rank : 0) + 1);
    const unsigned long long g0 = __shfl_sync(0xffffffffu, key[0], src0 & 31u);
    const unsigned long long g1 = __shfl_sync(0xffffffffu, key[1], src1 & 31u);
    const unsigned long long g2 = __shfl_sync(0xffffffffu, key[2], src2 & 31u);
    const unsigned long long mine = j == 0 ? g0 : (j == 1 ? g1 : g2);
    const int res = warp_resolve<Op, P>(vol, has ? mine : kEmptyKey, has);
    if (Op != kOpAllocate) {
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        const int cj = c_of[jj] - chunk;
        const int got = __shfl_sync(0xffffffffu, res, cj & 31);
        if (nk > jj && cj >= 0 && cj < 32) idx[jj] = got;
      }
    }
  }
  if (Op == kOpAllocate || !valid) return;

  // phase 3: five sums per accepted voxel
  float cr = 0.0f, cg = 0.0f, cb = 0.0f;
  const bool colour = f.rgb != nullptr;
  if (colour) {
    load_colour(f, u, v, cr, cg, cb);
  }
  if constexpr (M > 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (pack[k] & kPackValid) {
        const unsigned slot = (pack[k] >> 9) & 3u;
        const int id = slot == 0 ? idx[0] : (slot == 1 ? idx[1] : idx[2]);
        add_voxel_direct(vol, id, static_cast<int>(pack[k] & 511u), tv[k], colour, cr, cg, cb);
      }
    }
  } else {
    WalkDedupe walk;
    BlockCacheT slow;
    for (int k = 0; k <= 2 * f.M; ++k) {
      int gx, gy, gz;
      float zc;
      if (!sample_voxel(f, r, k, gx, gy, gz) || walk.seen_then_push(gx, gy, gz) ||
          !voxel_test(f, gx, gy, gz, zc))
        continue;
      const unsigned long long kk = block_key_of(gx, gy, gz);
      int id;
      if (kk == key[0]) {
        id = idx[0];
      } else if (kk == key[1]) {
        id = idx[1];
      } else if (kk == key[2]) {
        id = idx[2];
      } else {
        if (kk != slow.key) {
          slow.key = kk;
          slow.idx = resolve_single<Op, P>(vol, kk);
        }
        id = slow.idx;
      }
      add_voxel_direct(vol, id, local_index(gx, gy, gz), tsdf_value(f, r.d, zc), colour, cr, cg,
                       cb);
    }
  }
}

// MinBlocks: the CTAs per SM the register allocation must allow.
template <int Op, int P, int M, int MinBlocks>
__global__ void __launch_bounds__(kThreads, MinBlocks)
    warp_kernel(const __grid_constant__ FrameArgs f, const __grid_constant__ VolumeArgs vol,
                int tiles_x) {
  warp_body<Op, P, M>(f, vol, blockIdx.x, tiles_x);
}

template <int Op, int P>
static cudaError_t launch_warp_m(const FrameArgs& f, const VolumeArgs& vol, cudaStream_t s) {
  const int tx = tiles_of(f.W);
  const int tiles = tx * tiles_of(f.H);
  switch (f.M) {
    case 2: warp_kernel<Op, P, 2, 1><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
    case 4: warp_kernel<Op, P, 4, 1><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
    case 8: warp_kernel<Op, P, 8, 1><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
    default: warp_kernel<Op, P, 0, 1><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
  }
  return cudaGetLastError();
}

template <int Op>
static cudaError_t launch_warp_p(const FrameArgs& f, const VolumeArgs& vol, int probe_load,
                                 cudaStream_t s) {
  switch (probe_load) {
    case kLoadL2: return launch_warp_m<Op, kLoadL2>(f, vol, s);
    case kLoadRelaxed: return launch_warp_m<Op, kLoadRelaxed>(f, vol, s);
    default: return launch_warp_m<Op, kLoadCached>(f, vol, s);
  }
}

// ----------------------------------------------------------------------------
// batched kernels: many frames (one per volume) in one launch
// ----------------------------------------------------------------------------
// The grid is persistent (a multiple of the SM count, fixed per kernel, so a
// CUDA graph of the launch stays valid for any batch); CTAs walk the global
// tile numbering of all frames, find each tile's frame by binary search over
// the frames' first tiles, and run the single-frame tile body on it with the
// frame's arguments staged in shared memory.
__device__ __forceinline__ int find_session(const SessionArgs* S, int n, int tile) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (S[mid].tile_begin <= tile)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void load_session(SessionArgs& dst, const SessionArgs* src) {
  constexpr int kWords = sizeof(SessionArgs) / 4;
  for (int i = threadIdx.x; i < kWords; i += blockDim.x)
    reinterpret_cast<int*>(&dst)[i] = reinterpret_cast<const int*>(src)[i];
}

template <int P>
__global__ void __launch_bounds__(kThreads)
    batch_tile_allocate_kernel(const BatchHeader* __restrict__ table) {
  __shared__ TileShared T;
  __shared__ SessionArgs sa;
  __shared__ int s_sess;
  const int n = table->n;
  const int total = table->total_tiles;
  const SessionArgs* S = reinterpret_cast<const SessionArgs*>(table + 1);
  int cur = -1;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    if (threadIdx.x == 0) s_sess = find_session(S, n, tile);
    __syncthreads();
    const int s = s_sess;
    if (s != cur) {
      load_session(sa, S + s);
      cur = s;
    }
    __syncthreads();
    if (sa.f.M == 4)
      tile_allocate_body<P, 4>(T, sa.f, sa.vol, tile - sa.tile_begin, sa.tiles_x);
    else
      tile_allocate_body<P, 0>(T, sa.f, sa.vol, tile - sa.tile_begin, sa.tiles_x);
  }
}

// MF: 4 when every frame of the batch has half band M = 4 (the common case:
// the body is then compiled for that band alone, with fewer registers), else
// 0 and each tile dispatches on its frame's band.
template <int P, int MF>
__global__ void __launch_bounds__(kThreads, 4)
    batch_tile_fused_kernel(const BatchHeader* __restrict__ table) {
  __shared__ FusedTileShared S;
  __shared__ SessionArgs sa;
  __shared__ int s_sess;
  const int n = table->n;
  const int total = table->total_tiles;
  const SessionArgs* Sa = reinterpret_cast<const SessionArgs*>(table + 1);
  int cur = -1;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    if (threadIdx.x == 0) s_sess = find_session(Sa, n, tile);
    __syncthreads();
    const int s = s_sess;
    if (s != cur) {
      load_session(sa, Sa + s);
      cur = s;
    }
    __syncthreads();
    if (MF == 4 || sa.f.M == 4)
      tile_fused_body<P, 4>(S, sa.f, sa.vol, tile - sa.tile_begin, sa.tiles_x);
    else
      tile_fused_body<P, 0>(S, sa.f, sa.vol, tile - sa.tile_begin, sa.tiles_x);
    __syncthreads();  // S, sa and s_sess are rewritten for the next tile
  }
}

// Kind: kBatchScatter (stage B, paper's update), or a warp_body operation.
constexpr int kBatchScatter = 10;

template <int Kind, int P>
__global__ void __launch_bounds__(kThreads) batch_point_kernel(const BatchHeader* __restrict__ table) {
  __shared__ SessionArgs sa;
  __shared__ int s_sess;
  const int n = table->n;
  const int total = table->total_tiles;
  const SessionArgs* S = reinterpret_cast<const SessionArgs*>(table + 1);
  int cur = -1;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    if (threadIdx.x == 0) s_sess = find_session(S, n, tile);
    __syncthreads();
    const int s = s_sess;
    if (s != cur) {
      load_session(sa, S + s);
      cur = s;
    }
    __syncthreads();
    const int local = tile - sa.tile_begin;
    if constexpr (Kind == kBatchScatter) {
      if (sa.f.M == 4)
        scatter_body<4>(sa.f, sa.vol, local, sa.tiles_x);
      else
        scatter_body<0>(sa.f, sa.vol, local, sa.tiles_x);
    } else {
      if (sa.f.M == 4)
        warp_body<Kind, P, 4>(sa.f, sa.vol, local, sa.tiles_x);
      else
        warp_body<Kind, P, 0>(sa.f, sa.vol, local, sa.tiles_x);
    }
    __syncthreads();  // sa and s_sess are rewritten by the next tile
  }
}

// Each frame's sticky error word, gathered for one device-to-host copy.
__global__ void batch_status_kernel(const BatchHeader* __restrict__ table, unsigned* out) {
  const SessionArgs* S = reinterpret_cast<const SessionArgs*>(table + 1);
  for (int i = threadIdx.x; i < table->n; i += blockDim.x) out[i] = load_err_volatile(S[i].vol.hdr);
}

template <int P, int M>
static cudaError_t launch_tile_kernel(const FrameArgs& f, const VolumeArgs& vol,
                                      cudaStream_t s) {
  const int tx = tiles_of(f.W);
  tile_allocate_kernel<P, M><<<tx * tiles_of(f.H), kThreads, 0, s>>>(f, vol, tx);
  return cudaGetLastError();
}

template <int P>
static cudaError_t launch_tile_m(const FrameArgs& f, const VolumeArgs& vol, cudaStream_t s) {
  switch (f.M) {
    case 2: return launch_tile_kernel<P, 2>(f, vol, s);
    case 4: return launch_tile_kernel<P, 4>(f, vol, s);
    case 8: return launch_tile_kernel<P, 8>(f, vol, s);
    default: return launch_tile_kernel<P, 0>(f, vol, s);
  }
}

static cudaError_t launch_tile_p(const FrameArgs& f, const VolumeArgs& vol, int probe_load,
                                 cudaStream_t s) {
  switch (probe_load) {
    case kLoadL2: return launch_tile_m<kLoadL2>(f, vol, s);
    case kLoadRelaxed: return launch_tile_m<kLoadRelaxed>(f, vol, s);
    default: return launch_tile_m<kLoadCached>(f, vol, s);
  }
}

cudaError_t launch_allocate(const FrameArgs& f, const VolumeArgs& vol, int probe_load, int mode,
                            cudaStream_t s) {
  const int tx = tiles_of(f.W);
  const int tiles = tx * tiles_of(f.H);
  cudaError_t e = cudaSuccess;
  if (mode == 0) {
    switch (probe_load) {
      case kLoadL2: allocate_kernel<kLoadL2><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
      case kLoadRelaxed:
        allocate_kernel<kLoadRelaxed><<<tiles, kThreads, 0, s>>>(f, vol, tx);
        break;
      default: allocate_kernel<kLoadCached><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
    }
    e = cudaGetLastError();
  } else if (mode == 1) {
    e = launch_tile_p(f, vol, probe_load, s);
  } else {
    e = launch_warp_p<kOpAllocate>(f, vol, probe_load, s);
  }
  note_launch();
  return e;
}

cudaError_t launch_integrate(const FrameArgs& f, const VolumeArgs& vol, int mode,
                             cudaStream_t s) {
  const int tx = tiles_of(f.W);
  const int tiles = tx * tiles_of(f.H);
  cudaError_t e = cudaSuccess;
  if (mode == 0) {
    switch (f.M) {
      case 2: integrate_scatter_kernel<2><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
      case 4: integrate_scatter_kernel<4><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
      case 8: integrate_scatter_kernel<8><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
      default: integrate_scatter_kernel<0><<<tiles, kThreads, 0, s>>>(f, vol, tx); break;
    }
    e = cudaGetLastError();
  } else if (mode == 1) {
    e = launch_warp_m<kOpIntegrate, kLoadCached>(f, vol, s);
  } else {
    e = launch_integrate_tile(f, vol, s);
  }
  note_launch();
  return e;
}

template <int P, int M>
static cudaError_t launch_tile_fused_kernel(const FrameArgs& f, const VolumeArgs& vol,
                                            int mode, cudaStream_t s) {
  (void)mode;
  const int tx = tiles_of(f.W);
  tile_fused_kernel<P, M><<<tx * tiles_of(f.H), kThreads, 0, s>>>(f, vol, tx);
  return cudaGetLastError();
}

template <int P>
static cudaError_t launch_tile_fused_m(const FrameArgs& f, const VolumeArgs& vol, int mode,
                                       cudaStream_t s) {
  switch (f.M) {
    case 2: return launch_tile_fused_kernel<P, 2>(f, vol, mode, s);
    case 4: return launch_tile_fused_kernel<P, 4>(f, vol, mode, s);
    case 8: return launch_tile_fused_kernel<P, 8>(f, vol, mode, s);
    default: return launch_tile_fused_kernel<P, 0>(f, vol, mode, s);
  }
}

cudaError_t launch_fused(const FrameArgs& f, const VolumeArgs& vol, int probe_load, int mode,
                         int threads_per_point, cudaStream_t s) {
  if (threads_per_point != 1) {
    if (mode != 2 || probe_load != kLoadCached) return cudaErrorInvalidValue;
    return launch_fused_split(f, vol, threads_per_point, s);
  }
  cudaError_t e;
  if (mode == 2) {
    switch (probe_load) {
      case kLoadL2: e = launch_tile_fused_m<kLoadL2>(f, vol, mode, s); break;
      case kLoadRelaxed: e = launch_tile_fused_m<kLoadRelaxed>(f, vol, mode, s); break;
      default: e = launch_tile_fused_m<kLoadCached>(f, vol, mode, s); break;
    }
  } else {
    e = launch_warp_p<kOpFused>(f, vol, probe_load, s);
  }
  note_launch();
  return e;
}

// Persistent grid of a batched kernel: resident CTAs per SM x SMs, looked up
// once per kernel (so no runtime query runs while a launch is being captured).
template <typename K>
static int persistent_grid(K kernel, int factor) {
  struct Shape {
    int sms = 0, occ = 0;
  };
  // One per kernel instantiation, computed once (thread-safe static
  // initialisation) for the device current at the first call; a zero shape
  // (a failed query) makes the launch fail with an invalid configuration.
  static const Shape shape = [kernel]() {
    Shape sh;
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return sh;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return sh;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kThreads, 0) != cudaSuccess)
      return sh;
    sh.occ = occ < 1 ? 1 : occ;
    sh.sms = sms;
    return sh;
  }();
  const int occ = (factor > 0 && factor < shape.occ) ? factor : shape.occ;
  return occ * shape.sms;
}

template <typename K>
static cudaError_t launch_persistent(K kernel, const BatchHeader* table, int factor,
                                     int grid_limit, cudaStream_t s) {
  int grid = persistent_grid(kernel, factor);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  if (grid_limit > 0 && grid_limit < grid) grid = grid_limit;
  kernel<<<grid, kThreads, 0, s>>>(table);
  return cudaGetLastError();
}

template <int P>
static cudaError_t launch_batch_fused(const BatchHeader* table, bool all_m4, int factor,
                                      int grid_limit, cudaStream_t s) {
  if (all_m4) return launch_persistent(batch_tile_fused_kernel<P, 4>, table, factor, grid_limit, s);
  return launch_persistent(batch_tile_fused_kernel<P, 0>, table, factor, grid_limit, s);
}

cudaError_t launch_batch(const BatchHeader* table, int probe_load, int allocate_mode,
                         int integrate_mode, int fuse_mode, int factor, int grid_limit,
                         bool all_m4, int stages, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (fuse_mode == 2) {
    switch (probe_load) {
      case kLoadL2: return launch_batch_fused<kLoadL2>(table, all_m4, factor, grid_limit, s);
      case kLoadRelaxed: return launch_batch_fused<kLoadRelaxed>(table, all_m4, factor, grid_limit, s);
      default: return launch_batch_fused<kLoadCached>(table, all_m4, factor, grid_limit, s);
    }
  }
  if (fuse_mode == 1) {
    switch (probe_load) {
      case kLoadL2: return launch_persistent(batch_point_kernel<kOpFused, kLoadL2>, table, factor, grid_limit, s);
      case kLoadRelaxed:
        return launch_persistent(batch_point_kernel<kOpFused, kLoadRelaxed>, table, factor, grid_limit, s);
      default:
        return launch_persistent(batch_point_kernel<kOpFused, kLoadCached>, table, factor, grid_limit, s);
    }
  }
  if (!(stages & 1)) {
    // stage B alone
  } else if (allocate_mode == 2) {
    switch (probe_load) {
      case kLoadL2:
        e = launch_persistent(batch_point_kernel<kOpAllocate, kLoadL2>, table, factor, grid_limit, s);
        break;
      case kLoadRelaxed:
        e = launch_persistent(batch_point_kernel<kOpAllocate, kLoadRelaxed>, table, factor, grid_limit, s);
        break;
      default:
        e = launch_persistent(batch_point_kernel<kOpAllocate, kLoadCached>, table, factor, grid_limit, s);
        break;
    }
  } else {
    switch (probe_load) {
      case kLoadL2: e = launch_persistent(batch_tile_allocate_kernel<kLoadL2>, table, factor, grid_limit, s); break;
      case kLoadRelaxed:
        e = launch_persistent(batch_tile_allocate_kernel<kLoadRelaxed>, table, factor, grid_limit, s);
        break;
      default:
        e = launch_persistent(batch_tile_allocate_kernel<kLoadCached>, table, factor, grid_limit, s);
        break;
    }
  }
  if (e != cudaSuccess || !(stages & 2)) return e;
  if (integrate_mode == 1)
    return launch_persistent(batch_point_kernel<kOpIntegrate, kLoadCached>, table, factor, grid_limit, s);
  return launch_persistent(batch_point_kernel<kBatchScatter, kLoadCached>, table, factor, grid_limit, s);
}

cudaError_t launch_batch_status(const BatchHeader* table, unsigned* out, cudaStream_t s) {
  batch_status_kernel<<<1, 256, 0, s>>>(table, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_export(const VolumeArgs& vol, float* out, unsigned int n,
                          const unsigned int* list, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t total = static_cast<size_t>(n) * kBlockVoxels;
  const unsigned int grid = static_cast<unsigned int>((total + 255) / 256 < 65535 * 4
                                                          ? (total + 255) / 256
                                                          : 65535 * 4);
  export_kernel<<<grid, 256, 0, s>>>(vol, out, n, list);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_slot_list(const VolumeArgs& vol, unsigned int* list, int32_t* coords,
                             unsigned int cap, unsigned int* found, cudaStream_t s) {
  slot_list_kernel<<<1, kListThreads, 0, s>>>(vol, list, coords, cap, found);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_clear_used(const VolumeArgs& vol, int sm_count, cudaStream_t s) {
  if (vol.slot_index)
    clear_slots_kernel<<<sm_count * 8, 256, 0, s>>>(vol);
  else
    clear_used_kernel<<<sm_count * 8, 256, 0, s>>>(vol);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_extract(const VolumeArgs& vol, float v, float* tris, int32_t* cells,
                           unsigned int capacity, unsigned int* counter, int sm_count,
                           cudaStream_t s) {
  // persistent: every warp loops over blocks; 8 CTAs of 4 warps per SM
  extract_kernel<<<sm_count * 8, 32 * kExtractWarps, 0, s>>>(vol, v, tris, cells, capacity,
                                                            counter);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_table_stats(const VolumeArgs& vol, TableStatsDev* out, int sm_count,
                               cudaStream_t s) {
  table_stats_kernel<<<sm_count * 4, 256, 0, s>>>(vol, out);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  weight_sum_kernel<<<sm_count * 8, 256, 0, s>>>(vol, out);
  note_launch();
  return cudaGetLastError();
}

}  // namespace tsdf
