// The tile machinery shared by the kernel translation units: launch shape
// constants, the shared-memory key set and list of a pixel tile, the point
// walk's key collection, and the tile kernels of stage A and of the fused
// path (paper Section 2.2; the fused kernel's phases are described at
// tile_fused_body).
#pragma once

#include <cstdint>

#include "tsdf_device.cuh"

namespace tsdf {

constexpr int kThreads = 256;
constexpr int kTile = 16;
constexpr int kSetSlots = 2048;    // allocate_kernel: per-CTA key set (16 KB)
constexpr int kTileSet = 1024;     // tile kernel: key set slots (8 KB)
constexpr int kTileList = 768;     // tile kernel: compact key list (6 KB)

// Pixel of this thread in tile `tile`: a tile is 16 pixels wide and
// blockDim.x / 16 rows high; warp w covers the 8x4 patch (w & 1, w >> 1).
__device__ __forceinline__ void tile_pixel(int tile, int tiles_x, int& u, int& v) {
  const int tx = tile % tiles_x;
  const int ty = tile / tiles_x;
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  u = tx * kTile + (w & 1) * 8 + (lane & 7);
  v = ty * static_cast<int>(blockDim.x >> 4) + (w >> 1) * 4 + (lane >> 3);
}

// Insert into the CTA's shared-memory key set; false if the set is full.
__device__ __forceinline__ bool set_insert(unsigned long long* set, unsigned long long key,
                                           unsigned int h) {
  for (int i = 0; i < kSetSlots; ++i) {
    const unsigned int s = (h + i) & (kSetSlots - 1);
    const unsigned long long prev = atomicCAS(&set[s], kEmptyKey, key);
    if (prev == kEmptyKey || prev == key) return true;
  }
  return false;
}

// Walk state of one point for the generic loop: the last two in-range voxels.
struct WalkDedupe {
  int ax = INT_MIN, ay = 0, az = 0, bx = INT_MIN, by = 0, bz = 0;
  __device__ __forceinline__ bool seen_then_push(int x, int y, int z) {
    if ((x == ax && y == ay && z == az) || (x == bx && y == by && z == bz)) return true;
    bx = ax; by = ay; bz = az;
    ax = x; ay = y; az = z;
    return false;
  }
};

__device__ __forceinline__ unsigned long long block_key_of(int gx, int gy, int gz) {
  return pack_key(gx >> 3, gy >> 3, gz >> 3);
}

// ----------------------------------------------------------------------------
// stage A, the paper's protocol (Listing 1 per sample, waits for publication)
// ----------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(kThreads)
    allocate_kernel(const __grid_constant__ FrameArgs f, const __grid_constant__ VolumeArgs vol,
                    int tiles_x) {
  __shared__ unsigned long long s_set[kSetSlots];
  __shared__ unsigned int s_err;
  if (threadIdx.x == 0) s_err = load_err_volatile(vol.hdr);
  for (int i = threadIdx.x; i < kSetSlots; i += kThreads) s_set[i] = kEmptyKey;
  __syncthreads();
  if (s_err) return;  // poisoned volume: do nothing

  int u, v;
  tile_pixel(blockIdx.x, tiles_x, u, v);
  Ray r;
  bool valid = false;
  if (u < f.W && v < f.H)
    valid = make_ray(f, u, v, load_depth(f, static_cast<long long>(v) * f.W + u), r);
  const int lane = threadIdx.x & 31;
  unsigned long long last_key = kEmptyKey;
  WalkDedupe walk;
  for (int k = 0; k <= 2 * f.M; ++k) {
    bool cand = false;
    unsigned long long key = kEmptyKey;
    int bx = 0, by = 0, bz = 0;
    if (valid) {
      int gx, gy, gz;
      float zc;
      if (sample_voxel(f, r, k, gx, gy, gz) && !walk.seen_then_push(gx, gy, gz) &&
          voxel_test(f, gx, gy, gz, zc)) {
        bx = gx >> 3;
        by = gy >> 3;
        bz = gz >> 3;
        key = pack_key(bx, by, bz);
        if (key != last_key) {
          cand = true;
          last_key = key;
        }
      }
    }
    // warp-level dedupe before any compare-exchange
    const unsigned int m = __ballot_sync(0xffffffffu, cand);
    if (cand) {
      const unsigned int peers = __match_any_sync(m, key);
      if (lane == __ffs(peers) - 1) {
        if (!set_insert(s_set, key, hash_block(bx, by, bz))) insert_block<P>(vol, key, bx, by, bz);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSetSlots; i += kThreads) {
    const unsigned long long key = s_set[i];
    if (key != kEmptyKey) {
      int bx, by, bz;
      unpack_key(key, bx, by, bz);
      insert_block<P>(vol, key, bx, by, bz);
    }
  }
}

// One-entry cache of a resolved block.
struct BlockCacheT {
  unsigned long long key = kEmptyKey;
  int idx = -1;
};

// ----------------------------------------------------------------------------
// tile machinery shared by the tile kernels (stage A, stage B, fused)
// ----------------------------------------------------------------------------
// The distinct block keys of a 16x16 pixel tile live in a shared-memory set;
// the first thread to add a key appends it to a compact list. Each warp then
// resolves (inserts or looks up) the keys it appended in one warp-cooperative
// pass, so no CTA-wide barrier waits on a global round trip.
struct TileShared {
  unsigned long long set[kTileSet];
  unsigned long long list[kTileList];
  short pos[kTileSet];                 // list position of set[s], -1 if it did not fit
  int n;
  unsigned int err;
};

__device__ __forceinline__ unsigned int tile_hash(unsigned long long key) {
  return static_cast<unsigned int>((key * 0x9E3779B97F4A7C15ull) >> 40);
}

// Add a key. Returns its list position when this call appended it, -1 when it
// could not be listed (set or list full), -2 when it was already present.
__device__ __forceinline__ int tile_add(TileShared& T, unsigned long long key) {
  const unsigned int h = tile_hash(key);
  for (int i = 0; i < kTileSet; ++i) {
    const unsigned int s = (h + i) & (kTileSet - 1);
    const unsigned long long prev = atomicCAS(&T.set[s], kEmptyKey, key);
    if (prev == kEmptyKey) {
      int p = atomicAdd(&T.n, 1);
      if (p < kTileList)
        T.list[p] = key;
      else
        p = -1;
      T.pos[s] = static_cast<short>(p);
      return p;
    }
    if (prev == key) return -2;
  }
  return -1;
}

// List position of a key after the set is complete (after a barrier); -1 if
// the key is not listed.
__device__ __forceinline__ int tile_find(const TileShared& T, unsigned long long key) {
  const unsigned int h = tile_hash(key);
  for (int i = 0; i < kTileSet; ++i) {
    const unsigned int s = (h + i) & (kTileSet - 1);
    const unsigned long long k = T.set[s];
    if (k == key) return T.pos[s];
    if (k == kEmptyKey) return -1;
  }
  return -1;
}

// Distinct accepted blocks of one point, in walk order: up to three in
// registers, any further ones straight into the tile set.
struct PointKeys {
  unsigned long long k0 = kEmptyKey, k1 = kEmptyKey, k2 = kEmptyKey, last = kEmptyKey;
  int n = 0;
};

enum TileOp { kOpAllocate = 0, kOpIntegrate = 1, kOpFused = 2 };

// Resolve one key on its own (paths that could not use the tile list: rare,
// so kept out of line to keep the kernels' hot code small).
template <int Op, int P>
__device__ __noinline__ int resolve_single(const VolumeArgs& vol, unsigned long long key) {
  int bx, by, bz;
  unpack_key(key, bx, by, bz);
  if (Op == kOpAllocate) return insert_block<P, false>(vol, key, bx, by, bz);
  if (Op == kOpFused) return insert_block<P, true>(vol, key, bx, by, bz);
  return resolve_for_update(vol, lookup_block(vol, key, bx, by, bz));
}

template <int Op, int P>
__device__ __forceinline__ void point_key(PointKeys& pk, unsigned long long key, TileShared& T,
                                          const VolumeArgs& vol) {
  if (key == pk.last) return;
  pk.last = key;
  if (pk.n == 0) {
    pk.k0 = key;
  } else if (pk.n == 1) {
    pk.k1 = key;
  } else if (pk.n == 2) {
    pk.k2 = key;
  } else {
    // a fourth or later block of one point: rare; resolved by this thread
    if (tile_add(T, key) == -1) resolve_single<Op, P>(vol, key);
  }
  pk.n++;
}

__device__ __forceinline__ void tile_init(TileShared& T, const VolumeArgs& vol) {
  if (threadIdx.x == 0) {
    T.err = load_err_volatile(vol.hdr);
    T.n = 0;
  }
  for (int i = threadIdx.x; i < kTileSet; i += blockDim.x) T.set[i] = kEmptyKey;
}

// Pixel of this thread when TPP consecutive threads share one point: a tile
// is 16 pixels wide and blockDim.x / (16 TPP) rows high, and the points of a
// warp lie along one tile row.
template <int TPP>
__device__ __forceinline__ void tile_pixel_shared(int tile, int tiles_x, int& u, int& v) {
  const int tx = tile % tiles_x;
  const int ty = tile / tiles_x;
  const int p = static_cast<int>(threadIdx.x) / TPP;
  u = tx * kTile + (p & 15);
  v = ty * static_cast<int>(blockDim.x / (16 * TPP)) + (p >> 4);
}

// The thread's point (every thread of a point builds the same ray).
template <int TPP = 1>
__device__ __forceinline__ bool tile_ray(const FrameArgs& f, int tile, int tiles_x, Ray& r, int& u,
                                         int& v) {
  if constexpr (TPP == 1)
    tile_pixel(tile, tiles_x, u, v);
  else
    tile_pixel_shared<TPP>(tile, tiles_x, u, v);
  if (u >= f.W || v >= f.H) return false;
  return make_ray(f, u, v, load_depth(f, static_cast<long long>(v) * f.W + u), r);
}

// Pixel rows of one tile of a kernel whose points have TPP threads each.
template <int TPP>
constexpr int tile_rows() {
  return kThreads / (kTile * TPP);
}

// Each point's first three distinct blocks into the tile's key list, after a
// per-warp __match_any_sync dedupe. Every lane of the warp calls it.
template <int Op, int P>
__device__ __forceinline__ void tile_list_point_keys(TileShared& T, const VolumeArgs& vol,
                                                     const PointKeys& pk) {
  const unsigned lane = threadIdx.x & 31u;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const unsigned long long key = j == 0 ? pk.k0 : (j == 1 ? pk.k1 : pk.k2);
    const bool has = pk.n > j;
    const unsigned m = __ballot_sync(0xffffffffu, has);
    if (has) {
      const unsigned peers = __match_any_sync(m, key);
      if (lane == static_cast<unsigned>(__ffs(peers) - 1)) {
        // a key that cannot be listed is inserted by its adder at once
        if (tile_add(T, key) == -1) resolve_single<Op, P>(vol, key);
      }
    }
  }
}

// Phases 1 and 2 of every tile kernel: the point's walk and its distinct
// accepted blocks; a per-warp __match_any_sync dedupe of each point's first
// three blocks before the tile set; then each warp resolves the keys it
// appended to the tile list, warp-cooperatively (stage A: insert without
// waiting; stage B: look up; fused: insert and obtain the index). Every lane
// of every warp calls it.
template <int Op, int P, int M>
__device__ __forceinline__ void tile_collect(TileShared& T, const FrameArgs& f,
                                             const VolumeArgs& vol, const Ray& r, bool valid,
                                             Walk<M>& w, unsigned& acc, PointKeys& pk) {
  acc = 0;
  if (valid) {
    if constexpr (M > 0) {
      acc = walk_point<M>(f, r, w);
#pragma unroll
      for (int k = 0; k < 2 * M + 1; ++k)
        if ((acc >> k) & 1u) point_key<Op, P>(pk, block_key_of(w.gx[k], w.gy[k], w.gz[k]), T, vol);
    } else {
      // Generic half band. For allocation alone, a sample whose block already
      // holds an accepted voxel of this point cannot add a block, so its test
      // is skipped; duplicates of a voxel cannot add one either.
      WalkDedupe walk;
      for (int k = 0; k <= 2 * f.M; ++k) {
        int gx, gy, gz;
        float zc;
        if (!sample_voxel(f, r, k, gx, gy, gz)) continue;
        const unsigned long long key = block_key_of(gx, gy, gz);
        if (Op == kOpAllocate) {
          if (key == pk.last) continue;
        } else if (walk.seen_then_push(gx, gy, gz)) {
          continue;
        }
        if (voxel_test(f, gx, gy, gz, zc)) point_key<Op, P>(pk, key, T, vol);
      }
    }
  }
  tile_list_point_keys<Op, P>(T, vol, pk);
}

// Five sums of one accepted voxel, added straight to the pool.
__device__ __forceinline__ void add_voxel_direct(const VolumeArgs& vol, int idx, int l, float t,
                                                 bool colour, float cr, float cg, float cb) {
  if (idx < 0) return;
  add_contribution(vol, static_cast<size_t>(idx) * kBlockVoxels + l, t, colour,
                   cr, cg, cb);
}

// Stage A, tile strategy, for one 16x16 pixel tile: the tile's distinct keys
// are collected in the shared-memory set, then, after one barrier, the list is
// inserted by consecutive lanes, warp-cooperatively, without waiting. Every
// thread of the CTA calls it; it ends with a barrier, so T can be reused.
template <int P, int M>
__device__ __forceinline__ void tile_allocate_body(TileShared& T, const FrameArgs& f,
                                                   const VolumeArgs& vol, int tile, int tiles_x) {
  tile_init(T, vol);
  __syncthreads();
  if (T.err) {  // poisoned volume: do nothing (uniform across the CTA)
    __syncthreads();
    return;
  }
  Ray r;
  int u, v;
  const bool valid = tile_ray(f, tile, tiles_x, r, u, v);
  Walk<M> w;
  unsigned acc;
  PointKeys pk;
  tile_collect<kOpAllocate, P, M>(T, f, vol, r, valid, w, acc, pk);
  __syncthreads();
  const int n = T.n < kTileList ? T.n : kTileList;
  const unsigned lane = threadIdx.x & 31u;
  for (int base = (threadIdx.x & ~31); base < n; base += kThreads) {
    const int i = base + static_cast<int>(lane);
    const bool has = i < n;
    warp_insert_nowait<P>(vol, has ? T.list[i] : kEmptyKey, has);
  }
  __syncthreads();
}

template <int P, int M>
__global__ void __launch_bounds__(kThreads, 4)
    tile_allocate_kernel(const __grid_constant__ FrameArgs f,
                         const __grid_constant__ VolumeArgs vol, int tiles_x) {
  __shared__ TileShared T;
  tile_allocate_body<P, M>(T, f, vol, blockIdx.x, tiles_x);
}

// ----------------------------------------------------------------------------
// fused, tile strategy: one walk per point, both stages in one kernel
// ----------------------------------------------------------------------------
// Phase 1 is stage A's tile collection (walk, distinct keys, shared set and
// list). Phase 2 inserts the list warp-cooperatively and OBTAINS each key's
// pool index (a key won by another CTA may still be unpublished: that wait
// is bounded, and a winner never waits before publishing, so it cannot
// deadlock). Phase 3 adds every accepted voxel's sums, taking its block's
// index from the tile list in shared memory: no table probe at all, and the
// walk is not repeated. Safe without a grid barrier because a point only
// touches blocks whose indices it has resolved.
struct FusedTileShared {
  TileShared T;
  int idx[kTileList];
};

// Op: kOpFused (the fused path: phase 2 inserts and obtains the indices) or
// kOpIntegrate (stage B of the two-stage path, after stage A's kernel: phase
// 2 only looks the keys up, warp-cooperatively; the tile strategy of stage B).
// TPP > 1 (threads per point, with the half band compiled): the TPP
// consecutive threads of a point each walk a contiguous span of its 2M+1
// samples, so a tile holds 256 / TPP points and a frame launches TPP times as
// many CTAs -- more parallelism for small frames, at the price of one ray and
// a two-sample lead-in per thread. Per voxel the arithmetic is unchanged.
template <int P, int M, int TPP = 1, int Op = kOpFused>
__device__ __forceinline__ void tile_fused_body(FusedTileShared& S, const FrameArgs& f,
                                                const VolumeArgs& vol, int tile, int tiles_x) {
  static_assert(TPP == 1 || (M > 0 && (TPP & (TPP - 1)) == 0 && TPP <= 8),
                "threads per point: 1, or 2, 4, 8 with the half band compiled");
  static_assert(Op == kOpFused || Op == kOpIntegrate, "fused path or stage B");
  TileShared& T = S.T;
  tile_init(T, vol);
  __syncthreads();
  if (T.err) {  // poisoned volume: do nothing (uniform across the CTA)
    __syncthreads();
    return;
  }
  Ray r;
  int u, v;
  const bool valid = tile_ray<TPP>(f, tile, tiles_x, r, u, v);
  PointKeys pk;
  // phase 1: the walk and the tile's key list. With the half band compiled,
  // each accepted sample is reduced to one packed word and its tsdf value,
  // so little state is held across the barriers.
  constexpr int K = M > 0 ? (2 * M + 1 + TPP - 1) / TPP : 1;  // samples a thread
  unsigned smp[K];
  float tv[K];
  int bx0 = 0, by0 = 0, bz0 = 0;
  if constexpr (M > 0) {
    unsigned acc = 0;
    if (valid) {
      if constexpr (TPP == 1) {
        acc = walk_point_packed<M>(f, r, smp, tv, bx0, by0, bz0);
      } else {
        // thread j of the point: samples [j (2M+1) / TPP, (j+1) (2M+1) / TPP)
        const int j = static_cast<int>(threadIdx.x) % TPP;
        const int lo = j * (2 * M + 1) / TPP;
        const int hi = (j + 1) * (2 * M + 1) / TPP;
        acc = walk_point_span<M, K>(f, r, lo, hi - lo, smp, tv, bx0, by0, bz0);
      }
    } else {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        smp[k] = 0u;
        tv[k] = 0.0f;
      }
    }
    // a sample's block offset is bits 9..20 of its packed word: the 64-bit
    // key is built only where it changes
    unsigned last = 0u;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const unsigned q = smp[k];
      const unsigned blk = q & kSampleBlockBits;
      if ((q & kSampleValid) && blk != last) {
        last = blk;
        point_key<Op, P>(pk, sample_key(q, bx0, by0, bz0), T, vol);
      }
    }
    tile_list_point_keys<Op, P>(T, vol, pk);
  } else {
    Walk<M> w;
    unsigned acc;
    tile_collect<Op, P, M>(T, f, vol, r, valid, w, acc, pk);
  }
  __syncthreads();
  // phase 2: insert the list and obtain the indices (stage B: look them up)
  const int n = T.n < kTileList ? T.n : kTileList;
  const unsigned lane = threadIdx.x & 31u;
  for (int base = (threadIdx.x & ~31); base < n; base += blockDim.x) {
    const int i = base + static_cast<int>(lane);
    const bool has = i < n;
    const unsigned long long key = has ? T.list[i] : kEmptyKey;
    const int res = Op == kOpFused ? warp_insert_get<P>(vol, key, has)
                                   : warp_lookup_get<P>(vol, key, has);
    if (has) S.idx[i] = res;
  }
  __syncthreads();
  if (!valid) return;  // no barrier follows

  // phase 3: the sums, each block's index from the tile list
  float cr = 0.0f, cg = 0.0f, cb = 0.0f;
  const bool colour = f.rgb != nullptr;
  if (colour) {
    load_colour(f, u, v, cr, cg, cb);
  }
  // a key missing from the list (set or list full) is resolved on its own
  auto index_of = [&](unsigned long long key) -> int {
    const int p = tile_find(T, key);
    return p >= 0 ? S.idx[p] : resolve_single<Op, P>(vol, key);
  };
  if constexpr (M > 0) {
    unsigned last = 0u;  // block offset bits of the resolved block (0: none yet)
    int idx = -1;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const unsigned q = smp[k];
      if (!(q & kSampleValid)) continue;
      const unsigned blk = q & kSampleBlockBits;
      if (blk != last) {
        last = blk;
        idx = index_of(sample_key(q, bx0, by0, bz0));
      }
      if (idx >= 0)
        add_contribution(vol, static_cast<size_t>(idx) * kBlockVoxels + (q & 511u), tv[k], colour,
                         cr, cg, cb);
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
      const unsigned long long key = block_key_of(gx, gy, gz);
      if (key != bc.key) {
        bc.key = key;
        bc.idx = index_of(key);
      }
      if (bc.idx >= 0)
        add_contribution(vol, static_cast<size_t>(bc.idx) * kBlockVoxels + local_index(gx, gy, gz),
                         tsdf_value(f, r.d, zc), colour, cr, cg, cb);
    }
  }
}

// At most 64 registers a thread (four 256-thread CTAs per SM). The default
// instantiation (half band 4, one thread per point) fits without spilling;
// the cap measured faster than three CTAs per SM with more registers.
template <int P, int M, int TPP = 1, int Op = kOpFused>
__global__ void __launch_bounds__(kThreads, 4)
    tile_fused_kernel(const __grid_constant__ FrameArgs f, const __grid_constant__ VolumeArgs vol,
                      int tiles_x) {
  __shared__ FusedTileShared S;
  tile_fused_body<P, M, TPP, Op>(S, f, vol, blockIdx.x, tiles_x);
}

inline int tiles_of(int n) { return (n + kTile - 1) / kTile; }

}  // namespace tsdf
