// Kernels of hash-blocked TSDF fusion (paper Section 2.2, "Two passes"):
//   allocate_kernel   stage A: band walk -> block keys -> per-warp
//                     __match_any_sync dedupe -> per-CTA shared-memory key set
//                     -> one insert (Listing 1) per distinct key per CTA;
//   integrate_*       stage B: band walk -> lookup -> weighted sums into the
//                     five pool arrays (scatter variant = the paper's update
//                     stage; aggregated variant = per-CTA shared-memory
//                     pre-aggregation per voxel, then vector reductions);
//   export_kernel     read-out: per-voxel means (Section 2.2, sums -> means);
//   clear_used_kernel reset of the used prefix of the pool.
// A CTA covers a 16x16 pixel tile; each warp an 8x4 sub-tile, so the lanes of a
// warp see neighbouring rays and mostly the same blocks.
#include <climits>
#include <cstdint>

#include "tsdf_device.cuh"
#include "tsdf_launch.h"

namespace tsdf {

constexpr int kThreads = 256;
constexpr int kTile = 16;
constexpr int kSetSlots = 2048;  // per-CTA block-key set (16 KB)

__device__ __forceinline__ void tile_pixel(int tile, int tiles_x, int& u, int& v) {
  const int tx = tile % tiles_x;
  const int ty = tile / tiles_x;
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  u = tx * kTile + (w & 1) * 8 + (lane & 7);
  v = ty * kTile + (w >> 1) * 4 + (lane >> 3);
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

// Walk state of one point: the last two in-range voxels (two band samples are
// v apart on a unit ray, a voxel's diagonal is v*sqrt(3) < 2v, so only the
// previous two samples can repeat a voxel).
struct WalkDedupe {
  int ax = INT_MIN, ay = 0, az = 0, bx = INT_MIN, by = 0, bz = 0;
  __device__ __forceinline__ bool seen_then_push(int x, int y, int z) {
    if ((x == ax && y == ay && z == az) || (x == bx && y == by && z == bz)) return true;
    bx = ax; by = ay; bz = az;
    ax = x; ay = y; az = z;
    return false;
  }
};

// ----------------------------------------------------------------------------
// stage A
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
  if (u < f.W && v < f.H) valid = make_ray(f, u, v, __ldg(f.depth + v * f.W + u), r);
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
  // one global insert per distinct block of the tile
  for (int i = threadIdx.x; i < kSetSlots; i += kThreads) {
    const unsigned long long key = s_set[i];
    if (key != kEmptyKey) {
      int bx, by, bz;
      unpack_key(key, bx, by, bz);
      insert_block<P>(vol, key, bx, by, bz);
    }
  }
}

// ----------------------------------------------------------------------------
// stage B, scatter: five atomic additions per accepted voxel (Section 2.2)
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
    integrate_scatter_kernel(const __grid_constant__ FrameArgs f,
                             const __grid_constant__ VolumeArgs vol, int tiles_x) {
  __shared__ unsigned int s_err;
  if (threadIdx.x == 0) s_err = load_err_volatile(vol.hdr);
  __syncthreads();
  if (s_err) return;

  int u, v;
  tile_pixel(blockIdx.x, tiles_x, u, v);
  if (u >= f.W || v >= f.H) return;
  Ray r;
  if (!make_ray(f, u, v, __ldg(f.depth + v * f.W + u), r)) return;
  float cr = 0.0f, cg = 0.0f, cb = 0.0f;
  const bool colour = f.rgb != nullptr;
  if (colour) {
    const uint8_t* c = f.rgb + 3 * (static_cast<size_t>(v) * f.W + u);
    cr = static_cast<float>(c[0]);
    cg = static_cast<float>(c[1]);
    cb = static_cast<float>(c[2]);
  }
  unsigned long long ckey = kEmptyKey;
  int cidx = -1;
  WalkDedupe walk;
  for (int k = 0; k <= 2 * f.M; ++k) {
    int gx, gy, gz;
    float zc;
    if (!sample_voxel(f, r, k, gx, gy, gz) || walk.seen_then_push(gx, gy, gz) ||
        !voxel_test(f, gx, gy, gz, zc))
      continue;
    const int bx = gx >> 3, by = gy >> 3, bz = gz >> 3;
    const unsigned long long key = pack_key(bx, by, bz);
    if (key != ckey) {
      ckey = key;
      cidx = lookup_block(vol, key, bx, by, bz);
    }
    if (cidx < 0) continue;
    const size_t o = static_cast<size_t>(cidx) * kBlockVoxels + local_index(gx, gy, gz);
    atomicAdd(vol.ch[0] + o, tsdf_value(f, r.d, zc));
    atomicAdd(vol.ch[1] + o, 1.0f);
    if (colour) {
      atomicAdd(vol.ch[2] + o, cr);
      atomicAdd(vol.ch[3] + o, cg);
      atomicAdd(vol.ch[4] + o, cb);
    }
  }
}

// ----------------------------------------------------------------------------
// read-out and reset
// ----------------------------------------------------------------------------
__global__ void export_kernel(const __grid_constant__ VolumeArgs vol, float* __restrict__ out,
                              unsigned int n) {
  const size_t total = static_cast<size_t>(n) * kBlockVoxels;
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const size_t blk = i / kBlockVoxels;
    const size_t l = i % kBlockVoxels;
    const float w = vol.ch[1][i];
    float* o = out + blk * 5 * kBlockVoxels + l;
    const bool any = w > 0.0f;
    const float w255 = w * 255.0f;  // exact while w < 65793
    o[0] = any ? __fdiv_rn(vol.ch[0][i], w) : 0.0f;
    o[kBlockVoxels] = w;
    o[2 * kBlockVoxels] = any ? __fdiv_rn(vol.ch[2][i], w255) : 0.0f;
    o[3 * kBlockVoxels] = any ? __fdiv_rn(vol.ch[3][i], w255) : 0.0f;
    o[4 * kBlockVoxels] = any ? __fdiv_rn(vol.ch[4][i], w255) : 0.0f;
  }
}

// Zero the used prefix [0, min(count, pool)) of every channel; reads the count
// on the device so the host needs no round trip.
__global__ void clear_used_kernel(const __grid_constant__ VolumeArgs vol) {
  const unsigned int c = *reinterpret_cast<volatile unsigned int*>(&vol.hdr->count);
  const unsigned int n = c < vol.pool ? c : vol.pool;
  const size_t quads = static_cast<size_t>(n) * (kBlockVoxels / 4);
  const float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < quads;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
#pragma unroll
    for (int c5 = 0; c5 < 5; ++c5) reinterpret_cast<float4*>(vol.ch[c5])[i] = z;
  }
}

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
static inline int tiles_of(int n) { return (n + kTile - 1) / kTile; }

cudaError_t launch_allocate(const FrameArgs& f, const VolumeArgs& vol, int probe_load,
                            cudaStream_t s) {
  const int tx = tiles_of(f.W);
  const int tiles = tx * tiles_of(f.H);
  switch (probe_load) {
    case kLoadL2:
      allocate_kernel<kLoadL2><<<tiles, kThreads, 0, s>>>(f, vol, tx);
      break;
    case kLoadRelaxed:
      allocate_kernel<kLoadRelaxed><<<tiles, kThreads, 0, s>>>(f, vol, tx);
      break;
    default:
      allocate_kernel<kLoadCached><<<tiles, kThreads, 0, s>>>(f, vol, tx);
      break;
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_integrate(const FrameArgs& f, const VolumeArgs& vol, int mode,
                             cudaStream_t s) {
  const int tx = tiles_of(f.W);
  const int tiles = tx * tiles_of(f.H);
  (void)mode;
  integrate_scatter_kernel<<<tiles, kThreads, 0, s>>>(f, vol, tx);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_export(const VolumeArgs& vol, float* out, unsigned int n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t total = static_cast<size_t>(n) * kBlockVoxels;
  const unsigned int grid = static_cast<unsigned int>((total + 255) / 256 < 65535 * 4
                                                          ? (total + 255) / 256
                                                          : 65535 * 4);
  export_kernel<<<grid, 256, 0, s>>>(vol, out, n);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_clear_used(const VolumeArgs& vol, int sm_count, cudaStream_t s) {
  clear_used_kernel<<<sm_count * 8, 256, 0, s>>>(vol);
  note_launch();
  return cudaGetLastError();
}

}  // namespace tsdf
