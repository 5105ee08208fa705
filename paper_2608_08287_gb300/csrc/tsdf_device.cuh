// Device-side data structures and per-point geometry of hash-blocked TSDF
// fusion (paper Section 2). Shared by the stage A / stage B / fused kernels.
//
// Every floating-point step that decides an integer (voxel index, pixel index,
// accept/reject) is written with explicit round-to-nearest intrinsics
// (__fadd_rn, __fmul_rn, __fmaf_rn, __fdiv_rn, __frcp_rn, __fsqrt_rn) in one
// fixed order, so the compiler can neither contract nor reorder it and the
// decisions are reproducible by any IEEE-754 single-precision implementation
// of the same steps.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tsdf.h"
#include "tsdf_check.h"

namespace tsdf {

constexpr int kBlockEdge = 8;                 // Section 2.1: 8^3 voxels per block
constexpr int kBlockVoxels = 512;
constexpr int kKeyBias = 1 << 20;             // Section 2.1: 21-bit biased axes
constexpr int kMaxHalfBand = 16;              // M = lrintf(tau / v) <= 16
constexpr unsigned long long kEmptyKey = TSDF_EMPTY_KEY;
constexpr int kUnpublished = TSDF_UNPUBLISHED;   // index not yet published
constexpr int kFailedIdx = -2;                // slot won but pool exhausted
constexpr float kVoxelLimit = 8388608.0f;     // 2^23 voxels = 2^20 blocks

// 16-byte table entry (Section 2.1): 64-bit key, 32-bit block index, padding.
struct __align__(16) Entry {
  unsigned long long key;
  int idx;
  int pad;
};
static_assert(sizeof(Entry) == 16, "table entry must be 16 bytes");

// Volume header at offset 0 of the allocation.
struct __align__(256) Header {
  unsigned int count;  // blocks claimed (atomicAdd after winning a slot)
  unsigned int err;    // sticky TSDF_ERRBIT_* flags
  unsigned int pad[62];
};

// Packed key (Section 2.1): each axis biased by 2^20 into 21 bits.
__host__ __device__ __forceinline__ unsigned long long pack_key(int bx, int by, int bz) {
  return (static_cast<unsigned long long>(static_cast<unsigned int>(bx + kKeyBias)) << 42) |
         (static_cast<unsigned long long>(static_cast<unsigned int>(by + kKeyBias)) << 21) |
         static_cast<unsigned long long>(static_cast<unsigned int>(bz + kKeyBias));
}

__host__ __device__ __forceinline__ void unpack_key(unsigned long long key, int& bx, int& by,
                                                    int& bz) {
  const unsigned long long m = (1ull << 21) - 1;
  bx = static_cast<int>((key >> 42) & m) - kKeyBias;
  by = static_cast<int>((key >> 21) & m) - kKeyBias;
  bz = static_cast<int>(key & m) - kKeyBias;
}

// Multiply-xor hash (Section 3.1) with the primes of Teschner et al. (2003),
// products and xor taken mod 2^32.
__host__ __device__ __forceinline__ unsigned int hash_block(int bx, int by, int bz) {
  return (static_cast<unsigned int>(bx) * 73856093u) ^
         (static_cast<unsigned int>(by) * 19349669u) ^
         (static_cast<unsigned int>(bz) * 83492791u);
}

// Per-frame constants, passed by value (__grid_constant__) to every kernel.
struct FrameArgs {
  const float* depth;      // H x W, row-major
  const uint8_t* rgb;      // H x W x 3 or nullptr
  int W, H;
  float fx, fy, cx, cy;
  float R[9];              // camera-to-world rotation, row-major
  float t[3];              // camera-to-world translation
  // Voxel centre to camera frame as one affine map of the integer voxel g:
  // c = A g + b with A = v R^T (row j: v * column j of R) and
  // b = R^T (v/2 - t), so that c = R^T ((g + 1/2) v - t).
  float A[9];
  float b[3];
  float v, inv_v;          // voxel size and its IEEE reciprocal
  float tau, neg_tau, inv_tau;
  int M;                   // half band, samples k = 0..2M
  unsigned int* err;       // the volume's error word (range checks of image reads)
};

// Device view of one volume.
struct VolumeArgs {
  Entry* table;
  unsigned int mask;       // table_slots - 1
  unsigned int slots;
  int32_t* coords;         // pool x 3
  unsigned int pool;
  // The five sums of a voxel (Section 2.1), split 4 + 1 so that one vector
  // reduction carries four of them: pool x 512 records {tsdf sum, weight,
  // red sum, green sum} and pool x 512 blue sums.
  float4* twrg;
  float* blue;
  Header* hdr;
  unsigned long long timeout_ns;
  // Probes before a scan gives up: table_slots (unbounded in the paper's
  // sense: a full scan reports TABLE_FULL), or a smaller bound that gives up
  // SILENTLY -- the negative control of a bounded probe (Section 7), never a
  // default.
  unsigned int probe_limit;
  // Nonzero: a block's pool index is its table slot (Section 6, "Deriving the
  // location from the slot"); pool == table_slots, no index is published and
  // no thread waits.
  unsigned int slot_index;
};

// Diagnostic read-out of a volume (tsdf_volume_table_stats).
struct TableStatsDev {
  unsigned long long occupied;    // table entries holding a key
  unsigned long long probe_sum;   // sum over keys of (distance from home slot + 1)
  unsigned long long weight_sum;  // sum of voxel weights over the used blocks
  unsigned int probe_max;
  unsigned int pad;
};

// One frame of a batch: its frame and volume arguments and where its tiles
// start in the batch's global tile numbering.
struct SessionArgs {
  FrameArgs f;
  VolumeArgs vol;
  int tiles_x;
  int tile_begin;
};
static_assert(sizeof(SessionArgs) % 4 == 0, "session args are copied as words");

// Header of a batch's session table in device memory; SessionArgs[n] follow.
struct __align__(16) BatchHeader {
  int n;
  int total_tiles;
  int pad[2];
};

// ----------------------------------------------------------------------------
// geometry
// ----------------------------------------------------------------------------
struct Ray {
  float d;                 // the point's depth
  float px, py, pz;        // back-projected point, world frame
  float dx, dy, dz;        // unit view ray, world frame
};

// Back-project pixel (u, v) and build its unit view ray. False if the depth
// is invalid (not finite or not > 0).
__device__ __forceinline__ bool make_ray(const FrameArgs& f, int u, int v, float d, Ray& r) {
  if (!(isfinite(d) && d > 0.0f)) return false;
  const float rx = __fdiv_rn(__fsub_rn(static_cast<float>(u), f.cx), f.fx);
  const float ry = __fdiv_rn(__fsub_rn(static_cast<float>(v), f.cy), f.fy);
  r.d = d;
  // camera frame: the point and the unit ray
  const float cpx = __fmul_rn(rx, d), cpy = __fmul_rn(ry, d), cpz = d;
  const float n = __fsqrt_rn(__fmaf_rn(rx, rx, __fmaf_rn(ry, ry, 1.0f)));
  const float cdx = __fdiv_rn(rx, n), cdy = __fdiv_rn(ry, n), cdz = __fdiv_rn(1.0f, n);
  // world frame, once per point: P = R p + t, D = R d
  r.px = __fmaf_rn(f.R[2], cpz, __fmaf_rn(f.R[1], cpy, __fmaf_rn(f.R[0], cpx, f.t[0])));
  r.py = __fmaf_rn(f.R[5], cpz, __fmaf_rn(f.R[4], cpy, __fmaf_rn(f.R[3], cpx, f.t[1])));
  r.pz = __fmaf_rn(f.R[8], cpz, __fmaf_rn(f.R[7], cpy, __fmaf_rn(f.R[6], cpx, f.t[2])));
  r.dx = __fmaf_rn(f.R[2], cdz, __fmaf_rn(f.R[1], cdy, __fmul_rn(f.R[0], cdx)));
  r.dy = __fmaf_rn(f.R[5], cdz, __fmaf_rn(f.R[4], cdy, __fmul_rn(f.R[3], cdx)));
  r.dz = __fmaf_rn(f.R[8], cdz, __fmaf_rn(f.R[7], cdy, __fmul_rn(f.R[6], cdx)));
  return true;
}

// Voxel selected by band sample k (offset (k-M) v along the ray). False if the
// voxel's block coordinate does not fit the 21-bit key.
__device__ __forceinline__ bool sample_voxel(const FrameArgs& f, const Ray& r, int k, int& gx,
                                             int& gy, int& gz) {
  const float tk = __fmul_rn(static_cast<float>(k - f.M), f.v);
  const float wx = __fmaf_rn(tk, r.dx, r.px);
  const float wy = __fmaf_rn(tk, r.dy, r.py);
  const float wz = __fmaf_rn(tk, r.dz, r.pz);
  const float qx = floorf(__fmul_rn(wx, f.inv_v));
  const float qy = floorf(__fmul_rn(wy, f.inv_v));
  const float qz = floorf(__fmul_rn(wz, f.inv_v));
  const bool ok = (qx >= -kVoxelLimit) && (qx < kVoxelLimit) && (qy >= -kVoxelLimit) &&
                  (qy < kVoxelLimit) && (qz >= -kVoxelLimit) && (qz < kVoxelLimit);
  gx = ok ? static_cast<int>(qx) : 0;
  gy = ok ? static_cast<int>(qy) : 0;
  gz = ok ? static_cast<int>(qz) : 0;
  return ok;
}

// Occlusion test at the voxel centre, shared by both stages (Section 2.2):
// centre in front of the camera, nearest pixel inside the image with a valid
// depth d', centre no more than tau behind d'. Split in two so that a caller
// can issue the depth gathers of several samples before testing any of them:
// voxel_project computes the centre's camera depth zc and the row-major index
// of its nearest pixel (-1 when behind the camera or outside the image);
// voxel_accept takes the gathered d'.
__device__ __forceinline__ int voxel_project(const FrameArgs& f, int gx, int gy, int gz,
                                             float& zc) {
  // c = A g + b (the per-frame affine map of the voxel centre), g exact in float
  const float fgx = static_cast<float>(gx), fgy = static_cast<float>(gy),
              fgz = static_cast<float>(gz);
  const float ccz = __fmaf_rn(f.A[8], fgz, __fmaf_rn(f.A[7], fgy, __fmaf_rn(f.A[6], fgx, f.b[2])));
  zc = ccz;
  if (!(ccz > 0.0f)) return -1;
  const float ccx = __fmaf_rn(f.A[2], fgz, __fmaf_rn(f.A[1], fgy, __fmaf_rn(f.A[0], fgx, f.b[0])));
  const float ccy = __fmaf_rn(f.A[5], fgz, __fmaf_rn(f.A[4], fgy, __fmaf_rn(f.A[3], fgx, f.b[1])));
  const float iz = __frcp_rn(ccz);
  const float qu = floorf(__fadd_rn(__fmaf_rn(f.fx, __fmul_rn(ccx, iz), f.cx), 0.5f));
  const float qv = floorf(__fadd_rn(__fmaf_rn(f.fy, __fmul_rn(ccy, iz), f.cy), 0.5f));
  if (!(qu >= 0.0f && qu < static_cast<float>(f.W) && qv >= 0.0f &&
        qv < static_cast<float>(f.H)))
    return -1;
  return static_cast<int>(qv) * f.W + static_cast<int>(qu);
}

// Depth at row-major pixel index q (checked builds: q inside the image, else
// the BOUNDS bit and NaN, which no test accepts).
__device__ __forceinline__ float load_depth(const FrameArgs& f, long long q) {
  if (!index_ok_signed(q, static_cast<unsigned long long>(f.W) * static_cast<unsigned>(f.H),
                       f.err))
    return __int_as_float(0x7fc00000);
  return __ldg(f.depth + q);
}

// Colour codes of pixel (u, v) (checked builds: inside the image, else the
// BOUNDS bit and zeros).
__device__ __forceinline__ void load_colour(const FrameArgs& f, int u, int v, float& cr, float& cg,
                                            float& cb) {
  const long long q = static_cast<long long>(v) * f.W + u;
  if (!index_ok_signed(q, static_cast<unsigned long long>(f.W) * static_cast<unsigned>(f.H),
                       f.err)) {
    cr = cg = cb = 0.0f;
    return;
  }
  const uint8_t* c = f.rgb + 3 * static_cast<size_t>(q);
  cr = static_cast<float>(c[0]);
  cg = static_cast<float>(c[1]);
  cb = static_cast<float>(c[2]);
}

__device__ __forceinline__ bool voxel_accept(const FrameArgs& f, float d2, float zc) {
  return isfinite(d2) && d2 > 0.0f && __fsub_rn(d2, zc) >= f.neg_tau;
}

__device__ __forceinline__ bool voxel_test(const FrameArgs& f, int gx, int gy, int gz,
                                           float& zc) {
  const int q = voxel_project(f, gx, gy, gz, zc);
  if (q < 0) return false;
  return voxel_accept(f, load_depth(f, q), zc);
}

// The band walk of one point with the half band M known at compile time: all
// 2M+1 samples are unrolled, their depth gathers are issued together, and the
// result is a mask of accepted samples (after the once-per-point dedupe of
// voxels) with each sample's voxel and centre depth.
//
// The dedupe compares each sample with the previous one only. Every voxel
// coordinate is a monotone function of k -- t_k = (k - M) v, the rounded
// fused multiply-add t_k d + p, the product by 1/v and floor are each
// monotone -- and so is the range test, so the in-range samples are
// consecutive and a voxel equal to an earlier one is equal to all samples
// between them, the previous sample included. "Not an earlier voxel of this
// point" (Section 2.2) and "not the previous sample's voxel" are the same
// test.
template <int M>
struct Walk {
  static constexpr int K = 2 * M + 1;
  int gx[K], gy[K], gz[K];
  float zc[K];
};

template <int M>
__device__ __forceinline__ unsigned walk_point(const FrameArgs& f, const Ray& r, Walk<M>& w) {
  constexpr int K = 2 * M + 1;
  int q[K];
  unsigned in_range = 0;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const float tk = __fmul_rn(static_cast<float>(k - M), f.v);
    const float wx = __fmaf_rn(tk, r.dx, r.px);
    const float wy = __fmaf_rn(tk, r.dy, r.py);
    const float wz = __fmaf_rn(tk, r.dz, r.pz);
    const float qx = floorf(__fmul_rn(wx, f.inv_v));
    const float qy = floorf(__fmul_rn(wy, f.inv_v));
    const float qz = floorf(__fmul_rn(wz, f.inv_v));
    const bool ok = (qx >= -kVoxelLimit) && (qx < kVoxelLimit) && (qy >= -kVoxelLimit) &&
                    (qy < kVoxelLimit) && (qz >= -kVoxelLimit) && (qz < kVoxelLimit);
    w.gx[k] = ok ? static_cast<int>(qx) : 0;
    w.gy[k] = ok ? static_cast<int>(qy) : 0;
    w.gz[k] = ok ? static_cast<int>(qz) : 0;
    bool fresh = ok;
    if (k >= 1)
      fresh = fresh && !(((in_range >> (k - 1)) & 1u) && w.gx[k] == w.gx[k - 1] &&
                         w.gy[k] == w.gy[k - 1] && w.gz[k] == w.gz[k - 1]);
    in_range |= ok ? (1u << k) : 0u;
    q[k] = fresh ? voxel_project(f, w.gx[k], w.gy[k], w.gz[k], w.zc[k]) : -1;
  }
  float d2[K];
#pragma unroll
  for (int k = 0; k < K; ++k) d2[k] = q[k] >= 0 ? load_depth(f, q[k]) : 0.0f;
  unsigned acc = 0;
#pragma unroll
  for (int k = 0; k < K; ++k)
    acc |= (q[k] >= 0 && voxel_accept(f, d2[k], w.zc[k])) ? (1u << k) : 0u;
  return acc;
}

// Fire-and-forget float addition into the pool (PTX `red`): the thread never
// waits for a returned value. Written explicitly because a plain atomicAdd
// whose result is unused may still be issued as a returning atomic when the
// kernel holds other atomics.
__device__ __forceinline__ void red_add(float* p, float v) {
  asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ void red_add_v4(float4* p, float a, float b, float c, float d) {
  asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a),
               "f"(b), "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ void red_add_v2(float4* p, float a, float b) {
  asm volatile("red.relaxed.gpu.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b)
               : "memory");
}

// One contribution to voxel o of the pool (Section 2.2, "Update"): tsdf and a
// weight of 1, and the point's colour when the frame has one -- five sums in
// two fire-and-forget reductions (one 16-byte vector, one scalar). Checked
// builds: o inside the pool.
__device__ __forceinline__ void add_contribution(const VolumeArgs& vol, size_t o, float t,
                                                 bool colour, float cr, float cg, float cb) {
  if (!index_ok(o, static_cast<unsigned long long>(vol.pool) * kBlockVoxels, &vol.hdr->err))
    return;
  if (colour) {
    red_add_v4(vol.twrg + o, t, 1.0f, cr, cg);
    red_add(vol.blue + o, cb);
  } else {
    red_add_v2(vol.twrg + o, t, 1.0f);
  }
}

// Stored value: truncated, normalised signed distance at the voxel centre.
__device__ __forceinline__ float tsdf_value(const FrameArgs& f, float d, float zc) {
  return fminf(1.0f, fmaxf(-1.0f, __fsub_rn(d, zc) * f.inv_tau));
}

__device__ __forceinline__ int local_index(int gx, int gy, int gz) {
  return (gx & 7) | ((gy & 7) << 3) | ((gz & 7) << 6);
}

// A band sample packed in one word: accepted flag, the block's offset from
// the block of the point's first in-range sample (4 bits per axis,
// biased by 8: a band of at most 2*16+1 samples, one voxel apart, crosses at
// most four block boundaries per axis) and the voxel's local index.
constexpr unsigned kSampleValid = 1u << 31;

__device__ __forceinline__ unsigned pack_sample(int dbx, int dby, int dbz, int l) {
  return kSampleValid | (static_cast<unsigned>(dbx + 8) << 9) |
         (static_cast<unsigned>(dby + 8) << 13) | (static_cast<unsigned>(dbz + 8) << 17) |
         static_cast<unsigned>(l);
}

// The block offset fields of a packed sample (never all zero in a valid one:
// each biased offset is at least 4).
constexpr unsigned kSampleBlockBits = 0xFFFu << 9;

// The key of a packed sample's block, given the block its offsets are from.
__device__ __forceinline__ unsigned long long sample_key(unsigned q, int bx0, int by0, int bz0) {
  return pack_key(bx0 + static_cast<int>((q >> 9) & 15u) - 8,
                  by0 + static_cast<int>((q >> 13) & 15u) - 8,
                  bz0 + static_cast<int>((q >> 17) & 15u) - 8);
}

// The band walk over samples lo .. lo+n-1 of one point (n <= C): the same
// samples, dedupe and test as walk_point, each sample produced directly in
// packed form. A rolling window of the two previous voxels replaces the
// per-sample voxel arrays, so few registers are live at once. (Comparing
// with the previous voxel alone is the same test, see walk_point; with the
// two-voxel window the fused tile kernel's registers are allocated without
// spills, and it measured faster.) The window starts two samples before lo,
// so a walk split into spans over several threads dedupes exactly as the
// whole walk does. Packing is relative to the block of the
// span's first in-range sample. Returns the mask of accepted samples (bit i
// for sample lo+i); smp[i] and (with TSDF) tv[i] hold the packed voxel and the
// tsdf value of each accepted one.
template <int M, int C, bool TSDF = true>
__device__ __forceinline__ unsigned walk_point_span(const FrameArgs& f, const Ray& r, int lo,
                                                    int n, unsigned* smp, float* tv, int& bx0,
                                                    int& by0, int& bz0) {
  int q[C];
  float zc[C];
  int ax = 0, ay = 0, az = 0, cx = 0, cy = 0, cz = 0;  // previous two voxels
  bool a_ok = false, c_ok = false;                     // ... and whether in range
  bool have_base = false;
#pragma unroll
  for (int i = -2; i < C; ++i) {
    const int k = lo + i;
    const float tk = __fmul_rn(static_cast<float>(k - M), f.v);
    const float qx = floorf(__fmul_rn(__fmaf_rn(tk, r.dx, r.px), f.inv_v));
    const float qy = floorf(__fmul_rn(__fmaf_rn(tk, r.dy, r.py), f.inv_v));
    const float qz = floorf(__fmul_rn(__fmaf_rn(tk, r.dz, r.pz), f.inv_v));
    // samples before the band or past the span are never in range
    const bool ok = k >= 0 && i < n && (qx >= -kVoxelLimit) && (qx < kVoxelLimit) &&
                    (qy >= -kVoxelLimit) && (qy < kVoxelLimit) && (qz >= -kVoxelLimit) &&
                    (qz < kVoxelLimit);
    const int gx = ok ? static_cast<int>(qx) : 0;
    const int gy = ok ? static_cast<int>(qy) : 0;
    const int gz = ok ? static_cast<int>(qz) : 0;
    const bool fresh = ok && !(a_ok && gx == ax && gy == ay && gz == az) &&
                       !(c_ok && gx == cx && gy == cy && gz == cz);
    cx = ax; cy = ay; cz = az; c_ok = a_ok;
    ax = gx; ay = gy; az = gz; a_ok = ok;
    if (i < 0) continue;  // the sample before the span: voxel only
    if (ok && !have_base) {
      bx0 = gx >> 3;
      by0 = gy >> 3;
      bz0 = gz >> 3;
      have_base = true;
    }
    q[i] = fresh ? voxel_project(f, gx, gy, gz, zc[i]) : -1;
    smp[i] = fresh ? pack_sample((gx >> 3) - bx0, (gy >> 3) - by0, (gz >> 3) - bz0,
                                 local_index(gx, gy, gz))
                   : 0u;
  }
  float d2[C];
#pragma unroll
  for (int i = 0; i < C; ++i) d2[i] = q[i] >= 0 ? load_depth(f, q[i]) : 0.0f;
  unsigned acc = 0;
#pragma unroll
  for (int i = 0; i < C; ++i) {
    const bool a = q[i] >= 0 && voxel_accept(f, d2[i], zc[i]);
    acc |= a ? (1u << i) : 0u;
    if (TSDF) tv[i] = a ? tsdf_value(f, r.d, zc[i]) : 0.0f;
    if (!a) smp[i] = 0u;
  }
  return acc;
}

// The whole band walk of one point in packed form (all 2M+1 samples).
template <int M, bool TSDF = true>
__device__ __forceinline__ unsigned walk_point_packed(const FrameArgs& f, const Ray& r,
                                                      unsigned* smp, float* tv, int& bx0,
                                                      int& by0, int& bz0) {
  return walk_point_span<M, 2 * M + 1, TSDF>(f, r, 0, 2 * M + 1, smp, tv, bx0, by0, bz0);
}


// ----------------------------------------------------------------------------
// table access
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int load_idx_volatile(const Entry* e) {
  return *reinterpret_cast<const volatile int*>(&e->idx);
}

__device__ __forceinline__ unsigned int load_err_volatile(const Header* h) {
  return *reinterpret_cast<const volatile unsigned int*>(&h->err);
}

// Probe-load policies for stage A (Section 6.2: L1 residency of the probe
// decides speed; a GPU-scope atomic load bypasses L1).
enum ProbeLoad { kLoadCached = 0, kLoadL2 = 1, kLoadRelaxed = 2 };

template <int P>
__device__ __forceinline__ void load_entry(const Entry* e, unsigned long long& key, int& idx) {
  unsigned long long a, b;
  if (P == kLoadCached) {
    asm volatile("ld.global.ca.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(e) : "memory");
  } else if (P == kLoadL2) {
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(e) : "memory");
  } else {
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(a) : "l"(&e->key) : "memory");
    unsigned int i;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(i) : "l"(&e->idx) : "memory");
    b = i;
  }
  key = a;
  idx = static_cast<int>(static_cast<unsigned int>(b & 0xFFFFFFFFull));
}

// Wait until the winner of a slot publishes its block index (Section 2.3,
// "Publication is two steps"). Bounded: gives up after vol.timeout_ns of
// %globaltimer (or an iteration cap), sets PUBLISH_TIMEOUT and returns -1.
static __device__ __noinline__ int wait_published(const VolumeArgs& vol, const Entry* e) {
  int idx = load_idx_volatile(e);
  if (idx != kUnpublished) return idx >= 0 ? idx : -1;
  const unsigned long long t0 = global_timer_ns();
  unsigned int ns = 32;
  for (unsigned int it = 0; it < (1u << 22); ++it) {
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
    idx = load_idx_volatile(e);
    if (idx != kUnpublished) return idx >= 0 ? idx : -1;
    if (global_timer_ns() - t0 > vol.timeout_ns) break;
  }
  atomicOr(&vol.hdr->err, TSDF_ERRBIT_PUBLISH_TIMEOUT);
  return -1;
}

// Checked builds: slot s inside the table (else the BOUNDS bit, and the
// caller ends its probe).
__device__ __forceinline__ bool slot_ok(const VolumeArgs& vol, unsigned int s) {
  return index_ok(s, vol.slots, &vol.hdr->err);
}

// Writes a new block's coordinates at pool index i (checked builds: i inside
// the pool).
__device__ __forceinline__ void store_coords(const VolumeArgs& vol, unsigned int i, int bx, int by,
                                             int bz) {
  if (!index_ok(i, vol.pool, &vol.hdr->err)) return;
  int32_t* c = vol.coords + 3 * static_cast<size_t>(i);
  c[0] = bx;
  c[1] = by;
  c[2] = bz;
}

__device__ __forceinline__ void red_add_u32(unsigned int* p, unsigned int v) {
  asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// A scan that ran out of probes: with the unbounded probe that means every
// slot was visited, which is reported; a bounded probe (negative control)
// gives up without a trace.
__device__ __forceinline__ void probe_exhausted(const VolumeArgs& vol) {
  if (vol.probe_limit >= vol.slots) atomicOr(&vol.hdr->err, TSDF_ERRBIT_TABLE_FULL);
}

// Insert protocol of Listing 1 (Section 2.3): linear probe from the home slot;
// a plain load of the entry; on EMPTY a 64-bit compare-exchange; the winner
// takes a pool index from the counter, writes the block coordinate, fences and
// publishes the index; a thread that finds the key waits for publication.
// After a lost exchange the slot is re-examined with the key that won it (a
// set slot never changes, so if it holds our key this is a hit; moving on
// would duplicate the key). The scan is bounded only by the table size; a full
// scan reports TABLE_FULL (vol.probe_limit may lower the bound for the
// negative control). With vol.slot_index the slot is the pool index: the
// winner only counts the block, a thread that finds its key has its index at
// once, and nothing is published or waited for. Returns the pool index or -1
// on error.
// WAIT = false is the stage-A form used by fallbacks of the tile kernel: a
// thread that finds its key returns without waiting (returns 0), and the
// winner publishes without a fence (see warp_insert_nowait).
template <int P, bool WAIT = true>
__device__ int insert_block(const VolumeArgs& vol, unsigned long long key, int bx, int by,
                            int bz) {
  unsigned int s = hash_block(bx, by, bz) & vol.mask;
  for (unsigned int probe = 0; probe < vol.probe_limit; ++probe, s = (s + 1) & vol.mask) {
    if (!slot_ok(vol, s)) return -1;
    Entry* e = vol.table + s;
    unsigned long long k;
    int idx;
    load_entry<P>(e, k, idx);
    if (k == kEmptyKey) {
      const unsigned long long prev = atomicCAS(&e->key, kEmptyKey, key);
      if (prev == kEmptyKey) {
        if (vol.slot_index) {
          red_add_u32(&vol.hdr->count, 1u);  // counted only; the slot is the index
          return static_cast<int>(s);
        }
        const unsigned int i = atomicAdd(&vol.hdr->count, 1u);
        if (i >= vol.pool) {
          atomicOr(&vol.hdr->err, TSDF_ERRBIT_POOL_FULL);
          atomicExch(&e->idx, kFailedIdx);
          return -1;
        }
        store_coords(vol, i, bx, by, bz);
        if (WAIT) __threadfence();  // coordinates visible before the index
        atomicExch(&e->idx, static_cast<int>(i));
        return static_cast<int>(i);
      }
      k = prev;
      idx = kUnpublished;
    }
    if (k == key) {
      if (vol.slot_index) return static_cast<int>(s);
      if (!WAIT) return 0;
      return idx >= 0 ? idx : wait_published(vol, e);
    }
    // a poisoned volume stops long scans early
    if ((probe & 255u) == 255u &&
        (load_err_volatile(vol.hdr) & (TSDF_ERRBIT_POOL_FULL | TSDF_ERRBIT_TABLE_FULL)))
      return -1;
  }
  probe_exhausted(vol);
  return -1;
}

// Long probe chains, warp-cooperatively (at high load the multiply-xor hash
// leaves long clusters of occupied slots; probing them one slot per step
// costs one round trip per slot). Every lane of the warp calls it after a
// probe step. Each lane that has already probed kCoopAfter slots or more
// without finishing is taken in turn: the 32 lanes read 32 consecutive slots
// of its chain at once, and its slot jumps to the first one that holds its
// key or is empty -- the slot sequential probing would stop at, since an
// occupied slot never changes (a stale EMPTY read only makes it stop early,
// and the step then re-examines the slot). The scan never passes the probe
// limit.
constexpr unsigned kCoopAfter = 4;

__device__ __forceinline__ void warp_skip_long_chains(const VolumeArgs& vol,
                                                      unsigned long long key, bool& todo,
                                                      unsigned int& s, unsigned int& probe) {
  const unsigned lane = threadIdx.x & 31u;
  unsigned longs = __ballot_sync(0xffffffffu, todo && probe >= kCoopAfter);
  while (longs) {
    const int L = __ffs(longs) - 1;
    longs &= longs - 1;
    const unsigned long long lkey = __shfl_sync(0xffffffffu, key, L);
    unsigned int ls = __shfl_sync(0xffffffffu, s, L);
    unsigned int lprobe = __shfl_sync(0xffffffffu, probe, L);
    bool found = false, stopped = false;
    for (unsigned int step = 0; !found && lprobe < vol.probe_limit; ++step) {
      // a poisoned volume stops long scans early (every 8 windows)
      if ((step & 7u) == 7u &&
          (load_err_volatile(vol.hdr) & (TSDF_ERRBIT_POOL_FULL | TSDF_ERRBIT_TABLE_FULL))) {
        stopped = true;
        break;
      }
      const unsigned int left = vol.probe_limit - lprobe;
      const unsigned int window = left < 32u ? left : 32u;
      unsigned long long k = 0;
      if (lane < window && slot_ok(vol, (ls + lane) & vol.mask)) {
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];"
                     : "=l"(k)
                     : "l"(&vol.table[(ls + lane) & vol.mask].key)
                     : "memory");
      }
      const unsigned stop = __ballot_sync(0xffffffffu, lane < window && (k == kEmptyKey || k == lkey));
      if (stop) {
        const unsigned off = static_cast<unsigned>(__ffs(stop) - 1);
        ls = (ls + off) & vol.mask;
        lprobe += off;
        found = true;
      } else {
        ls = (ls + window) & vol.mask;
        lprobe += window;
      }
    }
    if (static_cast<int>(lane) == L) {
      s = ls;
      probe = lprobe;
      if (stopped) {
        todo = false;
      } else if (!found) {
        probe_exhausted(vol);
        todo = false;
      }
    }
  }
}

// Stage A insert without waiting, warp-cooperative: every lane of the warp
// calls it, each with at most one key (`has`). The probe and compare-exchange
// follow Listing 1 (Section 2.3) with the lost-CAS reading (re-examine the
// slot with the key that won it). Two differences, both safe because stage A
// is a pass of its own:
//  * a lane that finds its key already present returns at once: nothing in
//    this pass consumes the index, and the kernel boundary publishes every
//    index before stage B reads any;
//  * the lanes that win a slot in the same probe step take their pool indices
//    with ONE atomicAdd on the block counter (warp aggregation), and store the
//    index without a fence (no reader in this pass needs coordinates before
//    the index).
template <int P>
__device__ void warp_insert_nowait(const VolumeArgs& vol, unsigned long long key, bool has) {
  const unsigned lane = threadIdx.x & 31u;
  int bx = 0, by = 0, bz = 0;
  if (has) unpack_key(key, bx, by, bz);
  unsigned int s = has ? (hash_block(bx, by, bz) & vol.mask) : 0u;
  bool todo = has;
  unsigned int probe = 0, rounds = 0;
  while (__any_sync(0xffffffffu, todo)) {
    bool won = false;
    if (todo && !slot_ok(vol, s)) todo = false;
    Entry* e = vol.table + s;
    if (todo) {
      unsigned long long k;
      int idx;
      load_entry<P>(e, k, idx);
      if (k == kEmptyKey) {
        const unsigned long long prev = atomicCAS(&e->key, kEmptyKey, key);
        if (prev == kEmptyKey) {
          won = true;
          todo = false;
        } else {
          k = prev;
        }
      }
      if (todo) {
        if (k == key) {
          todo = false;
        } else {
          s = (s + 1) & vol.mask;
          if (++probe >= vol.probe_limit) {
            probe_exhausted(vol);
            todo = false;
          } else if ((probe & 255u) == 0u &&
                     (load_err_volatile(vol.hdr) &
                      (TSDF_ERRBIT_POOL_FULL | TSDF_ERRBIT_TABLE_FULL))) {
            todo = false;
          }
        }
      }
    }
    const unsigned wins = __ballot_sync(0xffffffffu, won);
    if (wins && vol.slot_index) {
      // the slot is the index: the block only has to be counted
      if (static_cast<int>(lane) == __ffs(wins) - 1) red_add_u32(&vol.hdr->count, __popc(wins));
    } else if (wins) {
      const int leader = __ffs(wins) - 1;
      unsigned base = 0;
      if (static_cast<int>(lane) == leader) base = atomicAdd(&vol.hdr->count, __popc(wins));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (won) {
        const unsigned i = base + __popc(wins & ((1u << lane) - 1u));
        if (i >= vol.pool) {
          atomicOr(&vol.hdr->err, TSDF_ERRBIT_POOL_FULL);
          atomicExch(&e->idx, kFailedIdx);
        } else {
          store_coords(vol, i, bx, by, bz);
          *reinterpret_cast<volatile int*>(&e->idx) = static_cast<int>(i);
        }
      }
    }
    // (a warp-uniform gate: short chains, the common case, never pay for it)
    if (++rounds >= kCoopAfter) warp_skip_long_chains(vol, key, todo, s, probe);
  }
}

// Stage A/fused insert that also yields the index, warp-cooperative: like
// warp_insert_nowait, but a lane that finds its key waits (bounded) for the
// winner to publish the index. Returns the pool index, or -1 on error (the
// error bit is set).
template <int P>
__device__ int warp_insert_get(const VolumeArgs& vol, unsigned long long key, bool has) {
  const unsigned lane = threadIdx.x & 31u;
  int bx = 0, by = 0, bz = 0;
  if (has) unpack_key(key, bx, by, bz);
  unsigned int s = has ? (hash_block(bx, by, bz) & vol.mask) : 0u;
  bool todo = has;
  unsigned int probe = 0, rounds = 0;
  int result = -1;
  const Entry* hit = nullptr;
  while (__any_sync(0xffffffffu, todo)) {
    bool won = false;
    if (todo && !slot_ok(vol, s)) todo = false;
    Entry* e = vol.table + s;
    if (todo) {
      unsigned long long k;
      int idx;
      load_entry<P>(e, k, idx);
      if (k == kEmptyKey) {
        const unsigned long long prev = atomicCAS(&e->key, kEmptyKey, key);
        if (prev == kEmptyKey) {
          won = true;
          todo = false;
        } else {
          k = prev;
          idx = kUnpublished;
        }
      }
      if (todo) {
        if (k == key) {
          todo = false;
          if (vol.slot_index)
            result = static_cast<int>(s);
          else if (idx >= 0)
            result = idx;
          else if (idx == kUnpublished)
            hit = e;  // wait below, outside the cooperative loop
        } else {
          s = (s + 1) & vol.mask;
          if (++probe >= vol.probe_limit) {
            probe_exhausted(vol);
            todo = false;
          } else if ((probe & 255u) == 0u &&
                     (load_err_volatile(vol.hdr) &
                      (TSDF_ERRBIT_POOL_FULL | TSDF_ERRBIT_TABLE_FULL))) {
            todo = false;
          }
        }
      }
    }
    const unsigned wins = __ballot_sync(0xffffffffu, won);
    if (wins && vol.slot_index) {
      if (static_cast<int>(lane) == __ffs(wins) - 1) red_add_u32(&vol.hdr->count, __popc(wins));
      if (won) result = static_cast<int>(s);
    } else if (wins) {
      const int leader = __ffs(wins) - 1;
      unsigned base = 0;
      if (static_cast<int>(lane) == leader) base = atomicAdd(&vol.hdr->count, __popc(wins));
      base = __shfl_sync(0xffffffffu, base, leader);
      if (won) {
        const unsigned i = base + __popc(wins & ((1u << lane) - 1u));
        if (i >= vol.pool) {
          atomicOr(&vol.hdr->err, TSDF_ERRBIT_POOL_FULL);
          atomicExch(&e->idx, kFailedIdx);
        } else {
          store_coords(vol, i, bx, by, bz);
          // Readers in this pass use the index only to address the pool, never
          // the coordinates, so no fence is needed before publishing it, and
          // a plain store is enough (nothing reads the old value).
          *reinterpret_cast<volatile int*>(&e->idx) = static_cast<int>(i);
          result = static_cast<int>(i);
        }
      }
    }
    // (a warp-uniform gate: short chains, the common case, never pay for it)
    if (++rounds >= kCoopAfter) warp_skip_long_chains(vol, key, todo, s, probe);
  }
  if (hit) result = wait_published(vol, hit);
  return result;
}

constexpr int kAbsent = -3;  // lookup: key not in the table

// Read-only lookup for stage B (after stage A's kernel has completed every
// publication): the table is read through the non-coherent read-only path.
// Returns the pool index, kFailedIdx (slot won but pool exhausted),
// kUnpublished (claimed but never published: an error) or kAbsent.
__device__ __forceinline__ int found_index(const VolumeArgs& vol, const ulonglong2& ent,
                                           unsigned int s) {
  return vol.slot_index ? static_cast<int>(s)
                        : static_cast<int>(static_cast<unsigned int>(ent.y & 0xFFFFFFFFull));
}

// The rest of a lookup whose first probe met another key, from slot s (probe
// number 1 on): the same slots in the same order, read four at a time with
// the four loads in flight together, so a chain of n slots costs about n/4
// round trips instead of n (the table does not change while lookups run).
// Out of line: at the loads a table is sized for, almost every lookup ends at
// its first probe.
static __device__ __noinline__ int lookup_chain(const VolumeArgs& vol, unsigned long long key,
                                                unsigned int s) {
  const ulonglong2* t = reinterpret_cast<const ulonglong2*>(vol.table);
  for (unsigned int probe = 1; probe < vol.probe_limit; probe += 4, s = (s + 4) & vol.mask) {
    if (!(slot_ok(vol, s) && slot_ok(vol, (s + 1) & vol.mask) && slot_ok(vol, (s + 2) & vol.mask) &&
          slot_ok(vol, (s + 3) & vol.mask)))
      return kAbsent;
    const ulonglong2 e0 = __ldg(t + s);
    const ulonglong2 e1 = __ldg(t + ((s + 1) & vol.mask));
    const ulonglong2 e2 = __ldg(t + ((s + 2) & vol.mask));
    const ulonglong2 e3 = __ldg(t + ((s + 3) & vol.mask));
    if (e0.x == key) return found_index(vol, e0, s);
    if (e0.x == kEmptyKey || probe + 1 >= vol.probe_limit) return kAbsent;
    if (e1.x == key) return found_index(vol, e1, (s + 1) & vol.mask);
    if (e1.x == kEmptyKey || probe + 2 >= vol.probe_limit) return kAbsent;
    if (e2.x == key) return found_index(vol, e2, (s + 2) & vol.mask);
    if (e2.x == kEmptyKey || probe + 3 >= vol.probe_limit) return kAbsent;
    if (e3.x == key) return found_index(vol, e3, (s + 3) & vol.mask);
    if (e3.x == kEmptyKey) return kAbsent;
  }
  return kAbsent;
}

__device__ __forceinline__ int lookup_block(const VolumeArgs& vol, unsigned long long key, int bx,
                                            int by, int bz) {
  const unsigned int s = hash_block(bx, by, bz) & vol.mask;
  if (!slot_ok(vol, s)) return kAbsent;
  const ulonglong2 ent = __ldg(reinterpret_cast<const ulonglong2*>(vol.table + s));
  if (ent.x == key) return found_index(vol, ent, s);
  if (ent.x == kEmptyKey || vol.probe_limit <= 1) return kAbsent;
  return lookup_chain(vol, key, (s + 1) & vol.mask);
}

// Stage B's view of a lookup: the pool index, or -1 to skip the contribution.
// A block that stage A claimed but never published cannot receive its
// contributions; that is reported (as PUBLISH_TIMEOUT), never silent.
__device__ __forceinline__ int resolve_for_update(const VolumeArgs& vol, int idx) {
  if (idx >= 0) return idx;
  if (idx == kUnpublished) atomicOr(&vol.hdr->err, TSDF_ERRBIT_PUBLISH_TIMEOUT);
  return -1;
}

// Stage B lookup, warp-cooperative (the tile strategy of stage B, after stage
// A's kernel has completed): every lane with a key probes its own chain, one
// slot per step, and chains still open after a few steps are fast-forwarded
// by the whole warp (warp_skip_long_chains stops at the first slot holding
// the key or empty, as the sequential probe would). Returns stage B's view:
// the pool index, or -1 to skip the contribution (see resolve_for_update).
template <int P>
__device__ int warp_lookup_get(const VolumeArgs& vol, unsigned long long key, bool has) {
  int bx = 0, by = 0, bz = 0;
  if (has) unpack_key(key, bx, by, bz);
  unsigned int s = has ? (hash_block(bx, by, bz) & vol.mask) : 0u;
  bool todo = has;
  unsigned int probe = 0, rounds = 0;
  int result = kAbsent;
  while (__any_sync(0xffffffffu, todo)) {
    if (todo && !slot_ok(vol, s)) todo = false;
    if (todo) {
      unsigned long long k;
      int idx;
      load_entry<P>(vol.table + s, k, idx);
      if (k == key) {
        todo = false;
        result = vol.slot_index ? static_cast<int>(s) : idx;
      } else if (k == kEmptyKey) {
        todo = false;
      } else {
        s = (s + 1) & vol.mask;
        if (++probe >= vol.probe_limit) todo = false;
      }
    }
    if (++rounds >= kCoopAfter) warp_skip_long_chains(vol, key, todo, s, probe);
  }
  return resolve_for_update(vol, result);
}

}  // namespace tsdf
