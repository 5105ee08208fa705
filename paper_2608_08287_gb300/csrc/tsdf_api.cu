// Host runtime of libtsdf: the C ABI declared in include/tsdf.h.
//
// A volume is one device allocation (header | table | block coordinates |
// five channel arrays) plus host-side state (parameters, options, a pinned
// status word, the poisoned flag, staging for host inputs). Every call checks
// its arguments before enqueuing anything and returns a status; no exception
// crosses the ABI.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "tsdf.h"
#include "tsdf_device.cuh"
#include "tsdf_internal.h"
#include "tsdf_launch.h"

using tsdf::align_up;
using tsdf::as_stream;
using tsdf::decode_err;
using tsdf::from_cuda;
using tsdf::kAlign;
using tsdf::Offsets;

namespace {

std::atomic<uint64_t> g_launches{0};

bool sizes_ok(uint32_t slots, uint32_t pool) {
  return slots >= 2 && (slots & (slots - 1)) == 0 && pool >= 1 && pool <= slots;
}

Offsets offsets_of(uint32_t slots, uint32_t pool) {
  Offsets o;
  size_t at = align_up(sizeof(tsdf::Header));
  o.table = at;
  at = align_up(at + static_cast<size_t>(slots) * sizeof(tsdf::Entry));
  o.coords = at;
  at = align_up(at + static_cast<size_t>(pool) * 3 * sizeof(int32_t));
  o.twrg = at;
  at = align_up(at + static_cast<size_t>(pool) * tsdf::kBlockVoxels * sizeof(float4));
  o.blue = at;
  at = align_up(at + static_cast<size_t>(pool) * tsdf::kBlockVoxels * sizeof(float));
  o.total = at;
  return o;
}

}  // namespace

namespace tsdf {
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

tsdf_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TSDF_OK;
  if (e == cudaErrorMemoryAllocation) return TSDF_ERR_OUT_OF_MEMORY;
  return TSDF_ERR_CUDA;
}

tsdf_status decode_err(uint32_t err) {
  if (err & TSDF_ERRBIT_POOL_FULL) return TSDF_ERR_POOL_FULL;
  if (err & TSDF_ERRBIT_TABLE_FULL) return TSDF_ERR_TABLE_FULL;
  if (err & TSDF_ERRBIT_PUBLISH_TIMEOUT) return TSDF_ERR_PUBLISH_TIMEOUT;
  if (err & TSDF_ERRBIT_BOUNDS) return TSDF_ERR_BOUNDS;
  return TSDF_OK;
}
}  // namespace tsdf

namespace {

// Enqueue the initialisation of an empty volume: table entries all-ones
// (key = EMPTY, index = -1), header zero, used prefix of the pool zero.
tsdf_status enqueue_clear(tsdf_volume* v, cudaStream_t s, bool whole_pool) {
  char* base = static_cast<char*>(v->mem);
  cudaError_t e;
  if (whole_pool) {
    e = cudaMemsetAsync(base + v->off.twrg, 0, v->off.total - v->off.twrg, s);
  } else {
    e = tsdf::launch_clear_used(v->va, v->sm_count, s);
  }
  if (e != cudaSuccess) return from_cuda(e);
  e = cudaMemsetAsync(base + v->off.table, 0xFF,
                      static_cast<size_t>(v->slots) * sizeof(tsdf::Entry), s);
  if (e != cudaSuccess) return from_cuda(e);
  e = cudaMemsetAsync(base, 0, sizeof(tsdf::Header), s);
  return from_cuda(e);
}

tsdf_status init_volume(tsdf_volume* v, void* mem, size_t bytes, bool owns, float voxel,
                        float trunc, uint32_t slots, uint32_t pool, cudaStream_t s) {
  v->voxel = voxel;
  v->trunc = trunc;
  v->half_band = static_cast<int>(lrintf(trunc / voxel));
  v->slots = slots;
  v->pool = pool;
  v->mem = mem;
  v->bytes = bytes;
  v->owns = owns;
  v->off = offsets_of(slots, pool);
  cudaError_t e = cudaGetDevice(&v->device);
  if (e != cudaSuccess) return from_cuda(e);
  e = cudaDeviceGetAttribute(&v->sm_count, cudaDevAttrMultiProcessorCount, v->device);
  if (e != cudaSuccess) return from_cuda(e);
  char* base = static_cast<char*>(mem);
  v->va.hdr = reinterpret_cast<tsdf::Header*>(base);
  v->va.table = reinterpret_cast<tsdf::Entry*>(base + v->off.table);
  v->va.mask = slots - 1;
  v->va.slots = slots;
  v->va.coords = reinterpret_cast<int32_t*>(base + v->off.coords);
  v->va.pool = pool;
  v->va.twrg = reinterpret_cast<float4*>(base + v->off.twrg);
  v->va.blue = reinterpret_cast<float*>(base + v->off.blue);
  v->va.timeout_ns = 1000000000ull;
  v->va.probe_limit = slots;
  v->va.slot_index = 0;
  e = cudaMallocHost(reinterpret_cast<void**>(&v->pinned), 2 * sizeof(uint32_t));
  if (e != cudaSuccess) {
    v->pinned = nullptr;
    return TSDF_ERR_OUT_OF_MEMORY;
  }
  return enqueue_clear(v, s, true);
}

bool params_ok(float voxel, float trunc) {
  if (!(std::isfinite(voxel) && voxel > 0.0f)) return false;
  if (!(std::isfinite(trunc) && trunc >= voxel)) return false;
  const long m = lrintf(trunc / voxel);
  return m >= 1 && m <= tsdf::kMaxHalfBand;
}

tsdf_status read_header(tsdf_volume* v, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(v->pinned, v->mem, 2 * sizeof(uint32_t),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

}  // namespace

namespace tsdf {
tsdf_status make_frame(const tsdf_volume* v, const float* depth, int w, int h,
                       const tsdf_intrinsics* intr, const tsdf_pose* pose, const uint8_t* rgb,
                       FrameArgs* f) {
  if (!v || !depth || !intr || !pose) return TSDF_ERR_INVALID_ARG;
  if (w < 1 || h < 1 || w > 32768 || h > 32768) return TSDF_ERR_INVALID_ARG;
  if (!(std::isfinite(intr->fx) && std::isfinite(intr->fy) && std::isfinite(intr->cx) &&
        std::isfinite(intr->cy) && intr->fx != 0.0f && intr->fy != 0.0f))
    return TSDF_ERR_INVALID_ARG;
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(pose->m[i])) return TSDF_ERR_INVALID_ARG;
  f->depth = depth;
  f->rgb = rgb;
  f->W = w;
  f->H = h;
  f->fx = intr->fx;
  f->fy = intr->fy;
  f->cx = intr->cx;
  f->cy = intr->cy;
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) f->R[3 * i + j] = pose->m[4 * i + j];
    f->t[i] = pose->m[4 * i + 3];
  }
  // The voxel-centre map c = A g + b, A = v R^T, b = R^T (v/2 - t), in this
  // fixed order of single-precision operations (the library is built with
  // contraction off, and the fused steps are explicit).
  float half_minus_t[3];
  for (int i = 0; i < 3; ++i) half_minus_t[i] = std::fmaf(0.5f, v->voxel, -f->t[i]);
  for (int j = 0; j < 3; ++j) {
    for (int i = 0; i < 3; ++i) f->A[3 * j + i] = v->voxel * f->R[3 * i + j];
    f->b[j] = std::fmaf(f->R[6 + j], half_minus_t[2],
                        std::fmaf(f->R[3 + j], half_minus_t[1], f->R[j] * half_minus_t[0]));
  }
  f->v = v->voxel;
  f->inv_v = 1.0f / v->voxel;
  f->tau = v->trunc;
  f->neg_tau = -v->trunc;
  f->inv_tau = 1.0f / v->trunc;
  f->M = v->half_band;
  f->err = &v->va.hdr->err;
  return TSDF_OK;
}

int auto_threads_per_point(int fuse_mode, int probe_load, int half_band, int sm_count,
                           long long tiles) {
  if (fuse_mode != 2 || probe_load != kLoadCached ||
      (half_band != 2 && half_band != 4 && half_band != 8))
    return 1;
  const long long slots = 4ll * (sm_count > 0 ? sm_count : 1);
  int t = 1;
  while (t < 4 && tiles * (2 * t) <= slots) t *= 2;
  return t;
}

}  // namespace tsdf

using tsdf::make_frame;

namespace {

// Threads per point of the fused tile kernel for a width x height frame: an
// explicit setting as it is, else the automatic choice.
int threads_per_point(const tsdf_volume* vol, int width, int height) {
  if (vol->fuse_mode != 2) return 1;
  if (vol->threads_per_point != 0) return vol->threads_per_point;
  return tsdf::auto_threads_per_point(vol->fuse_mode, vol->probe_load, vol->half_band,
                                      vol->sm_count, tsdf::tiles_of_frame(width, height));
}

// Host-side header of a checkpoint, followed by the volume's whole device
// allocation.
struct CheckpointHeader {
  char magic[8];
  float voxel, trunc;
  uint32_t slots, pool, slot_index, poisoned, dirty, pad;
  uint64_t bytes;  // device bytes that follow
  uint8_t reserved[16];
};
static_assert(sizeof(CheckpointHeader) == 64, "the checkpoint header is 64 bytes");
constexpr char kCheckpointMagic[8] = {'T', 'S', 'D', 'F', 'C', 'K', 'P', '1'};

bool on_volume_device(const tsdf_volume* vol) {
  int dev = 0;
  return cudaGetDevice(&dev) == cudaSuccess && dev == vol->device;
}

}  // namespace

extern "C" {

size_t tsdf_volume_bytes(uint32_t table_slots, uint32_t pool_blocks) {
  if (!sizes_ok(table_slots, pool_blocks)) return 0;
  return offsets_of(table_slots, pool_blocks).total;
}

tsdf_status tsdf_volume_create(float voxel_size, float truncation, uint32_t table_slots,
                               uint32_t pool_blocks, tsdf_volume** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!sizes_ok(table_slots, pool_blocks) || !params_ok(voxel_size, truncation))
    return TSDF_ERR_INVALID_ARG;
  const size_t bytes = tsdf_volume_bytes(table_slots, pool_blocks);
  void* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TSDF_ERR_OUT_OF_MEMORY;
  }
  tsdf_volume* v = new (std::nothrow) tsdf_volume();
  if (!v) {
    cudaFree(mem);
    return TSDF_ERR_OUT_OF_MEMORY;
  }
  tsdf_status st = init_volume(v, mem, bytes, true, voxel_size, truncation, table_slots,
                               pool_blocks, nullptr);
  if (st == TSDF_OK) st = from_cuda(cudaStreamSynchronize(nullptr));
  if (st != TSDF_OK) {
    tsdf_volume_destroy(v);
    return st;
  }
  *out = v;
  return TSDF_OK;
}

tsdf_status tsdf_volume_create_in(void* dev_mem, size_t bytes, float voxel_size,
                                  float truncation, uint32_t table_slots,
                                  uint32_t pool_blocks, void* stream, tsdf_volume** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (!dev_mem || (reinterpret_cast<uintptr_t>(dev_mem) % kAlign) != 0)
    return TSDF_ERR_INVALID_ARG;
  if (!sizes_ok(table_slots, pool_blocks) || !params_ok(voxel_size, truncation))
    return TSDF_ERR_INVALID_ARG;
  if (bytes < tsdf_volume_bytes(table_slots, pool_blocks)) return TSDF_ERR_INVALID_ARG;
  tsdf_volume* v = new (std::nothrow) tsdf_volume();
  if (!v) return TSDF_ERR_OUT_OF_MEMORY;
  const tsdf_status st = init_volume(v, dev_mem, bytes, false, voxel_size, truncation,
                                     table_slots, pool_blocks, as_stream(stream));
  if (st != TSDF_OK) {
    tsdf_volume_destroy(v);
    return st;
  }
  *out = v;
  return TSDF_OK;
}

tsdf_status tsdf_volume_reset(tsdf_volume* vol, void* stream) {
  if (!vol) return TSDF_ERR_INVALID_ARG;
  const tsdf_status st = enqueue_clear(vol, as_stream(stream), false);
  if (st == TSDF_OK) {
    vol->poisoned = false;
    vol->dirty = false;
  }
  return st;
}

void tsdf_volume_destroy(tsdf_volume* vol) {
  if (!vol) return;
  cudaDeviceSynchronize();
  if (vol->owns && vol->mem) cudaFree(vol->mem);
  if (vol->stage) cudaFree(vol->stage);
  if (vol->stream_stage) cudaFree(vol->stream_stage);
  if (vol->err_words) cudaFreeHost(vol->err_words);
  if (vol->err_gathered) cudaFreeHost(vol->err_gathered);
  if (vol->err_dev) cudaFree(vol->err_dev);
  for (int b = 0; b < 2; ++b) {
    if (vol->ev_copied[b]) cudaEventDestroy(vol->ev_copied[b]);
    if (vol->ev_free[b]) cudaEventDestroy(vol->ev_free[b]);
  }
  if (vol->copy_stream) cudaStreamDestroy(vol->copy_stream);
  if (vol->pinned) cudaFreeHost(vol->pinned);
  delete vol;
}

tsdf_status tsdf_volume_set_option(tsdf_volume* vol, tsdf_option opt, int64_t value) {
  if (!vol) return TSDF_ERR_INVALID_ARG;
  switch (opt) {
    case TSDF_OPT_PROBE_LOAD:
      if (value < 0 || value > 2) return TSDF_ERR_INVALID_ARG;
      if (value != tsdf::kLoadCached && vol->threads_per_point > 1)
        return TSDF_ERR_INVALID_ARG;  // the split walk exists for the default load only
      vol->probe_load = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_PUBLISH_TIMEOUT_NS:
      if (value < 1000 || value > 10000000000ll) return TSDF_ERR_INVALID_ARG;
      vol->va.timeout_ns = static_cast<unsigned long long>(value);
      return TSDF_OK;
    case TSDF_OPT_INTEGRATE_MODE:
      if (value < 0 || value > 2) return TSDF_ERR_INVALID_ARG;
      vol->integrate_mode = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_THREADS:
      if (value != 256) return TSDF_ERR_INVALID_ARG;
      vol->threads = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_ALLOCATE_MODE:
      if (value < 0 || value > 2) return TSDF_ERR_INVALID_ARG;
      vol->allocate_mode = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_FUSE_MODE:
      if (value < 0 || value > 2) return TSDF_ERR_INVALID_ARG;
      vol->fuse_mode = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_SLOT_INDEX:
      if (value < 0 || value > 1) return TSDF_ERR_INVALID_ARG;
      if (value == 1 && vol->pool != vol->slots) return TSDF_ERR_INVALID_ARG;
      if (vol->dirty && static_cast<unsigned int>(value) != vol->va.slot_index)
        return TSDF_ERR_INVALID_ARG;  // the layout of the stored blocks would change
      vol->va.slot_index = static_cast<unsigned int>(value);
      return TSDF_OK;
    case TSDF_OPT_THREADS_PER_POINT:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
        return TSDF_ERR_INVALID_ARG;
      if (value > 1 && (vol->probe_load != tsdf::kLoadCached ||
                         (vol->half_band != 2 && vol->half_band != 4 && vol->half_band != 8)))
        return TSDF_ERR_INVALID_ARG;
      vol->threads_per_point = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_PROBE_BOUND:
      if (value < 0) return TSDF_ERR_INVALID_ARG;
      vol->va.probe_limit = (value == 0 || value >= static_cast<int64_t>(vol->slots))
                                ? vol->slots
                                : static_cast<unsigned int>(value);
      return TSDF_OK;
    default:
      break;
  }
  return TSDF_ERR_INVALID_ARG;
}

tsdf_status tsdf_volume_layout(const tsdf_volume* vol, tsdf_layout* out) {
  if (!vol || !out) return TSDF_ERR_INVALID_ARG;
  std::memset(out, 0, sizeof(*out));
  out->base = vol->mem;
  out->bytes = vol->off.total;
  out->block_count = &vol->va.hdr->count;
  out->error_word = &vol->va.hdr->err;
  out->table = vol->va.table;
  out->block_coords = vol->va.coords;
  out->voxel_sums = reinterpret_cast<float*>(vol->va.twrg);
  out->blue_sums = vol->va.blue;
  out->voxel_sums_offset = vol->off.twrg;
  out->blue_sums_offset = vol->off.blue;
  out->table_slots = vol->slots;
  out->pool_blocks = vol->pool;
  out->table_offset = vol->off.table;
  out->coords_offset = vol->off.coords;
  return TSDF_OK;
}

tsdf_status tsdf_allocate_async(tsdf_volume* vol, const float* depth_dev, int width,
                                int height, const tsdf_intrinsics* intr,
                                const tsdf_pose* pose, void* stream) {
  tsdf::FrameArgs f;
  tsdf_status st = make_frame(vol, depth_dev, width, height, intr, pose, nullptr, &f);
  if (st != TSDF_OK) return st;
  if (vol->poisoned) return TSDF_ERR_POISONED;
  vol->dirty = true;
  return from_cuda(tsdf::launch_allocate(f, vol->va, vol->probe_load, vol->allocate_mode, as_stream(stream)));
}

tsdf_status tsdf_integrate_async(tsdf_volume* vol, const float* depth_dev, int width,
                                 int height, const tsdf_intrinsics* intr,
                                 const tsdf_pose* pose, const uint8_t* rgb_dev,
                                 void* stream) {
  tsdf::FrameArgs f;
  tsdf_status st = make_frame(vol, depth_dev, width, height, intr, pose, rgb_dev, &f);
  if (st != TSDF_OK) return st;
  if (vol->poisoned) return TSDF_ERR_POISONED;
  vol->dirty = true;
  return from_cuda(tsdf::launch_integrate(f, vol->va, vol->integrate_mode, as_stream(stream)));
}

tsdf_status tsdf_fuse_frame_async(tsdf_volume* vol, const float* depth_dev, int width,
                                  int height, const tsdf_intrinsics* intr,
                                  const tsdf_pose* pose, const uint8_t* rgb_dev,
                                  void* stream) {
  tsdf::FrameArgs f;
  tsdf_status st = make_frame(vol, depth_dev, width, height, intr, pose, rgb_dev, &f);
  if (st != TSDF_OK) return st;
  if (vol->poisoned) return TSDF_ERR_POISONED;
  vol->dirty = true;
  if (vol->fuse_mode != 0)
    return from_cuda(tsdf::launch_fused(f, vol->va, vol->probe_load, vol->fuse_mode,
                                        threads_per_point(vol, width, height),
                                        as_stream(stream)));
  cudaError_t e = tsdf::launch_allocate(f, vol->va, vol->probe_load, vol->allocate_mode,
                                        as_stream(stream));
  if (e == cudaSuccess) e = tsdf::launch_integrate(f, vol->va, vol->integrate_mode,
                                                   as_stream(stream));
  return from_cuda(e);
}

tsdf_status tsdf_volume_status(tsdf_volume* vol, void* stream) {
  if (!vol) return TSDF_ERR_INVALID_ARG;
  const tsdf_status st = read_header(vol, as_stream(stream));
  if (st != TSDF_OK) return st;
  const tsdf_status dev = decode_err(vol->pinned[1]);
  if (dev != TSDF_OK) vol->poisoned = true;
  return dev;
}

tsdf_status tsdf_fuse_frame(tsdf_volume* vol, const float* depth_dev, int width, int height,
                            const tsdf_intrinsics* intr, const tsdf_pose* pose,
                            const uint8_t* rgb_dev, void* stream) {
  const tsdf_status st =
      tsdf_fuse_frame_async(vol, depth_dev, width, height, intr, pose, rgb_dev, stream);
  if (st != TSDF_OK) return st;
  return tsdf_volume_status(vol, stream);
}

tsdf_status tsdf_fuse_frame_host(tsdf_volume* vol, const float* depth_host, int width,
                                 int height, const tsdf_intrinsics* intr,
                                 const tsdf_pose* pose, const uint8_t* rgb_host,
                                 void* stream) {
  tsdf::FrameArgs f;
  tsdf_status st = make_frame(vol, depth_host, width, height, intr, pose, rgb_host, &f);
  if (st != TSDF_OK) return st;
  if (vol->poisoned) return TSDF_ERR_POISONED;
  const size_t npx = static_cast<size_t>(width) * height;
  const size_t dbytes = align_up(npx * sizeof(float));
  const size_t need = dbytes + (rgb_host ? npx * 3 : 0);
  if (vol->stage_bytes < need) {
    if (vol->stage) {
      cudaStreamSynchronize(as_stream(stream));
      cudaFree(vol->stage);
      vol->stage = nullptr;
      vol->stage_bytes = 0;
    }
    if (cudaMalloc(&vol->stage, need) != cudaSuccess) {
      cudaGetLastError();
      return TSDF_ERR_OUT_OF_MEMORY;
    }
    vol->stage_bytes = need;
  }
  char* sbase = static_cast<char*>(vol->stage);
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(sbase, depth_host, npx * sizeof(float),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && rgb_host)
    e = cudaMemcpyAsync(sbase + dbytes, rgb_host, npx * 3, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return from_cuda(e);
  return tsdf_fuse_frame(vol, reinterpret_cast<const float*>(sbase), width, height, intr, pose,
                         rgb_host ? reinterpret_cast<const uint8_t*>(sbase + dbytes) : nullptr,
                         stream);
}

tsdf_status tsdf_volume_block_count(tsdf_volume* vol, void* stream, uint32_t* n) {
  if (!vol || !n) return TSDF_ERR_INVALID_ARG;
  const tsdf_status st = read_header(vol, as_stream(stream));
  if (st != TSDF_OK) return st;
  *n = vol->pinned[0] < vol->pool ? vol->pinned[0] : vol->pool;
  return TSDF_OK;
}

tsdf_status tsdf_export_blocks(tsdf_volume* vol, int32_t* coords_host, float* voxels_host,
                               uint32_t capacity, uint32_t* n_out, void* stream) {
  if (!vol || !n_out) return TSDF_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  uint32_t n = 0;
  tsdf_status st = tsdf_volume_block_count(vol, stream, &n);
  if (st != TSDF_OK) return st;
  *n_out = n;
  if (!coords_host && !voxels_host) return TSDF_OK;
  if (capacity < n) return TSDF_ERR_INVALID_ARG;
  if (n == 0) return TSDF_OK;
  cudaError_t e = cudaSuccess;
  const int32_t* coords_dev = vol->va.coords;
  const unsigned int* list = nullptr;
  char* scratch = nullptr;
  if (vol->va.slot_index) {
    // the blocks sit at their slots: list the occupied slots first
    const size_t list_bytes = align_up(static_cast<size_t>(n) * sizeof(unsigned int));
    const size_t coord_bytes = align_up(static_cast<size_t>(n) * 3 * sizeof(int32_t));
    e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), list_bytes + coord_bytes + kAlign, s);
    if (e == cudaSuccess) {
      list = reinterpret_cast<const unsigned int*>(scratch);
      coords_dev = reinterpret_cast<const int32_t*>(scratch + list_bytes);
      e = tsdf::launch_slot_list(vol->va, reinterpret_cast<unsigned int*>(scratch),
                                 reinterpret_cast<int32_t*>(scratch + list_bytes), n,
                                 reinterpret_cast<unsigned int*>(scratch + list_bytes +
                                                                 coord_bytes),
                                 s);
    }
  }
  if (e == cudaSuccess && coords_host)
    e = cudaMemcpyAsync(coords_host, coords_dev, static_cast<size_t>(n) * 3 * sizeof(int32_t),
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && voxels_host) {
    const size_t bytes = static_cast<size_t>(n) * 5 * tsdf::kBlockVoxels * sizeof(float);
    float* tmp = nullptr;
    e = cudaMallocAsync(reinterpret_cast<void**>(&tmp), bytes, s);
    if (e == cudaSuccess) {
      e = tsdf::launch_export(vol->va, tmp, n, list, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(voxels_host, tmp, bytes, cudaMemcpyDeviceToHost, s);
      const cudaError_t e2 = cudaFreeAsync(tmp, s);
      if (e == cudaSuccess) e = e2;
    }
  }
  if (scratch) {
    const cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

tsdf_status tsdf_extract_mesh_async(tsdf_volume* vol, float* triangles_dev, int32_t* cells_dev,
                                    uint32_t capacity, uint32_t* count_dev, void* stream) {
  if (!vol || !count_dev) return TSDF_ERR_INVALID_ARG;
  if (capacity && !triangles_dev && !cells_dev) return TSDF_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(triangles_dev) % alignof(float)) != 0 ||
      (reinterpret_cast<uintptr_t>(cells_dev) % 16) != 0 ||
      (reinterpret_cast<uintptr_t>(count_dev) % alignof(uint32_t)) != 0)
    return TSDF_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMemsetAsync(count_dev, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess)
    e = tsdf::launch_extract(vol->va, vol->voxel, triangles_dev, cells_dev, capacity, count_dev,
                             vol->sm_count, s);
  return from_cuda(e);
}

tsdf_status tsdf_extract_mesh(tsdf_volume* vol, float* triangles_host, int32_t* cells_host,
                              uint32_t capacity, uint32_t* n_out, tsdf_extract_timing* timing,
                              void* stream) {
  if (!vol || !n_out) return TSDF_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  const bool fetch = (triangles_host || cells_host) && capacity > 0;
  const size_t tri_bytes = triangles_host ? static_cast<size_t>(capacity) * 9 * sizeof(float) : 0;
  const size_t cell_bytes = cells_host ? static_cast<size_t>(capacity) * 4 * sizeof(int32_t) : 0;
  char* buf = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
  if (e == cudaSuccess)
    e = cudaMallocAsync(reinterpret_cast<void**>(&buf),
                        kAlign + (fetch ? align_up(tri_bytes) + cell_bytes : 0), s);
  uint32_t* counter = reinterpret_cast<uint32_t*>(buf);
  float* tris = fetch && triangles_host ? reinterpret_cast<float*>(buf + kAlign) : nullptr;
  int32_t* cells =
      fetch && cells_host ? reinterpret_cast<int32_t*>(buf + kAlign + align_up(tri_bytes)) : nullptr;
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
  tsdf_status st = from_cuda(e);
  if (st == TSDF_OK)
    st = tsdf_extract_mesh_async(vol, tris, cells, fetch ? capacity : 0, counter, stream);
  if (st == TSDF_OK) st = from_cuda(cudaEventRecord(ev[1], s));
  if (st == TSDF_OK)
    st = from_cuda(cudaMemcpyAsync(vol->pinned, counter, sizeof(uint32_t),
                                   cudaMemcpyDeviceToHost, s));
  if (st == TSDF_OK) st = from_cuda(cudaStreamSynchronize(s));
  uint32_t n = 0;
  if (st == TSDF_OK) {
    n = vol->pinned[0];
    *n_out = n;
    if (fetch && n > capacity) st = TSDF_ERR_INVALID_ARG;  // nothing is copied
  }
  float d2h_ms = 0.0f, compute_ms = 0.0f;
  if (st == TSDF_OK && fetch && n > 0) {
    e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess && triangles_host)
      e = cudaMemcpyAsync(triangles_host, tris, static_cast<size_t>(n) * 9 * sizeof(float),
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && cells_host)
      e = cudaMemcpyAsync(cells_host, cells, static_cast<size_t>(n) * 4 * sizeof(int32_t),
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&d2h_ms, ev[2], ev[3]);
    st = from_cuda(e);
  }
  if (st == TSDF_OK) st = from_cuda(cudaEventElapsedTime(&compute_ms, ev[0], ev[1]));
  if (buf) cudaFreeAsync(buf, s);
  cudaStreamSynchronize(s);
  for (int i = 0; i < 4; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (st == TSDF_OK && timing) {
    timing->compute_ms = compute_ms;
    timing->d2h_ms = d2h_ms;
    timing->d2h_bytes = fetch ? static_cast<uint64_t>(n) *
                                    ((triangles_host ? 36u : 0u) + (cells_host ? 16u : 0u))
                              : 0;
  }
  return st;
}

tsdf_status tsdf_volume_table_stats(tsdf_volume* vol, void* stream, tsdf_table_stats* out) {
  if (!vol || !out) return TSDF_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  tsdf::TableStatsDev* dev = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dev), sizeof(*dev), s);
  if (e != cudaSuccess) return from_cuda(e);
  tsdf::TableStatsDev host{};
  e = cudaMemsetAsync(dev, 0, sizeof(*dev), s);
  if (e == cudaSuccess) e = tsdf::launch_table_stats(vol->va, dev, vol->sm_count, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&host, dev, sizeof(host), cudaMemcpyDeviceToHost, s);
  const cudaError_t e2 = cudaFreeAsync(dev, s);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  uint32_t n = 0;
  const tsdf_status st = tsdf_volume_block_count(vol, stream, &n);
  if (st != TSDF_OK) return st;
  out->occupied_slots = host.occupied;
  out->probe_sum = host.probe_sum;
  out->probe_max = host.probe_max;
  out->blocks = n;
  out->weight_sum = host.weight_sum;
  return TSDF_OK;
}

tsdf_status tsdf_volume_copy(tsdf_volume* dst, const tsdf_volume* src, void* stream) {
  if (!dst || !src || dst == src) return TSDF_ERR_INVALID_ARG;
  if (dst->slots != src->slots || dst->pool != src->pool || dst->voxel != src->voxel ||
      dst->trunc != src->trunc || dst->device != src->device ||
      dst->va.slot_index != src->va.slot_index)
    return TSDF_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != dst->device) return TSDF_ERR_INVALID_ARG;
  const cudaError_t e = cudaMemcpyAsync(dst->mem, src->mem, src->off.total,
                                        cudaMemcpyDeviceToDevice, as_stream(stream));
  if (e != cudaSuccess) return from_cuda(e);
  dst->poisoned = src->poisoned;
  dst->dirty = src->dirty;
  return TSDF_OK;
}

size_t tsdf_volume_checkpoint_bytes(const tsdf_volume* vol) {
  return vol ? sizeof(CheckpointHeader) + vol->off.total : 0;
}

tsdf_status tsdf_volume_save(const tsdf_volume* vol, void* host, size_t bytes, void* stream) {
  if (!vol || !host || bytes < tsdf_volume_checkpoint_bytes(vol)) return TSDF_ERR_INVALID_ARG;
  if (!on_volume_device(vol)) return TSDF_ERR_INVALID_ARG;
  CheckpointHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kCheckpointMagic, sizeof(h.magic));
  h.voxel = vol->voxel;
  h.trunc = vol->trunc;
  h.slots = vol->slots;
  h.pool = vol->pool;
  h.slot_index = vol->va.slot_index;
  h.poisoned = vol->poisoned ? 1u : 0u;
  h.dirty = vol->dirty ? 1u : 0u;
  h.bytes = vol->off.total;
  char* out = static_cast<char*>(host);
  std::memcpy(out, &h, sizeof(h));
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(out + sizeof(h), vol->mem, vol->off.total,
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

tsdf_status tsdf_volume_load(tsdf_volume* vol, const void* host, size_t bytes, void* stream) {
  if (!vol || !host || bytes < sizeof(CheckpointHeader)) return TSDF_ERR_INVALID_ARG;
  CheckpointHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (std::memcmp(h.magic, kCheckpointMagic, sizeof(h.magic)) != 0 || h.voxel != vol->voxel ||
      h.trunc != vol->trunc || h.slots != vol->slots || h.pool != vol->pool ||
      h.slot_index != vol->va.slot_index || h.bytes != vol->off.total ||
      bytes < sizeof(h) + vol->off.total)
    return TSDF_ERR_INVALID_ARG;
  if (!on_volume_device(vol)) return TSDF_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaMemcpyAsync(vol->mem, static_cast<const char*>(host) + sizeof(h),
                                  vol->off.total, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  vol->poisoned = h.poisoned != 0;
  vol->dirty = h.dirty != 0;
  return TSDF_OK;
}

uint64_t tsdf_block_key(int32_t bx, int32_t by, int32_t bz) {
  return tsdf::pack_key(bx, by, bz);
}

uint32_t tsdf_block_slot(int32_t bx, int32_t by, int32_t bz, uint32_t table_slots) {
  return tsdf::hash_block(bx, by, bz) & (table_slots - 1u);
}

const char* tsdf_status_string(tsdf_status s) {
  switch (s) {
    case TSDF_OK: return "TSDF_OK";
    case TSDF_ERR_INVALID_ARG: return "TSDF_ERR_INVALID_ARG";
    case TSDF_ERR_OUT_OF_MEMORY: return "TSDF_ERR_OUT_OF_MEMORY";
    case TSDF_ERR_POOL_FULL: return "TSDF_ERR_POOL_FULL";
    case TSDF_ERR_TABLE_FULL: return "TSDF_ERR_TABLE_FULL";
    case TSDF_ERR_PUBLISH_TIMEOUT: return "TSDF_ERR_PUBLISH_TIMEOUT";
    case TSDF_ERR_BOUNDS: return "TSDF_ERR_BOUNDS";
    case TSDF_ERR_POISONED: return "TSDF_ERR_POISONED";
    case TSDF_ERR_CUDA: return "TSDF_ERR_CUDA";
  }
  return "TSDF_ERR_UNKNOWN";
}

const char* tsdf_version(void) { return "libtsdf 0.1 (sm_103a)"; }

uint64_t tsdf_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

tsdf_status tsdf_set_l2_fetch_bytes(int bytes, int* previous) {
  if (bytes != 0 && bytes != 32 && bytes != 64 && bytes != 128) return TSDF_ERR_INVALID_ARG;
  size_t cur = 0;
  if (cudaDeviceGetLimit(&cur, cudaLimitMaxL2FetchGranularity) != cudaSuccess) {
    cudaGetLastError();
    return TSDF_ERR_CUDA;
  }
  if (cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, static_cast<size_t>(bytes)) !=
      cudaSuccess) {
    cudaGetLastError();
    return TSDF_ERR_CUDA;
  }
  if (previous) *previous = static_cast<int>(cur);
  return TSDF_OK;
}

}  // extern "C"
