// Batched fusion: many frames, each into its own volume, either as one launch
// per frame over several streams the batch owns (TSDF_OPT_BATCH_STREAMS > 0,
// the default), or in one persistent launch per stage (or one fused launch),
// optionally replayed from a CUDA graph.
//
// Per-frame launches: the frames are taken largest first and dealt
// round-robin over the batch's streams, so the big frames start together and
// the small ones fill the GPU around them; each stream waits for an event on
// the caller's stream before its first launch, and the caller's stream waits
// for each stream's last. Each frame runs the single-frame kernels with its
// arguments in the kernel's parameter space, with the threads per point the
// whole call's tile count gives (one when the batch fills the GPU).
//
// A batch owns two session tables (double buffering): a pinned host copy the
// caller's frames are written into, and a device copy the kernels read. Each
// call uses the other table, after waiting for the event recorded when that
// table's previous launch finished, so the host prepares batch i+1 while
// batch i runs. With graphs on, each table's copy-and-launch sequence is
// captured once per configuration and replayed; the kernels' grids are
// persistent, so one graph serves batches of any composition. Batches too small
// to fill that grid are launched directly with a grid of their own size.
#include <algorithm>
#include <cstring>
#include <new>

#include <cuda_runtime.h>

#include "tsdf.h"
#include "tsdf_device.cuh"
#include "tsdf_internal.h"
#include "tsdf_launch.h"

using tsdf::as_stream;
using tsdf::from_cuda;

namespace {
constexpr int kMaxLanes = 16;     // streams a batch can own
constexpr int kDefaultLanes = 8;  // TSDF_OPT_BATCH_STREAMS at creation
}  // namespace

struct tsdf_batch {
  int device = 0;
  int max_frames = 0;
  size_t table_bytes = 0;
  void* table_dev[2] = {nullptr, nullptr};
  void* table_host[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  int slot = 0;
  int last_slot = -1;
  int last_n = 0;
  tsdf_volume** last_vols = nullptr;
  unsigned* status_dev = nullptr;
  unsigned* status_host = nullptr;
  // configuration
  int probe_load = 0, allocate_mode = 1, integrate_mode = 0, fuse_mode = 2, factor = 0;
  int stages = 3;  // two-stage path: 1 = stage A, 2 = stage B, 3 = both
  int use_graph = 0;
  cudaStream_t capture = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  long long exec_key[2] = {-1, -1};
  // per-frame launches (TSDF_OPT_BATCH_STREAMS): lanes in use, lanes made,
  // the lanes and the event each records after its last launch, the fork
  // event
  int lanes = 0;
  int lanes_made = 0;
  cudaStream_t lane[kMaxLanes] = {};
  cudaEvent_t lane_done[kMaxLanes] = {};
  cudaEvent_t fork = nullptr;
  // the caller's index of each entry of the last call's table (the table
  // holds the frames largest first)
  int* order = nullptr;
};

namespace {

long long config_key(const tsdf_batch* b, bool all_m4) {
  return ((((((static_cast<long long>(b->probe_load) * 4 + b->allocate_mode) * 4 +
              b->integrate_mode) * 4 + b->fuse_mode) * 64) + b->factor) * 4 + b->stages) * 2 +
         (all_m4 ? 1 : 0);
}

void drop_graphs(tsdf_batch* b) {
  for (int i = 0; i < 2; ++i) {
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    b->exec[i] = nullptr;
    b->exec_key[i] = -1;
  }
}

cudaError_t enqueue(tsdf_batch* b, int slot, size_t bytes, int grid_limit, bool all_m4,
                    cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(b->table_dev[slot], b->table_host[slot], bytes,
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return tsdf::launch_batch(static_cast<const tsdf::BatchHeader*>(b->table_dev[slot]),
                            b->probe_load, b->allocate_mode, b->integrate_mode, b->fuse_mode,
                            b->factor, grid_limit, all_m4, b->stages, s);
}

// A batch smaller than this many tiles is launched directly with a grid of its
// own size: a replayed graph's persistent grid would mostly idle.
constexpr int kGraphMinTiles = 2048;

// Make lanes up to k (streams that do not synchronise with the legacy default
// stream, and their events).
cudaError_t make_lanes(tsdf_batch* b, int k) {
  if (!b->fork) {
    const cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      b->fork = nullptr;
      return e;
    }
  }
  while (b->lanes_made < k) {
    const int i = b->lanes_made;
    cudaError_t e = cudaStreamCreateWithFlags(&b->lane[i], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      b->lane[i] = nullptr;
      return e;
    }
    e = cudaEventCreateWithFlags(&b->lane_done[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaStreamDestroy(b->lane[i]);
      b->lane[i] = nullptr;
      b->lane_done[i] = nullptr;
      return e;
    }
    ++b->lanes_made;
  }
  return cudaSuccess;
}

// Launch one frame's fusion with the batch's strategy on stream s; its
// threads per point are chosen for all `batch_tiles` tiles of the call, which
// run together (a frame that would be split alone is not when the batch fills
// the GPU: there the split only adds work).
cudaError_t launch_one(const tsdf_batch* b, const tsdf::SessionArgs& a, long long batch_tiles,
                       int half_band, int sm_count, cudaStream_t s) {
  if (b->fuse_mode != 0) {
    const int tpp = tsdf::auto_threads_per_point(b->fuse_mode, b->probe_load, half_band,
                                                 sm_count, batch_tiles);
    return tsdf::launch_fused(a.f, a.vol, b->probe_load, b->fuse_mode, tpp, s);
  }
  cudaError_t e = cudaSuccess;
  if (b->stages & 1) e = tsdf::launch_allocate(a.f, a.vol, b->probe_load, b->allocate_mode, s);
  if (e == cudaSuccess && (b->stages & 2)) e = tsdf::launch_integrate(a.f, a.vol, b->integrate_mode, s);
  return e;
}

// Per-frame launches of the n frames whose arguments are in S (table order,
// largest frames first), over the batch's lanes, forked from and joined back
// into s.
cudaError_t enqueue_lanes(tsdf_batch* b, const tsdf::SessionArgs* S, int n, long long tiles,
                          cudaStream_t s) {
  const int lanes = std::min(b->lanes, n);
  cudaError_t e = cudaEventRecord(b->fork, s);
  for (int j = 0; j < lanes && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(b->lane[j], b->fork, 0);
  if (e != cudaSuccess) return e;
  for (int j = 0; j < n && e == cudaSuccess; ++j) {
    const tsdf_volume* v = b->last_vols[j];
    e = launch_one(b, S[j], tiles, v->half_band, v->sm_count, b->lane[j % lanes]);
  }
  // the join is enqueued even after a failed launch, so `s` stays ordered
  // after whatever the lanes did take
  for (int j = 0; j < lanes; ++j) {
    cudaError_t ej = cudaEventRecord(b->lane_done[j], b->lane[j]);
    if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, b->lane_done[j], 0);
    if (e == cudaSuccess) e = ej;
  }
  return e;
}

}  // namespace

extern "C" {

tsdf_status tsdf_batch_create(int max_frames, tsdf_batch** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (max_frames < 1 || max_frames > 65536) return TSDF_ERR_INVALID_ARG;
  tsdf_batch* b = new (std::nothrow) tsdf_batch();
  if (!b) return TSDF_ERR_OUT_OF_MEMORY;
  b->max_frames = max_frames;
  b->table_bytes =
      sizeof(tsdf::BatchHeader) + static_cast<size_t>(max_frames) * sizeof(tsdf::SessionArgs);
  cudaError_t e = cudaGetDevice(&b->device);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaMalloc(&b->table_dev[i], b->table_bytes);
    if (e == cudaSuccess) e = cudaMallocHost(&b->table_host[i], b->table_bytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->status_dev, sizeof(unsigned) * max_frames);
  if (e == cudaSuccess) e = cudaMallocHost(&b->status_host, sizeof(unsigned) * max_frames);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = make_lanes(b, kDefaultLanes);
  if (e == cudaSuccess) b->lanes = kDefaultLanes;
  b->last_vols = new (std::nothrow) tsdf_volume*[max_frames];
  b->order = new (std::nothrow) int[max_frames];
  if (e != cudaSuccess || !b->last_vols || !b->order) {
    cudaGetLastError();
    tsdf_batch_destroy(b);
    return e == cudaErrorMemoryAllocation || e == cudaSuccess ? TSDF_ERR_OUT_OF_MEMORY
                                                              : TSDF_ERR_CUDA;
  }
  *out = b;
  return TSDF_OK;
}

void tsdf_batch_destroy(tsdf_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  drop_graphs(b);
  for (int i = 0; i < 2; ++i) {
    if (b->table_dev[i]) cudaFree(b->table_dev[i]);
    if (b->table_host[i]) cudaFreeHost(b->table_host[i]);
    if (b->done[i]) cudaEventDestroy(b->done[i]);
  }
  if (b->status_dev) cudaFree(b->status_dev);
  if (b->status_host) cudaFreeHost(b->status_host);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (int i = 0; i < b->lanes_made; ++i) {
    cudaStreamDestroy(b->lane[i]);
    cudaEventDestroy(b->lane_done[i]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  delete[] b->last_vols;
  delete[] b->order;
  delete b;
}

tsdf_status tsdf_batch_set_option(tsdf_batch* b, tsdf_option opt, int64_t value) {
  if (!b) return TSDF_ERR_INVALID_ARG;
  switch (opt) {
    case TSDF_OPT_PROBE_LOAD:
      if (value < 0 || value > 2) return TSDF_ERR_INVALID_ARG;
      b->probe_load = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_ALLOCATE_MODE:
      if (value < 1 || value > 2) return TSDF_ERR_INVALID_ARG;
      b->allocate_mode = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_INTEGRATE_MODE:
      if (value < 0 || value > 1) return TSDF_ERR_INVALID_ARG;
      b->integrate_mode = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_FUSE_MODE:
      if (value < 0 || value > 2) return TSDF_ERR_INVALID_ARG;
      b->fuse_mode = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_CTAS_PER_SM:
      if (value < 0 || value > 32) return TSDF_ERR_INVALID_ARG;
      b->factor = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_USE_GRAPH:
      if (value < 0 || value > 1) return TSDF_ERR_INVALID_ARG;
      b->use_graph = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_BATCH_STAGES:
      if (value < 1 || value > 3) return TSDF_ERR_INVALID_ARG;
      b->stages = static_cast<int>(value);
      return TSDF_OK;
    case TSDF_OPT_BATCH_STREAMS: {
      if (value < 0 || value > kMaxLanes) return TSDF_ERR_INVALID_ARG;
      const cudaError_t e = make_lanes(b, static_cast<int>(value));
      if (e != cudaSuccess) {
        cudaGetLastError();
        return TSDF_ERR_CUDA;
      }
      b->lanes = static_cast<int>(value);
      return TSDF_OK;
    }
    default:
      return TSDF_ERR_INVALID_ARG;
  }
}

tsdf_status tsdf_fuse_batch_async(tsdf_batch* b, const tsdf_frame* frames, int n, void* stream) {
  if (!b || !frames || n < 1 || n > b->max_frames) return TSDF_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return TSDF_ERR_INVALID_ARG;
  // validate everything before touching the table
  for (int i = 0; i < n; ++i) {
    tsdf_volume* v = frames[i].volume;
    if (!v || v->device != b->device) return TSDF_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (frames[j].volume == v) return TSDF_ERR_INVALID_ARG;  // one frame per volume
    tsdf::FrameArgs f;
    const tsdf_status st = tsdf::make_frame(v, frames[i].depth, frames[i].width,
                                            frames[i].height, &frames[i].intr, &frames[i].pose,
                                            frames[i].rgb, &f);
    if (st != TSDF_OK) return st;
    if (v->poisoned) return TSDF_ERR_POISONED;
  }
  const int slot = b->slot;
  b->slot ^= 1;
  if (b->used[slot]) {
    const cudaError_t e = cudaEventSynchronize(b->done[slot]);
    if (e != cudaSuccess) return from_cuda(e);
  }
  char* host = static_cast<char*>(b->table_host[slot]);
  tsdf::BatchHeader* hdr = reinterpret_cast<tsdf::BatchHeader*>(host);
  tsdf::SessionArgs* S = reinterpret_cast<tsdf::SessionArgs*>(hdr + 1);
  // the table holds the frames largest first: the per-frame launches are
  // issued in that order and the persistent kernels walk the tiles in it, so
  // the big frames start first and the small ones fill in behind them.
  // order[j] is the caller's index of table entry j.
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::stable_sort(b->order, b->order + n, [frames](int x, int y) {
    return static_cast<long long>(frames[x].width) * frames[x].height >
           static_cast<long long>(frames[y].width) * frames[y].height;
  });
  int tiles = 0;
  bool all_m4 = true;
  for (int j = 0; j < n; ++j) {
    const tsdf_frame& fr = frames[b->order[j]];
    tsdf_volume* v = fr.volume;
    tsdf::make_frame(v, fr.depth, fr.width, fr.height, &fr.intr, &fr.pose, fr.rgb, &S[j].f);
    S[j].vol = v->va;
    all_m4 = all_m4 && S[j].f.M == 4;
    v->dirty = true;
    S[j].tiles_x = (fr.width + 15) / 16;
    S[j].tile_begin = tiles;
    tiles += S[j].tiles_x * ((fr.height + 15) / 16);
    b->last_vols[j] = v;
  }
  hdr->n = n;
  hdr->total_tiles = tiles;
  b->last_slot = slot;
  b->last_n = n;
  cudaStream_t s = as_stream(stream);
  cudaError_t e = cudaSuccess;
  if (b->lanes > 0) {
    e = enqueue_lanes(b, S, n, tiles, s);
    // the session table still goes to the device: tsdf_batch_status reads
    // each frame's volume header through it
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->table_dev[slot], b->table_host[slot],
                          sizeof(tsdf::BatchHeader) + static_cast<size_t>(n) *
                                                          sizeof(tsdf::SessionArgs),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(b->done[slot], s);
    b->used[slot] = true;
    return from_cuda(e);
  }
  if (b->use_graph && tiles >= kGraphMinTiles) {
    const long long key = config_key(b, all_m4);
    if (b->exec_key[slot] != key) {
      if (b->exec[slot]) cudaGraphExecDestroy(b->exec[slot]);
      b->exec[slot] = nullptr;
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        // the whole table capacity is copied, so the graph serves any n
        const cudaError_t e1 = enqueue(b, slot, b->table_bytes, 0, all_m4, b->capture);
        e = cudaStreamEndCapture(b->capture, &g);
        if (e == cudaSuccess) e = e1;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec[slot], g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        cudaGetLastError();
        b->exec[slot] = nullptr;
        return TSDF_ERR_CUDA;
      }
      b->exec_key[slot] = key;
    }
    e = cudaGraphLaunch(b->exec[slot], s);
  } else {
    const size_t bytes =
        sizeof(tsdf::BatchHeader) + static_cast<size_t>(n) * sizeof(tsdf::SessionArgs);
    e = enqueue(b, slot, bytes, tiles, all_m4, s);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->done[slot], s);
  if (e != cudaSuccess) return from_cuda(e);
  tsdf::note_launch();
  if (b->fuse_mode == 0 && b->stages == 3) tsdf::note_launch();
  b->used[slot] = true;
  return TSDF_OK;
}

tsdf_status tsdf_batch_status(tsdf_batch* b, void* stream, tsdf_status* per_frame, int n) {
  if (!b || b->last_slot < 0) return TSDF_ERR_INVALID_ARG;
  if (per_frame && n < b->last_n) return TSDF_ERR_INVALID_ARG;
  cudaStream_t s = as_stream(stream);
  cudaError_t e = tsdf::launch_batch_status(
      static_cast<const tsdf::BatchHeader*>(b->table_dev[b->last_slot]), b->status_dev, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->status_host, b->status_dev, sizeof(unsigned) * b->last_n,
                        cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  // table entry j is the caller's frame order[j]; the first error in the
  // caller's order is returned
  tsdf_status worst = TSDF_OK;
  int worst_at = b->last_n;
  for (int j = 0; j < b->last_n; ++j) {
    const tsdf_status st = tsdf::decode_err(b->status_host[j]);
    const int i = b->order[j];
    if (st != TSDF_OK) {
      b->last_vols[j]->poisoned = true;
      if (i < worst_at) {
        worst = st;
        worst_at = i;
      }
    }
    if (per_frame) per_frame[i] = st;
  }
  return worst;
}

}  // extern "C"
