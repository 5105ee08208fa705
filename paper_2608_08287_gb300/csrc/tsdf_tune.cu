// Autotuning: time every fusion strategy (and, for batches, the launch shape;
// for a volume, the threads per point of the fused tile kernel) on the
// caller's own frames and keep the fastest.
//
// A single volume is tuned on a scratch copy of itself: before every timed
// repetition the scratch is restored from the volume (tsdf_volume_copy) and
// L2 is evicted by writing a buffer twice its size, so every candidate fuses
// the same frame into the same state from a cold cache. The volume itself is
// not modified; only its strategy options are set to the winner.
//
// A batch is tuned on its frames' volumes, which must be empty: before every
// repetition they are reset (so every repetition fuses into empty volumes),
// and they are left empty. The search is staged: the default (one launch per
// frame over 8 streams), the strategies with the persistent grid at full
// occupancy and graphs on, then the CTAs-per-SM cap of the best of those,
// then graphs off, then the best persistent strategy launched per frame over
// 4, 8 and 16 streams.
//
// Each configuration's time is the median of `reps` repetitions after one
// untimed warm-up, with CUDA events on the caller's stream.
#include <algorithm>
#include <vector>

#include <cuda_runtime.h>

#include "tsdf.h"
#include "tsdf_internal.h"

namespace {

struct Config {
  int allocate_mode, integrate_mode, fuse_mode, probe_load, ctas_per_sm, use_graph;
  int threads_per_point = 1;
  int batch_streams = 0;  // batches: TSDF_OPT_BATCH_STREAMS
};

float median(std::vector<float> v) {
  std::sort(v.begin(), v.end());
  const size_t n = v.size();
  return n % 2 ? v[n / 2] : 0.5f * (v[n / 2 - 1] + v[n / 2]);
}

// Device scratch for evicting L2: twice its size.
struct Evict {
  void* buf = nullptr;
  size_t bytes = 0;
  cudaError_t init(int device, cudaStream_t s) {
    int l2 = 0;
    cudaError_t e = cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
    if (e != cudaSuccess) return e;
    bytes = 2 * static_cast<size_t>(l2 > 0 ? l2 : (64 << 20));
    return cudaMallocAsync(&buf, bytes, s);
  }
  cudaError_t run(cudaStream_t s, int i) const { return cudaMemsetAsync(buf, i & 0xFF, bytes, s); }
  void release(cudaStream_t s) {
    if (buf) cudaFreeAsync(buf, s);
    buf = nullptr;
  }
};

struct Events {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t init() {
    cudaError_t e = cudaEventCreate(&a);
    return e == cudaSuccess ? cudaEventCreate(&b) : e;
  }
  ~Events() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

tsdf_status apply_volume(tsdf_volume* v, const Config& c) {
  // no split walk first: the probe load may only change then
  tsdf_status st = tsdf_volume_set_option(v, TSDF_OPT_THREADS_PER_POINT, 1);
  if (st == TSDF_OK) st = tsdf_volume_set_option(v, TSDF_OPT_ALLOCATE_MODE, c.allocate_mode);
  if (st == TSDF_OK) st = tsdf_volume_set_option(v, TSDF_OPT_INTEGRATE_MODE, c.integrate_mode);
  if (st == TSDF_OK) st = tsdf_volume_set_option(v, TSDF_OPT_FUSE_MODE, c.fuse_mode);
  if (st == TSDF_OK) st = tsdf_volume_set_option(v, TSDF_OPT_PROBE_LOAD, c.probe_load);
  if (st == TSDF_OK)
    st = tsdf_volume_set_option(v, TSDF_OPT_THREADS_PER_POINT, c.threads_per_point);
  return st;
}

tsdf_status apply_batch(tsdf_batch* b, const Config& c) {
  tsdf_status st = tsdf_batch_set_option(b, TSDF_OPT_ALLOCATE_MODE, c.allocate_mode);
  if (st == TSDF_OK) st = tsdf_batch_set_option(b, TSDF_OPT_INTEGRATE_MODE, c.integrate_mode);
  if (st == TSDF_OK) st = tsdf_batch_set_option(b, TSDF_OPT_FUSE_MODE, c.fuse_mode);
  if (st == TSDF_OK) st = tsdf_batch_set_option(b, TSDF_OPT_PROBE_LOAD, c.probe_load);
  if (st == TSDF_OK) st = tsdf_batch_set_option(b, TSDF_OPT_CTAS_PER_SM, c.ctas_per_sm);
  if (st == TSDF_OK) st = tsdf_batch_set_option(b, TSDF_OPT_USE_GRAPH, c.use_graph);
  if (st == TSDF_OK) st = tsdf_batch_set_option(b, TSDF_OPT_BATCH_STREAMS, c.batch_streams);
  return st;
}

void fill(tsdf_tuning* out, const Config& c, float best, float dflt, int n) {
  out->allocate_mode = c.allocate_mode;
  out->integrate_mode = c.integrate_mode;
  out->fuse_mode = c.fuse_mode;
  out->probe_load = c.probe_load;
  out->ctas_per_sm = c.ctas_per_sm;
  out->use_graph = c.use_graph;
  out->candidates = n;
  out->best_ms = best;
  out->default_ms = dflt;
  out->threads_per_point = c.threads_per_point;
  out->batch_streams = c.batch_streams;
}

}  // namespace

extern "C" {

tsdf_status tsdf_autotune_frame(tsdf_volume* vol, const float* depth_dev, int width, int height,
                                const tsdf_intrinsics* intr, const tsdf_pose* pose,
                                const uint8_t* rgb_dev, int reps, void* stream,
                                tsdf_tuning* out) {
  if (!vol || !out || reps < 1 || reps > 1000) return TSDF_ERR_INVALID_ARG;
  tsdf::FrameArgs f;
  tsdf_status st = tsdf::make_frame(vol, depth_dev, width, height, intr, pose, rgb_dev, &f);
  if (st != TSDF_OK) return st;
  if (vol->poisoned) return TSDF_ERR_POISONED;
  cudaStream_t s = tsdf::as_stream(stream);

  tsdf_volume* scratch = nullptr;
  st = tsdf_volume_create(vol->voxel, vol->trunc, vol->slots, vol->pool, &scratch);
  if (st != TSDF_OK) return st;
  if (vol->va.slot_index) st = tsdf_volume_set_option(scratch, TSDF_OPT_SLOT_INDEX, 1);
  scratch->va.probe_limit = vol->va.probe_limit;
  Evict evict;
  Events ev;
  cudaError_t e = evict.init(vol->device, s);
  if (e == cudaSuccess) e = ev.init();
  if (st == TSDF_OK && e != cudaSuccess) st = tsdf::from_cuda(e);

  // the default (fused tile kernel, threads per point chosen per frame)
  // first, then every stage A x stage B pair, the fused warp kernel, the
  // other probe loads of the default, and the default with 1, 2, 4 and 8
  // threads per point set explicitly
  const Config dflt{1, 0, 2, 0, 0, 0, 0};
  std::vector<Config> cands{dflt};
  for (int a = 0; a <= 2; ++a)
    for (int i = 0; i <= 2; ++i) cands.push_back({a, i, 0, 0, 0, 0, 1});
  cands.push_back({1, 0, 1, 0, 0, 0, 1});
  cands.push_back({1, 0, 2, 1, 0, 0, 1});
  cands.push_back({1, 0, 2, 2, 0, 0, 1});
  cands.push_back({1, 0, 2, 0, 0, 0, 1});
  if (vol->half_band == 2 || vol->half_band == 4 || vol->half_band == 8)
    for (int t = 2; t <= 8; t *= 2) cands.push_back({1, 0, 2, 0, 0, 0, t});

  std::vector<float> times;
  for (size_t c = 0; c < cands.size() && st == TSDF_OK; ++c) {
    st = apply_volume(scratch, cands[c]);
    std::vector<float> t;
    for (int r = 0; r <= reps && st == TSDF_OK; ++r) {
      st = tsdf_volume_copy(scratch, vol, stream);
      if (st != TSDF_OK) break;
      e = evict.run(s, r);
      if (e == cudaSuccess) e = cudaEventRecord(ev.a, s);
      if (e != cudaSuccess) {
        st = tsdf::from_cuda(e);
        break;
      }
      st = tsdf_fuse_frame_async(scratch, depth_dev, width, height, intr, pose, rgb_dev, stream);
      if (st != TSDF_OK) break;
      e = cudaEventRecord(ev.b, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(ev.b);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev.a, ev.b);
      if (e != cudaSuccess) {
        st = tsdf::from_cuda(e);
        break;
      }
      if (r > 0) t.push_back(ms);
    }
    // a frame that overflows the volume, or times out, has no valid timing
    if (st == TSDF_OK) st = tsdf_volume_status(scratch, stream);
    if (st == TSDF_OK) times.push_back(median(t));
  }
  evict.release(s);
  if (st == TSDF_OK) st = tsdf::from_cuda(cudaStreamSynchronize(s));
  tsdf_volume_destroy(scratch);
  if (st != TSDF_OK) return st;
  const size_t best = std::min_element(times.begin(), times.end()) - times.begin();
  fill(out, cands[best], times[best], times[0], static_cast<int>(cands.size()));
  return apply_volume(vol, cands[best]);
}

tsdf_status tsdf_batch_autotune(tsdf_batch* batch, const tsdf_frame* frames, int n, int reps,
                                void* stream, tsdf_tuning* out) {
  if (!batch || !frames || !out || n < 1 || reps < 1 || reps > 1000) return TSDF_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    const tsdf_volume* v = frames[i].volume;
    if (!v || v->dirty || v->poisoned) return TSDF_ERR_INVALID_ARG;  // must be empty
  }
  cudaStream_t s = tsdf::as_stream(stream);
  Evict evict;
  Events ev;
  cudaError_t e = evict.init(frames[0].volume->device, s);
  if (e == cudaSuccess) e = ev.init();
  tsdf_status st = tsdf::from_cuda(e);

  auto run = [&](const Config& c, float* result) -> tsdf_status {
    tsdf_status rs = apply_batch(batch, c);
    std::vector<float> t;
    for (int r = 0; r <= reps && rs == TSDF_OK; ++r) {
      for (int i = 0; i < n && rs == TSDF_OK; ++i) rs = tsdf_volume_reset(frames[i].volume, stream);
      if (rs != TSDF_OK) break;
      cudaError_t re = evict.run(s, r);
      if (re == cudaSuccess) re = cudaEventRecord(ev.a, s);
      if (re != cudaSuccess) return tsdf::from_cuda(re);
      rs = tsdf_fuse_batch_async(batch, frames, n, stream);
      if (rs != TSDF_OK) break;
      re = cudaEventRecord(ev.b, s);
      if (re == cudaSuccess) re = cudaEventSynchronize(ev.b);
      float ms = 0.0f;
      if (re == cudaSuccess) re = cudaEventElapsedTime(&ms, ev.a, ev.b);
      if (re != cudaSuccess) return tsdf::from_cuda(re);
      if (r > 0) t.push_back(ms);
    }
    if (rs == TSDF_OK) rs = tsdf_batch_status(batch, stream, nullptr, 0);
    if (rs == TSDF_OK) *result = median(t);
    return rs;
  };

  int tried = 0;
  // the batch's defaults: the fused tile kernel, one launch per frame over 8
  // streams
  const Config dflt{1, 0, 2, 0, 0, 1, 1, 8};
  Config best = dflt;
  float best_ms = 0.0f, dflt_ms = 0.0f;
  if (st == TSDF_OK) st = run(dflt, &dflt_ms);
  ++tried;
  best_ms = dflt_ms;
  // the best persistent-launch configuration (TSDF_OPT_BATCH_STREAMS 0)
  Config best_p{1, 0, 2, 0, 0, 1, 1, 0};
  float best_p_ms = -1.0f;
  auto consider = [&](const Config& c) {
    if (st != TSDF_OK) return;
    float ms = 0.0f;
    st = run(c, &ms);
    ++tried;
    if (st != TSDF_OK) return;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
    if (c.batch_streams == 0 && (best_p_ms < 0.0f || ms < best_p_ms)) {
      best_p_ms = ms;
      best_p = c;
    }
  };
  // stage 1: strategies in one persistent launch (the batched kernels take
  // stage A strategies 1 and 2)
  consider({1, 0, 2, 0, 0, 1, 1, 0});
  consider({1, 0, 0, 0, 0, 1, 1, 0});
  consider({1, 1, 0, 0, 0, 1, 1, 0});
  consider({2, 0, 0, 0, 0, 1, 1, 0});
  consider({2, 1, 0, 0, 0, 1, 1, 0});
  consider({1, 0, 1, 0, 0, 1, 1, 0});
  // stage 2: resident CTAs per SM of the persistent grid
  const Config strat = best_p;
  for (int f = 1; f <= 4; ++f) {
    Config c = strat;
    c.ctas_per_sm = f;
    consider(c);
  }
  // stage 3: direct launches instead of graph replays
  Config direct = best_p;
  direct.use_graph = 0;
  consider(direct);
  // stage 4: the best persistent strategy launched per frame over 4, 8 and 16
  // streams (8 with the default strategy was timed first)
  for (int k = 4; k <= 16; k *= 2) {
    Config c = best_p;
    c.ctas_per_sm = 0;
    c.use_graph = 1;
    c.batch_streams = k;
    if (k == 8 && c.allocate_mode == dflt.allocate_mode &&
        c.integrate_mode == dflt.integrate_mode && c.fuse_mode == dflt.fuse_mode &&
        c.probe_load == dflt.probe_load)
      continue;
    consider(c);
  }
  for (int i = 0; i < n && st == TSDF_OK; ++i) st = tsdf_volume_reset(frames[i].volume, stream);
  evict.release(s);
  if (st == TSDF_OK) st = tsdf::from_cuda(cudaStreamSynchronize(s));
  if (st != TSDF_OK) return st;
  fill(out, best, best_ms, dflt_ms, tried);
  return apply_batch(batch, best);
}

}  // extern "C"
