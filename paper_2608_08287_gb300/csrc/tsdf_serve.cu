// Native serving core: continuous batching of frames from many sessions.
//
// The caller submits frames (host buffers, pinned for asynchronous copies)
// tagged with their arrival time; tsdf_server_poll drives the loop:
//   1. every launch whose completion event has fired is retired: its frames
//      get their completion time, their staging slots are freed;
//   2. (mode 0) the head frame of every session is copied into device staging
//      as soon as a staging slot is free, on a copy stream of its own, so
//      that frames queued behind a running launch are on the device when
//      their turn comes;
//   3. while fewer than max_inflight launches are in flight, the frames at the
//      head of every session that has none in flight (oldest arrival first,
//      at most max_batch) are launched -- as one batched fusion (mode 0; a
//      batch of one frame takes the single-frame path, and the launch waits
//      for the frames' copies) on a stream of its own, so that it runs beside
//      the launches already in flight, or one frame per launch with its copy
//      just before it, all on the caller's stream (mode 1, the baseline).
// Each session's frames therefore run in arrival order (at most one frame of
// a session in flight, and the next launched only after it retired), frames
// that arrive while others run join the next launch, and nothing is allocated
// after creation.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "tsdf.h"
#include "tsdf_internal.h"

namespace {

struct Pending {
  tsdf_volume* vol;
  const float* depth;
  const uint8_t* rgb;
  int w, h;
  tsdf_intrinsics intr;
  tsdf_pose pose;
  double arrival;
  uint64_t tag;
  int reset;  // empty the volume before fusing this frame
  int slot = -1;  // staging slot once its copy is enqueued (mode 0), else -1
};

struct InFlight {
  cudaEvent_t ev;
  std::vector<Pending> frames;
  std::vector<int> slots;
  int lane = -1;  // mode 0: the stream it runs on
};

}  // namespace

struct tsdf_server {
  int mode = 0;
  int max_batch = 0, max_inflight = 0;
  size_t slot_bytes = 0;
  int max_pixels = 0;
  char* staging = nullptr;
  std::vector<int> free_slots;
  // mode 0: one batch context per launch stream, so launches in flight never
  // share a batch's session tables or its streams
  std::vector<tsdf_batch*> batches;
  cudaStream_t stream = nullptr;
  cudaStream_t copy_stream = nullptr;      // mode 0: the eager copies
  std::vector<cudaEvent_t> slot_copied;    // mode 0: per staging slot, its copy done
  std::vector<cudaStream_t> lanes;         // mode 0: one stream per launch in flight
  std::vector<int> free_lanes;
  cudaEvent_t caller_ev = nullptr;         // mode 0: the caller's stream, before a launch
  std::unordered_map<tsdf_volume*, std::deque<Pending>> queues;
  std::unordered_map<tsdf_volume*, int> busy;
  std::deque<InFlight> inflight;
  std::vector<cudaEvent_t> events;  // free events
  std::deque<tsdf_completion> done;
  std::chrono::steady_clock::time_point t0;
  int pending = 0;
  tsdf_status sticky = TSDF_OK;
};

namespace {

double now_s(const tsdf_server* s) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// A failed copy, event or stream call makes the server's status CUDA (the
// first error is kept); the frames already accepted still complete.
void note_cuda(tsdf_server* s, cudaError_t e) {
  if (e == cudaSuccess) return;
  cudaGetLastError();
  if (s->sticky == TSDF_OK) s->sticky = TSDF_ERR_CUDA;
}

// Copy a frame into staging slot `slot` on stream cs.
void copy_in(tsdf_server* s, const Pending& p, int slot, cudaStream_t cs) {
  char* dst = s->staging + static_cast<size_t>(slot) * s->slot_bytes;
  const size_t npx = static_cast<size_t>(p.w) * p.h;
  const size_t dbytes = tsdf::align_up(npx * sizeof(float));
  note_cuda(s, cudaMemcpyAsync(dst, p.depth, npx * sizeof(float), cudaMemcpyHostToDevice, cs));
  if (p.rgb)
    note_cuda(s, cudaMemcpyAsync(dst + dbytes, p.rgb, npx * 3, cudaMemcpyHostToDevice, cs));
}

// Mode 0: give every session's head frame a staging slot and enqueue its copy
// on the copy stream (oldest arrival first, while slots last).
void copy_heads(tsdf_server* s) {
  std::vector<std::pair<double, tsdf_volume*>> heads;
  for (auto& kv : s->queues)
    if (!kv.second.empty() && kv.second.front().slot < 0)
      heads.emplace_back(kv.second.front().arrival, kv.first);
  std::sort(heads.begin(), heads.end());
  for (const auto& h : heads) {
    if (s->free_slots.empty()) return;
    Pending& p = s->queues[h.second].front();
    p.slot = s->free_slots.back();
    s->free_slots.pop_back();
    copy_in(s, p, p.slot, s->copy_stream);
    note_cuda(s, cudaEventRecord(s->slot_copied[p.slot], s->copy_stream));
  }
}

// Launch one batch (or one frame) from the queue heads. Returns false if
// nothing was ready.
bool launch_some(tsdf_server* s) {
  // eligible sessions: a queued frame, nothing in flight; oldest head first
  std::vector<std::pair<double, tsdf_volume*>> ready;
  for (auto& kv : s->queues)
    if (!kv.second.empty() && s->busy[kv.first] == 0)
      ready.emplace_back(kv.second.front().arrival, kv.first);
  if (ready.empty() || s->events.empty()) return false;
  std::sort(ready.begin(), ready.end());
  if (s->mode == 0) {
    // only heads whose copy is enqueued (every head has one while slots last)
    ready.erase(std::remove_if(ready.begin(), ready.end(),
                               [s](const std::pair<double, tsdf_volume*>& r) {
                                 return s->queues[r.second].front().slot < 0;
                               }),
                ready.end());
    if (ready.empty()) return false;
    if (s->free_lanes.empty()) return false;
  } else if (s->free_slots.empty()) {
    return false;
  }
  int take = s->mode == 1 ? 1 : s->max_batch;
  if (take > static_cast<int>(ready.size())) take = static_cast<int>(ready.size());
  if (s->mode == 1 && take > static_cast<int>(s->free_slots.size()))
    take = static_cast<int>(s->free_slots.size());
  InFlight f;
  cudaStream_t ls = s->stream;
  if (s->mode == 0) {
    // a stream of its own, ordered after the caller's stream
    f.lane = s->free_lanes.back();
    s->free_lanes.pop_back();
    ls = s->lanes[f.lane];
    note_cuda(s, cudaEventRecord(s->caller_ev, s->stream));
    note_cuda(s, cudaStreamWaitEvent(ls, s->caller_ev, 0));
  }
  std::vector<tsdf_frame> frames;
  frames.reserve(take);
  for (int i = 0; i < take; ++i) {
    tsdf_volume* v = ready[i].second;
    Pending p = s->queues[v].front();
    s->queues[v].pop_front();
    int slot = p.slot;
    if (slot < 0) {  // mode 1: the copy goes on the launch stream, just before
      slot = s->free_slots.back();
      s->free_slots.pop_back();
    }
    if (p.reset) {
      const tsdf_status rs = tsdf_volume_reset(v, ls);
      if (rs != TSDF_OK && s->sticky == TSDF_OK) s->sticky = rs;
    }
    char* dst = s->staging + static_cast<size_t>(slot) * s->slot_bytes;
    const size_t npx = static_cast<size_t>(p.w) * p.h;
    const size_t dbytes = tsdf::align_up(npx * sizeof(float));
    if (p.slot < 0)
      copy_in(s, p, slot, ls);
    else
      note_cuda(s, cudaStreamWaitEvent(ls, s->slot_copied[slot], 0));
    tsdf_frame fr;
    fr.volume = v;
    fr.depth = reinterpret_cast<const float*>(dst);
    fr.rgb = p.rgb ? reinterpret_cast<const uint8_t*>(dst + dbytes) : nullptr;
    fr.width = p.w;
    fr.height = p.h;
    fr.intr = p.intr;
    fr.pose = p.pose;
    frames.push_back(fr);
    f.frames.push_back(p);
    f.slots.push_back(slot);
    s->busy[v] = 1;
  }
  tsdf_status st;
  if (frames.size() == 1) {
    const tsdf_frame& fr = frames[0];
    st = tsdf_fuse_frame_async(fr.volume, fr.depth, fr.width, fr.height, &fr.intr, &fr.pose,
                               fr.rgb, ls);
  } else {
    st = tsdf_fuse_batch_async(s->batches[f.lane], frames.data(), static_cast<int>(frames.size()),
                               ls);
  }
  if (st != TSDF_OK && s->sticky == TSDF_OK) s->sticky = st;
  f.ev = s->events.back();
  s->events.pop_back();
  note_cuda(s, cudaEventRecord(f.ev, ls));
  s->inflight.push_back(std::move(f));
  return true;
}

void retire(tsdf_server* s) {
  while (!s->inflight.empty()) {
    InFlight& f = s->inflight.front();
    const cudaError_t q = cudaEventQuery(f.ev);
    if (q == cudaErrorNotReady) break;
    note_cuda(s, q);  // any other error: retired with the server's error status
    const double t = now_s(s);
    for (size_t i = 0; i < f.frames.size(); ++i) {
      const Pending& p = f.frames[i];
      s->done.push_back({p.tag, p.arrival, t, s->sticky});
      s->busy[p.vol] = 0;
      s->free_slots.push_back(f.slots[i]);
      --s->pending;
    }
    if (f.lane >= 0) s->free_lanes.push_back(f.lane);
    s->events.push_back(f.ev);
    s->inflight.pop_front();
  }
}

}  // namespace

extern "C" {

tsdf_status tsdf_server_create(int mode, int max_batch, int max_inflight, int max_frame_pixels,
                               int staging_frames, int use_graph, void* stream,
                               tsdf_server** out) {
  if (!out) return TSDF_ERR_INVALID_ARG;
  *out = nullptr;
  if (mode < 0 || mode > 1 || max_batch < 1 || max_inflight < 1 || max_inflight > 64 ||
      max_frame_pixels < 1 || staging_frames < max_batch)
    return TSDF_ERR_INVALID_ARG;
  tsdf_server* s = new (std::nothrow) tsdf_server();
  if (!s) return TSDF_ERR_OUT_OF_MEMORY;
  s->mode = mode;
  s->max_batch = mode == 1 ? 1 : max_batch;
  s->max_inflight = max_inflight;
  s->max_pixels = max_frame_pixels;
  s->slot_bytes = tsdf::align_up(tsdf::align_up(static_cast<size_t>(max_frame_pixels) * 4) +
                                 static_cast<size_t>(max_frame_pixels) * 3);
  s->stream = tsdf::as_stream(stream);
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaMalloc(&s->staging, s->slot_bytes * staging_frames);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return TSDF_ERR_OUT_OF_MEMORY;
  }
  for (int i = staging_frames - 1; i >= 0; --i) s->free_slots.push_back(i);
  for (int i = 0; i < max_inflight; ++i) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      tsdf_server_destroy(s);
      return TSDF_ERR_CUDA;
    }
    s->events.push_back(ev);
  }
  if (mode == 0) {
    if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      s->copy_stream = nullptr;
      tsdf_server_destroy(s);
      return TSDF_ERR_CUDA;
    }
    s->slot_copied.assign(staging_frames, nullptr);
    for (int i = 0; i < staging_frames; ++i) {
      if (cudaEventCreateWithFlags(&s->slot_copied[i], cudaEventDisableTiming) != cudaSuccess) {
        s->slot_copied[i] = nullptr;
        tsdf_server_destroy(s);
        return TSDF_ERR_CUDA;
      }
    }
    if (cudaEventCreateWithFlags(&s->caller_ev, cudaEventDisableTiming) != cudaSuccess) {
      s->caller_ev = nullptr;
      tsdf_server_destroy(s);
      return TSDF_ERR_CUDA;
    }
    for (int i = 0; i < max_inflight; ++i) {
      cudaStream_t ls = nullptr;
      if (cudaStreamCreateWithFlags(&ls, cudaStreamNonBlocking) != cudaSuccess) {
        tsdf_server_destroy(s);
        return TSDF_ERR_CUDA;
      }
      s->lanes.push_back(ls);
      s->free_lanes.push_back(max_inflight - 1 - i);
    }
  }
  tsdf_status st = TSDF_OK;
  if (mode == 0) {
    for (int i = 0; i < max_inflight && st == TSDF_OK; ++i) {
      tsdf_batch* bt = nullptr;
      st = tsdf_batch_create(max_batch, &bt);
      if (st == TSDF_OK) s->batches.push_back(bt);
      if (st == TSDF_OK && use_graph) st = tsdf_batch_set_option(bt, TSDF_OPT_USE_GRAPH, 1);
    }
  }
  if (st != TSDF_OK) {
    tsdf_server_destroy(s);
    return st;
  }
  *out = s;
  return TSDF_OK;
}

void tsdf_server_destroy(tsdf_server* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  for (cudaStream_t ls : s->lanes) {
    cudaStreamSynchronize(ls);
    cudaStreamDestroy(ls);
  }
  if (s->caller_ev) cudaEventDestroy(s->caller_ev);
  for (auto& f : s->inflight) s->events.push_back(f.ev);
  for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
  if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
  for (cudaEvent_t ev : s->slot_copied)
    if (ev) cudaEventDestroy(ev);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  for (tsdf_batch* bt : s->batches) tsdf_batch_destroy(bt);
  if (s->staging) cudaFree(s->staging);
  delete s;
}

double tsdf_server_clock(const tsdf_server* s) { return s ? now_s(s) : 0.0; }

tsdf_status tsdf_server_submit(tsdf_server* s, const tsdf_request* r) {
  if (!s || !r || !r->volume || !r->depth || r->width < 1 || r->height < 1)
    return TSDF_ERR_INVALID_ARG;
  if (static_cast<long long>(r->width) * r->height > s->max_pixels) return TSDF_ERR_INVALID_ARG;
  s->queues[r->volume].push_back({r->volume, r->depth, r->rgb, r->width, r->height, r->intr,
                                  r->pose, r->arrival_s, r->tag, r->reset_volume});
  ++s->pending;
  return TSDF_OK;
}

int tsdf_server_poll(tsdf_server* s, tsdf_completion* out, int capacity) {
  if (!s) return -1;
  retire(s);
  if (s->mode == 0) copy_heads(s);
  while (static_cast<int>(s->inflight.size()) < s->max_inflight && launch_some(s)) {
    if (s->mode == 0) copy_heads(s);
  }
  int n = 0;
  while (n < capacity && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  return n;
}

int tsdf_server_pending(const tsdf_server* s) { return s ? s->pending : -1; }

tsdf_status tsdf_server_replay(tsdf_server* s, const tsdf_request* reqs, int n,
                               tsdf_completion* out) {
  if (!s || (n > 0 && (!reqs || !out))) return TSDF_ERR_INVALID_ARG;
  for (int i = 1; i < n; ++i)
    if (reqs[i].arrival_s < reqs[i - 1].arrival_s) return TSDF_ERR_INVALID_ARG;
  // completions are written in request order: index requests by tag position
  std::unordered_map<uint64_t, int> where;
  where.reserve(static_cast<size_t>(n) * 2);
  for (int i = 0; i < n; ++i) where[reqs[i].tag] = i;
  if (static_cast<int>(where.size()) != n) return TSDF_ERR_INVALID_ARG;  // tags must be unique
  const double start = now_s(s);
  int next = 0, got = 0;
  std::vector<tsdf_completion> buf(256);
  while (got < n) {
    const double t = now_s(s) - start;
    while (next < n && reqs[next].arrival_s <= t) {
      tsdf_request r = reqs[next++];
      r.arrival_s += start;
      const tsdf_status st = tsdf_server_submit(s, &r);
      if (st != TSDF_OK) return st;
    }
    const int k = tsdf_server_poll(s, buf.data(), static_cast<int>(buf.size()));
    for (int i = 0; i < k; ++i) {
      tsdf_completion c = buf[i];
      c.arrival_s -= start;
      c.done_s -= start;
      out[where[c.tag]] = c;
    }
    got += k;
  }
  return s->sticky;
}

}  // extern "C"
