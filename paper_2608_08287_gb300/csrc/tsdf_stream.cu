// tsdf_fuse_frames_host: a sequence of frames given in host memory, fused in
// order with each frame's host-to-device copy overlapping the fusion of the
// frame before it.
//
// tsdf_fuse_frame_host serialises three things per frame: the copy of the
// frame in, the fusion kernel, and the read-back of the status word, with the
// host waiting in between. A camera stream does not need that: frame i+1 can
// be copied while frame i fuses, and the status words can be read after the
// last frame. This file keeps, per volume that owns the staging, two staging
// slots (frame i uses slot i mod 2), a copy stream, two events marking each
// slot as filled and two marking it as free again (the kernel that read it
// has finished), and a pinned array of per-frame error words. All are made on
// first use and grown when a call needs more; nothing is allocated while a
// call's work is in flight.
#include <cstring>

#include <cuda_runtime.h>

#include "tsdf.h"
#include "tsdf_internal.h"

using tsdf::align_up;
using tsdf::as_stream;
using tsdf::decode_err;
using tsdf::from_cuda;

namespace {

size_t frame_stage_bytes(const tsdf_frame& fr) {
  const size_t npx = static_cast<size_t>(fr.width) * static_cast<size_t>(fr.height);
  return align_up(npx * sizeof(float)) + (fr.rgb ? align_up(npx * 3) : 0);
}

// Streams, events, staging and pinned words of the owning volume, large
// enough for slots of slot_bytes and n frames. Called before anything of the
// call is enqueued; the previous call on this volume has synchronised.
tsdf_status ensure_resources(tsdf_volume* v, size_t slot_bytes, int n) {
  if (!v->copy_stream) {
    if (cudaStreamCreateWithFlags(&v->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
      v->copy_stream = nullptr;
      cudaGetLastError();
      return TSDF_ERR_CUDA;
    }
  }
  for (int b = 0; b < 2; ++b) {
    if (!v->ev_copied[b] &&
        cudaEventCreateWithFlags(&v->ev_copied[b], cudaEventDisableTiming) != cudaSuccess) {
      v->ev_copied[b] = nullptr;
      cudaGetLastError();
      return TSDF_ERR_CUDA;
    }
    if (!v->ev_free[b] &&
        cudaEventCreateWithFlags(&v->ev_free[b], cudaEventDisableTiming) != cudaSuccess) {
      v->ev_free[b] = nullptr;
      cudaGetLastError();
      return TSDF_ERR_CUDA;
    }
  }
  if (v->stream_slot_bytes < slot_bytes) {
    if (v->stream_stage) cudaFree(v->stream_stage);
    v->stream_stage = nullptr;
    v->stream_slot_bytes = 0;
    if (cudaMalloc(&v->stream_stage, 2 * slot_bytes) != cudaSuccess) {
      v->stream_stage = nullptr;
      cudaGetLastError();
      return TSDF_ERR_OUT_OF_MEMORY;
    }
    v->stream_slot_bytes = slot_bytes;
  }
  if (v->err_capacity < n) {
    if (v->err_words) cudaFreeHost(v->err_words);
    v->err_words = nullptr;
    v->err_capacity = 0;
    if (cudaMallocHost(reinterpret_cast<void**>(&v->err_words), sizeof(uint32_t) * n) !=
        cudaSuccess) {
      v->err_words = nullptr;
      cudaGetLastError();
      return TSDF_ERR_OUT_OF_MEMORY;
    }
    v->err_capacity = n;
  }
  return TSDF_OK;
}

}  // namespace

extern "C" tsdf_status tsdf_fuse_frames_host(const tsdf_frame* frames, int n,
                                             tsdf_status* status, void* stream) {
  if (!frames || n < 1 || !status) return TSDF_ERR_INVALID_ARG;
  tsdf_volume* owner = frames[0].volume;
  if (!owner) return TSDF_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != owner->device) return TSDF_ERR_INVALID_ARG;
  // Every frame is checked before anything is enqueued.
  size_t slot = 0;
  for (int i = 0; i < n; ++i) {
    const tsdf_frame& fr = frames[i];
    tsdf::FrameArgs f;
    const tsdf_status st = tsdf::make_frame(fr.volume, fr.depth, fr.width, fr.height, &fr.intr,
                                            &fr.pose, fr.rgb, &f);
    if (st != TSDF_OK) return st;
    if (fr.volume->device != owner->device) return TSDF_ERR_INVALID_ARG;
    const size_t b = frame_stage_bytes(fr);
    if (b > slot) slot = b;
  }
  tsdf_status st = ensure_resources(owner, slot, n);
  if (st != TSDF_OK) return st;

  cudaStream_t s = as_stream(stream);
  cudaStream_t cs = owner->copy_stream;
  char* stage = static_cast<char*>(owner->stream_stage);
  // the first copy into each slot waits for whatever was enqueued on `stream`
  // before this call (earlier users of the staging have synchronised, so this
  // only orders the copies after the caller's own preceding work)
  cudaError_t e = cudaEventRecord(owner->ev_free[0], s);
  if (e == cudaSuccess) e = cudaEventRecord(owner->ev_free[1], s);
  int enqueued = 0;
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const tsdf_frame& fr = frames[i];
    tsdf_volume* v = fr.volume;
    status[i] = TSDF_OK;
    if (v->poisoned) {
      status[i] = TSDF_ERR_POISONED;
      continue;
    }
    const int b = i & 1;
    const size_t npx = static_cast<size_t>(fr.width) * static_cast<size_t>(fr.height);
    char* dst = stage + b * owner->stream_slot_bytes;
    char* dst_rgb = dst + align_up(npx * sizeof(float));
    e = cudaStreamWaitEvent(cs, owner->ev_free[b], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dst, fr.depth, npx * sizeof(float), cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && fr.rgb)
      e = cudaMemcpyAsync(dst_rgb, fr.rgb, npx * 3, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess) e = cudaEventRecord(owner->ev_copied[b], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, owner->ev_copied[b], 0);
    if (e != cudaSuccess) break;
    st = tsdf_fuse_frame_async(v, reinterpret_cast<const float*>(dst), fr.width, fr.height,
                               &fr.intr, &fr.pose,
                               fr.rgb ? reinterpret_cast<const uint8_t*>(dst_rgb) : nullptr,
                               stream);
    if (st != TSDF_OK) {
      status[i] = st;
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaErrorLaunchFailure;
      break;
    }
    e = cudaMemcpyAsync(owner->err_words + i, &v->va.hdr->err, sizeof(uint32_t),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(owner->ev_free[b], s);
    enqueued = i + 1;
  }
  // one wait for the whole sequence (the copy stream's work is ordered
  // before `stream`'s through the events)
  const cudaError_t e_sync = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e_sync;
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (int i = enqueued; i < n; ++i)
      if (status[i] == TSDF_OK) status[i] = TSDF_ERR_CUDA;
    for (int i = 0; i < enqueued; ++i)
      if (status[i] == TSDF_OK) status[i] = TSDF_ERR_CUDA;
    return TSDF_ERR_CUDA;
  }
  // Per-frame status from the sticky error words: the first frame of a volume
  // whose word is set reports the error and poisons the volume; its later
  // frames did nothing on the device (the kernels skip a poisoned volume) and
  // report POISONED.
  tsdf_status first = TSDF_OK;
  for (int i = 0; i < n; ++i) {
    tsdf_volume* v = frames[i].volume;
    if (status[i] == TSDF_OK && owner->err_words[i] != 0u) {
      status[i] = v->poisoned ? TSDF_ERR_POISONED : decode_err(owner->err_words[i]);
      v->poisoned = true;
    }
    if (first == TSDF_OK && status[i] != TSDF_OK) first = status[i];
  }
  return first;
}
