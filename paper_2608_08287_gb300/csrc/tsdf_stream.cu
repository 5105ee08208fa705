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
//
// A frame's error word is read right after its kernel only when a later frame
// of the call goes into the same volume (its sticky bits would otherwise mix
// with the later frame's); the last frame of each volume is read after the
// last kernel -- the words gathered by one small kernel into a device array,
// copied back at once -- so a sequence of frames into distinct volumes runs
// its kernels back to back.
#include <cstring>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "tsdf.h"
#include "tsdf_internal.h"
#include "tsdf_launch.h"

using tsdf::align_up;
using tsdf::as_stream;
using tsdf::decode_err;
using tsdf::from_cuda;

namespace {

// Error words of up to kGather volumes copied into one device array.
constexpr int kGather = 256;
struct GatherArgs {
  unsigned int* dst;
  int n;
  const unsigned int* src[kGather];
};

__global__ void gather_err_kernel(const __grid_constant__ GatherArgs a) {
  const int i = static_cast<int>(threadIdx.x);
  if (i < a.n) a.dst[i] = *reinterpret_cast<const volatile unsigned int*>(a.src[i]);
}

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
    if (v->err_gathered) cudaFreeHost(v->err_gathered);
    if (v->err_dev) cudaFree(v->err_dev);
    v->err_words = v->err_gathered = v->err_dev = nullptr;
    v->err_capacity = 0;
    if (cudaMallocHost(reinterpret_cast<void**>(&v->err_words), sizeof(uint32_t) * n) !=
            cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&v->err_gathered), sizeof(uint32_t) * n) !=
            cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&v->err_dev), sizeof(uint32_t) * n) != cudaSuccess) {
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

  // which frames have a later frame in the same volume
  std::unordered_map<const tsdf_volume*, int> last_of;
  last_of.reserve(static_cast<size_t>(n) * 2);
  for (int i = 0; i < n; ++i) last_of[frames[i].volume] = i;

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
    if (last_of[v] != i)
      e = cudaMemcpyAsync(owner->err_words + i, &v->va.hdr->err, sizeof(uint32_t),
                          cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(owner->ev_free[b], s);
    enqueued = i + 1;
  }
  // the last frame of each volume: its word after every kernel of the call,
  // gathered on the device and copied back in one piece
  std::vector<int> gathered;
  for (int i = 0; i < enqueued; ++i)
    if (status[i] == TSDF_OK && last_of[frames[i].volume] == i) gathered.push_back(i);
  for (size_t c = 0; c < gathered.size() && e == cudaSuccess; c += kGather) {
    GatherArgs a;
    a.dst = owner->err_dev + c;
    a.n = static_cast<int>(gathered.size() - c < static_cast<size_t>(kGather)
                               ? gathered.size() - c
                               : kGather);
    for (int j = 0; j < a.n; ++j) a.src[j] = &frames[gathered[c + j]].volume->va.hdr->err;
    gather_err_kernel<<<1, kGather, 0, s>>>(a);
    e = cudaGetLastError();
    tsdf::note_launch();
  }
  if (e == cudaSuccess && !gathered.empty())
    e = cudaMemcpyAsync(owner->err_gathered, owner->err_dev, sizeof(uint32_t) * gathered.size(),
                        cudaMemcpyDeviceToHost, s);
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
  for (size_t j = 0; j < gathered.size(); ++j)
    owner->err_words[gathered[j]] = owner->err_gathered[j];
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
