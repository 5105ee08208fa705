// Internal host-side definitions shared by the host runtime files
// (tsdf_api.cu, tsdf_batch.cu). Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "tsdf.h"
#include "tsdf_device.cuh"

namespace tsdf {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte offsets of a volume's sections inside its one allocation.
struct Offsets {
  size_t table, coords, twrg, blue, total;
};

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

tsdf_status from_cuda(cudaError_t e);
tsdf_status decode_err(uint32_t err);

// Threads per point of the fused tile kernel chosen for work of `tiles`
// 16 x 16 pixel tiles running alone on the GPU (one frame, or all frames of a
// batch launched together): the largest of 1, 2, 4 whose CTAs (tiles x TPP)
// still fit the GPU's resident slots at four CTAs per SM -- work that fills
// the GPU keeps one thread per point -- where the split walk exists (fuse
// mode 2, the default probe load, half band 2, 4 or 8), else 1.
int auto_threads_per_point(int fuse_mode, int probe_load, int half_band, int sm_count,
                           long long tiles);
inline long long tiles_of_frame(int width, int height) {
  return static_cast<long long>((width + 15) / 16) * ((height + 15) / 16);
}

}  // namespace tsdf

struct tsdf_volume {
  int device = 0;
  int sm_count = 0;
  float voxel = 0.0f, trunc = 0.0f;
  int half_band = 0;
  uint32_t slots = 0, pool = 0;
  void* mem = nullptr;
  size_t bytes = 0;
  bool owns = false;
  tsdf::Offsets off{};
  tsdf::VolumeArgs va{};
  bool poisoned = false;
  bool dirty = false;          // something was fused since creation or the last reset
  uint32_t* pinned = nullptr;  // {count, err}
  int probe_load = tsdf::kLoadCached;
  int allocate_mode = 1;
  int integrate_mode = 0;
  int fuse_mode = 2;
  int threads_per_point = 0;  // of the fused tile kernel (0: chosen per frame)
  int threads = 256;
  void* stage = nullptr;
  size_t stage_bytes = 0;
  // streaming host input (tsdf_fuse_frames_host), made on first use: two
  // staging slots, a copy stream, slot filled / slot free events, and pinned
  // per-frame error words
  void* stream_stage = nullptr;
  size_t stream_slot_bytes = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_free[2] = {nullptr, nullptr};
  uint32_t* err_words = nullptr;      // pinned, one word per frame of a call
  uint32_t* err_gathered = nullptr;   // pinned, the words gathered on the device
  uint32_t* err_dev = nullptr;        // device, where they are gathered
  int err_capacity = 0;
};

namespace tsdf {
// Validate a frame and build its kernel arguments (no CUDA call).
tsdf_status make_frame(const tsdf_volume* v, const float* depth, int w, int h,
                       const tsdf_intrinsics* intr, const tsdf_pose* pose, const uint8_t* rgb,
                       FrameArgs* f);
}  // namespace tsdf
