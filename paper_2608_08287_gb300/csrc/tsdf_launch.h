// Internal interface between the host runtime (tsdf_api.cu) and the kernels
// (tsdf_kernels.cu). Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "tsdf_device.cuh"

namespace tsdf {

// Launch accounting: every kernel launch the library enqueues is counted.
void note_launch();

cudaError_t launch_allocate(const FrameArgs& f, const VolumeArgs& vol, int probe_load, int mode,
                            cudaStream_t s);
// Stage B: mode 0 = per-thread lookups, 1 = warp kernel, 2 = tile kernel.
cudaError_t launch_integrate(const FrameArgs& f, const VolumeArgs& vol, int mode,
                             cudaStream_t s);
// The fused path. threads_per_point > 1 (2, 4 or 8) takes the fused tile
// kernel with each point's walk split over that many threads; it exists for
// fuse mode 2, the default probe load and half bands 2, 4 and 8
// (cudaErrorInvalidValue otherwise).
cudaError_t launch_fused(const FrameArgs& f, const VolumeArgs& vol, int probe_load, int mode,
                         int threads_per_point, cudaStream_t s);
// Stage B, tile strategy (integrate mode 2): the fused tile kernel's phases
// with phase 2 looking the tile's keys up instead of inserting them.
cudaError_t launch_integrate_tile(const FrameArgs& f, const VolumeArgs& vol, cudaStream_t s);
// The split-walk fused tile kernels (their own translation unit).
cudaError_t launch_fused_split(const FrameArgs& f, const VolumeArgs& vol, int threads_per_point,
                               cudaStream_t s);
// Batched launches (all frames of a session table): allocate + integrate, or
// the fused kernel. factor caps the resident CTAs per SM (0 = as many as fit).
// grid_limit > 0 caps the grid (e.g. at the batch's tile count). all_m4: every
// frame has half band 4 (selects the fused kernel compiled for that band).
// stages (fuse mode 0): 1 = stage A only, 2 = stage B only, 3 = both.
cudaError_t launch_batch(const BatchHeader* table, int probe_load, int allocate_mode,
                         int integrate_mode, int fuse_mode, int factor, int grid_limit,
                         bool all_m4, int stages, cudaStream_t s);
cudaError_t launch_batch_status(const BatchHeader* table, unsigned* out, cudaStream_t s);
// Means of n blocks into out (n x 5 x 512); block j is pool block list[j], or
// j when list is null.
cudaError_t launch_export(const VolumeArgs& vol, float* out, unsigned int n,
                          const unsigned int* list, cudaStream_t s);
// Slot-index volumes: occupied slots in slot order (list) and their block
// coordinates, at most cap of them; *found = occupied slots.
cudaError_t launch_slot_list(const VolumeArgs& vol, unsigned int* list, int32_t* coords,
                             unsigned int cap, unsigned int* found, cudaStream_t s);
// Zero the used pool blocks (before the table is cleared).
cudaError_t launch_clear_used(const VolumeArgs& vol, int sm_count, cudaStream_t s);
// Marching-tetrahedra surface of the volume: triangles (9 floats each) and
// cell records (4 int32 each), either may be null; writes at most capacity of
// them and adds the total to *counter (which the caller zeroes first).
cudaError_t launch_extract(const VolumeArgs& vol, float v, float* tris, int32_t* cells,
                           unsigned int capacity, unsigned int* counter, int sm_count,
                           cudaStream_t s);
// Accumulate table occupancy, probe lengths and the pool's total weight into
// *out (which the caller zeroes first).
cudaError_t launch_table_stats(const VolumeArgs& vol, TableStatsDev* out, int sm_count,
                               cudaStream_t s);

}  // namespace tsdf
