// The fused tile kernel with each point's band walk split over 2, 4 or 8
// threads (tile_fused_body, TPP > 1), for the half bands compiled in the
// single-thread kernels (2, 4, 8) and the default probe load; and stage B's
// tile kernel (tile_fused_body with Op = kOpIntegrate). A translation unit of
// its own so that it compiles in parallel with the other kernels.
#include "tsdf_device.cuh"
#include "tsdf_launch.h"
#include "tsdf_tile.cuh"

namespace tsdf {

template <int M, int TPP>
static cudaError_t launch_split(const FrameArgs& f, const VolumeArgs& vol, cudaStream_t s) {
  const int tx = tiles_of(f.W);
  constexpr int rows = tile_rows<TPP>();
  const int ty = (f.H + rows - 1) / rows;
  tile_fused_kernel<kLoadCached, M, TPP><<<tx * ty, kThreads, 0, s>>>(f, vol, tx);
  return cudaGetLastError();
}

template <int M>
static cudaError_t launch_split_t(const FrameArgs& f, const VolumeArgs& vol, int tpp,
                                  cudaStream_t s) {
  switch (tpp) {
    case 2: return launch_split<M, 2>(f, vol, s);
    case 4: return launch_split<M, 4>(f, vol, s);
    case 8: return launch_split<M, 8>(f, vol, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int M>
static cudaError_t launch_integrate_m(const FrameArgs& f, const VolumeArgs& vol, cudaStream_t s) {
  const int tx = tiles_of(f.W);
  tile_fused_kernel<kLoadCached, M, 1, kOpIntegrate><<<tx * tiles_of(f.H), kThreads, 0, s>>>(
      f, vol, tx);
  return cudaGetLastError();
}

cudaError_t launch_integrate_tile(const FrameArgs& f, const VolumeArgs& vol, cudaStream_t s) {
  switch (f.M) {
    case 2: return launch_integrate_m<2>(f, vol, s);
    case 4: return launch_integrate_m<4>(f, vol, s);
    case 8: return launch_integrate_m<8>(f, vol, s);
    default: return launch_integrate_m<0>(f, vol, s);
  }
}

cudaError_t launch_fused_split(const FrameArgs& f, const VolumeArgs& vol, int threads_per_point,
                               cudaStream_t s) {
  cudaError_t e;
  switch (f.M) {
    case 2: e = launch_split_t<2>(f, vol, threads_per_point, s); break;
    case 4: e = launch_split_t<4>(f, vol, threads_per_point, s); break;
    case 8: e = launch_split_t<8>(f, vol, threads_per_point, s); break;
    default: return cudaErrorInvalidValue;
  }
  if (e == cudaSuccess) note_launch();
  return e;
}

}  // namespace tsdf
