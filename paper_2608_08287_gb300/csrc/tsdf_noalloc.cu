// tsdf_fuse_frame_host_noalloc: fuse a frame given in host memory without
// allocating anything.
//
// tsdf_fuse_frame_host copies the caller's host depth and colour into device
// staging that the volume allocates on first use. Some callers cannot let a
// library do that: a real-time capture loop must not stall on cudaMalloc (it
// can block and synchronise the whole device), a process whose device memory
// is fully budgeted by its own allocator cannot have a library take more
// behind its back, and a host application that loads this library as a plugin
// may forbid plugins from owning device memory at all. For them, this entry
// point stages the frame in a fixed array compiled into the library instead.
//
// The staging array is a file-scope __device__ array of
// TSDF_NOALLOC_MAX_PIXELS * 7 bytes (4 MiB of depth plus 3 MiB of colour).
// Every GPU that loads the library holds it until the process exits. Host code
// cannot use the array's name as a device address, so the first call on each
// device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it; later calls reuse it. The cache lives as long as
// the process's CUDA context: cudaDeviceReset is not supported between calls
// (it would also destroy every volume).
#include <mutex>

#include <cuda_runtime.h>

#include "tsdf.h"
#include "tsdf_internal.h"

namespace {

constexpr size_t kDepthBytes = static_cast<size_t>(TSDF_NOALLOC_MAX_PIXELS) * sizeof(float);
constexpr size_t kRgbBytes = static_cast<size_t>(TSDF_NOALLOC_MAX_PIXELS) * 3;
static_assert(kDepthBytes % 256 == 0, "colour staging must stay 256-byte aligned");

// The staging itself. Each call overwrites the part it uses before any kernel
// reads it, so nothing in it has to start at zero.
static __device__ __align__(256) unsigned char g_staging[kDepthBytes + kRgbBytes];

constexpr int kMaxDevices = 256;
std::mutex g_mutex;
void* g_staging_addr[kMaxDevices] = {};

// Device address of g_staging on the current device (looked up once per device).
tsdf_status staging_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TSDF_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return TSDF_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (g_staging_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_staging);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return TSDF_ERR_CUDA;
    }
    g_staging_addr[dev] = p;
  }
  *out = g_staging_addr[dev];
  return TSDF_OK;
}

}  // namespace

extern "C" tsdf_status tsdf_fuse_frame_host_noalloc(tsdf_volume* vol, const float* depth_host,
                                                    int width, int height,
                                                    const tsdf_intrinsics* intr,
                                                    const tsdf_pose* pose,
                                                    const uint8_t* rgb_host, void* stream) {
  if (!vol || !depth_host || !intr || !pose || width < 1 || height < 1)
    return TSDF_ERR_INVALID_ARG;
  const size_t npx = static_cast<size_t>(width) * static_cast<size_t>(height);
  if (npx > static_cast<size_t>(TSDF_NOALLOC_MAX_PIXELS)) return TSDF_ERR_INVALID_ARG;
  // Every check the fuse call makes before it enqueues work is made here,
  // before the staging copies: a call that is refused leaves no copy in
  // flight into the shared array.
  tsdf::FrameArgs f;
  tsdf_status st = tsdf::make_frame(vol, depth_host, width, height, intr, pose, rgb_host, &f);
  if (st != TSDF_OK) return st;
  if (vol->poisoned) return TSDF_ERR_POISONED;
  void* base = nullptr;
  st = staging_address(&base);
  if (st != TSDF_OK) return st;
  unsigned char* depth_dev = static_cast<unsigned char*>(base);
  unsigned char* rgb_dev = depth_dev + kDepthBytes;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(depth_dev, depth_host, npx * sizeof(float),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && rgb_host)
    e = cudaMemcpyAsync(rgb_dev, rgb_host, npx * 3, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(s);  // a first copy may be in flight
    return TSDF_ERR_CUDA;
  }
  // Both stages, then wait for the stream and read the status: the staging is
  // free for the next call once this returns. The fuse call synchronises the
  // stream on success and on every device status; a launch that fails returns
  // before that, so the copies are waited for here.
  st = tsdf_fuse_frame(vol, reinterpret_cast<const float*>(depth_dev), width, height, intr,
                       pose, rgb_host ? rgb_dev : nullptr, stream);
  if (st != TSDF_OK) cudaStreamSynchronize(s);
  return st;
}
