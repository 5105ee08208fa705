// Range checks of the checked build (-DTSDF_CHECKED), the stand-in for a
// memory checker: before an access, an index into the block pool, the hash
// table, the block-coordinate array or a frame's depth or colour image is
// compared with its bound. An index out of range sets TSDF_ERRBIT_BOUNDS in
// the volume's sticky error word (the fuse call then returns
// TSDF_ERR_BOUNDS) and the caller skips the access. Default builds compile
// the checks out: index_ok is then `true` and costs nothing.
//
// Plain C++ apart from the CUDA annotations, so that the check itself can be
// compiled and exercised on the host.
#pragma once

#include "tsdf.h"

#if defined(__CUDACC__)
#define TSDF_CHECK_FN __host__ __device__ __forceinline__
#else
#define TSDF_CHECK_FN inline
#endif

namespace tsdf {

#ifdef TSDF_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// Records an out-of-range index in the error word err (may be null).
TSDF_CHECK_FN void report_bounds(unsigned int* err) {
  if (!err) return;
#if defined(__CUDA_ARCH__)
  atomicOr(err, static_cast<unsigned int>(TSDF_ERRBIT_BOUNDS));
#else
  *err |= static_cast<unsigned int>(TSDF_ERRBIT_BOUNDS);
#endif
}

// True when index i lies in [0, n); otherwise (checked builds) the BOUNDS bit
// is set in *err and the caller must skip the access.
TSDF_CHECK_FN bool index_ok(unsigned long long i, unsigned long long n, unsigned int* err) {
  if (!kChecked) return true;
  if (i < n) return true;
  report_bounds(err);
  return false;
}

// The same for a signed index (negative is out of range).
TSDF_CHECK_FN bool index_ok_signed(long long i, unsigned long long n, unsigned int* err) {
  if (!kChecked) return true;
  if (i >= 0 && static_cast<unsigned long long>(i) < n) return true;
  report_bounds(err);
  return false;
}

}  // namespace tsdf
