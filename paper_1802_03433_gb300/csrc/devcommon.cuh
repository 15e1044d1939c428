// Definitions shared by the precompiled kernels and the kernels the library
// compiles at run time with NVRTC (jit.cu): fixed-width integer types, the
// device error bits latched per mesh, and the padded local-row stride.  Under
// NVRTC no host header is available, so the integer types are declared here
// (LP64: long is 64 bits on the x86-64 and AArch64 targets).
#pragma once

#ifdef __CUDACC_RTC__
typedef int int32_t;
typedef long int64_t;
typedef unsigned char uint8_t;
typedef unsigned int uint32_t;
#else
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace fea {

// Bits of the device error word latched per mesh.
enum : int {
  DEV_ERR_INDEX = 1,
  DEV_ERR_DEGENERATE = 2,
  DEV_ERR_OVERFLOW = 4,
  DEV_ERR_TIMEOUT = 8,
};

// Local rows of nl values of `bytes` bytes each are lstride(nl, bytes) values
// apart: a whole number of 32-byte DRAM sectors, written in full (padding
// included), so no sector is ever left partly written (a partly written
// sector costs a DRAM read-fill).
__host__ __device__ constexpr int lstride(int nl, int bytes) { return ((nl * bytes + 31) / 32) * 32 / bytes; }

// Bounds checks of the checked build (compiled with -DFEA_CHECKED, the
// library libfea_checked.so): an index outside [0, n) latches DEV_ERR_INDEX
// in the error word and the caller skips the access (a gather reads entry 0
// instead).  In the normal build the test is the constant true and compiles
// away.  The inputs are validated when a mesh is created, so a failing check
// points at the library, not at the caller.
__device__ __forceinline__ bool index_ok(int64_t i, int64_t n, int* err) {
#ifdef FEA_CHECKED
  if (i >= 0 && i < n) return true;
  if (err) atomicOr(err, DEV_ERR_INDEX);
  return false;
#else
  (void)i;
  (void)n;
  (void)err;
  return true;
#endif
}

// A gather index: i itself, or 0 (after latching DEV_ERR_INDEX) when the
// checked build finds it outside [0, n).
__device__ __forceinline__ int32_t checked_index(int32_t i, int64_t n, int* err) {
  return index_ok(i, n, err) ? i : 0;
}

}  // namespace fea
