// device.cuh -- small device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mrc {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Device error word bits (ORed into a per-call int32).
constexpr int32_t kErrBadToken = 1;    // token id outside [0, vocab)
constexpr int32_t kErrBadOffsets = 2;  // offsets not non-decreasing from 0
constexpr int32_t kErrTimeout = 4;     // a bounded wait gave up
constexpr int32_t kErrTable = 8;       // a per-document table overflowed (cannot happen at load <= 1/2)
constexpr int32_t kErrTooLong = 16;    // a document longer than the supported maximum
constexpr int32_t kErrOverflow = 32;   // a candidate buffer overflowed (pairs may be missing)

__device__ __forceinline__ void set_err(int32_t* err, int32_t bit) {
  if (err) atomicOr(err, bit);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

}  // namespace mrc
