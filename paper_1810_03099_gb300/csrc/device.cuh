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

// FP32 rescoring score of two unit signatures: the dot product over k entries, accumulated in
// four partial sums (entry q goes to sum q mod 4, in increasing q) that are added as
// (s0 + s1) + (s2 + s3). Every rescoring path uses this one order, so a pair gets the same
// score wherever it is rescored. Rows are read as float4 when k is a multiple of 4 (row
// starts are then 16-byte aligned); the order of the arithmetic is the same either way.
// X_L2: x is read through L2 only (rows written earlier in the same kernel).
template <bool X_L2 = false>
__device__ __forceinline__ float unit_dot(const float* __restrict__ x, const float* __restrict__ y, int k) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  if (k == 64) {  // the usual signature length: all 16 row loads of each side in flight at once
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* y4 = reinterpret_cast<const float4*>(y);
    float4 a[16], b[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      a[q] = X_L2 ? __ldcg(x4 + q) : __ldg(x4 + q);
      b[q] = __ldg(y4 + q);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      s0 = fmaf(a[q].x, b[q].x, s0);
      s1 = fmaf(a[q].y, b[q].y, s1);
      s2 = fmaf(a[q].z, b[q].z, s2);
      s3 = fmaf(a[q].w, b[q].w, s3);
    }
  } else if ((k & 3) == 0) {
    const float4* x4 = reinterpret_cast<const float4*>(x);
    const float4* y4 = reinterpret_cast<const float4*>(y);
#pragma unroll 4
    for (int q = 0; q < (k >> 2); ++q) {
      const float4 a = X_L2 ? __ldcg(x4 + q) : __ldg(x4 + q), b = __ldg(y4 + q);
      s0 = fmaf(a.x, b.x, s0);
      s1 = fmaf(a.y, b.y, s1);
      s2 = fmaf(a.z, b.z, s2);
      s3 = fmaf(a.w, b.w, s3);
    }
  } else {
    for (int q = 0; q < k; ++q) {
      const float a = X_L2 ? __ldcg(x + q) : __ldg(x + q), b = __ldg(y + q);
      switch (q & 3) {
        case 0: s0 = fmaf(a, b, s0); break;
        case 1: s1 = fmaf(a, b, s1); break;
        case 2: s2 = fmaf(a, b, s2); break;
        default: s3 = fmaf(a, b, s3); break;
      }
    }
  }
  return (s0 + s1) + (s2 + s3);
}

}  // namespace mrc
