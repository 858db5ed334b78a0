// simhash_match.cu -- Hamming matching of 64-bit Simhash fingerprints (row a7).
//
// Section III compares two Simhash values by their Hamming distance, the
// number of differing bits: popcount(a XOR b). A pair is emitted when the
// distance is <= hamming_max.
//
// Each CTA owns 256 rows of `a` (one fingerprint per thread, in a register)
// and one chunk of 1024 columns of `b` staged in shared memory; every thread
// sweeps the chunk with broadcast shared-memory reads. For all-pairs (b ==
// a) only chunks that hold some j > i are launched. The inner loop is integer
// ALU work: two 32-bit XORs, two POPCs, an add and a compare per pair, so the
// kernel is bound by the integer issue rate (the index sweep is HBM-bound only
// when `a` has very few rows).
#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

constexpr int kRows = 256;
constexpr int kChunk = 1024;

__global__ void __launch_bounds__(kRows) k_simhash_match(const uint64_t* __restrict__ a, int64_t na,
                                                         const uint64_t* __restrict__ b, int64_t nb, int32_t tri,
                                                         int32_t hmax, mrc_pair* pairs, unsigned long long* count,
                                                         int64_t capacity) {
  __shared__ __align__(16) uint64_t sb[kChunk];
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  const int64_t c0 = (int64_t)blockIdx.y * kChunk;
  if (tri && c0 + kChunk <= r0 + 1) return;  // no column j > i anywhere in this block
  const int64_t i = r0 + threadIdx.x;
  const int m = (int)(nb - c0 < kChunk ? nb - c0 : kChunk);
  for (int x = threadIdx.x; x < m; x += kRows) sb[x] = b[c0 + x];
  __syncthreads();
  if (i >= na) return;
  const uint64_t ai = a[i];
  const uint32_t alo = (uint32_t)ai, ahi = (uint32_t)(ai >> 32);
  const int mm = m & ~1;
  for (int x = 0; x < mm; x += 2) {
    const uint4 two = *reinterpret_cast<const uint4*>(&sb[x]);
    const int h0 = __popc(alo ^ two.x) + __popc(ahi ^ two.y);
    const int h1 = __popc(alo ^ two.z) + __popc(ahi ^ two.w);
    if (min(h0, h1) <= hmax) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int h = e ? h1 : h0;
        const int64_t j = c0 + x + e;
        if (h <= hmax && (!tri || j > i)) {
          const unsigned long long at = atomicAdd(count, 1ull);
          if (at < (unsigned long long)capacity) {
            mrc_pair pr;
            pr.i = (int32_t)i;
            pr.j = (int32_t)j;
            pr.score = (float)h;
            pairs[at] = pr;
          }
        }
      }
    }
  }
  if (m & 1) {
    const uint64_t bx = sb[m - 1];
    const int h = __popcll(ai ^ bx);
    const int64_t j = c0 + m - 1;
    if (h <= hmax && (!tri || j > i)) {
      const unsigned long long at = atomicAdd(count, 1ull);
      if (at < (unsigned long long)capacity) {
        mrc_pair pr;
        pr.i = (int32_t)i;
        pr.j = (int32_t)j;
        pr.score = (float)h;
        pairs[at] = pr;
      }
    }
  }
}

}  // namespace

cudaError_t launch_simhash_match(mrc_ctx* ctx, const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb,
                                 int32_t hmax, mrc_pair* pairs, unsigned long long* count, int64_t capacity) {
  const int tri = b == nullptr;
  if (tri) {
    b = a;
    nb = na;
  }
  if (na <= 0 || nb <= 0) return cudaSuccess;
  const int64_t gx = (na + kRows - 1) / kRows, gy = (nb + kChunk - 1) / kChunk;
  if (gx > 0x7FFFFFFF || gy > 65535) return cudaErrorInvalidValue;
  const double pairs_eval = tri ? (double)na * (double)(na - 1) / 2.0 : (double)na * (double)nb;
  cudaEvent_t ev = nullptr;
  // algorithmic bytes: both fingerprint arrays read once; ops: 6 integer instructions per pair
  timing_begin(ctx, "simhash_match", 8.0 * (double)(na + (tri ? 0 : nb)), 6.0 * pairs_eval, &ev);
  k_simhash_match<<<dim3((unsigned)gx, (unsigned)gy), kRows, 0, ctx->stream>>>(a, na, b, nb, tri, hmax, pairs, count,
                                                                              capacity);
  timing_end(ctx, ev);
  return cudaGetLastError();
}

}  // namespace mrc
