// simhash_match.cu -- Hamming matching of 64-bit Simhash fingerprints (row a7).
//
// Section III compares two Simhash values by their Hamming distance, the
// number of differing bits: popcount(a XOR b). A pair is emitted when the
// distance is <= hamming_max.
//
// Each CTA owns 256 rows of `a` (one fingerprint per thread, in a register)
// and one chunk of 512 columns of `b` staged in shared memory as separate low
// and high 32-bit halves; every thread sweeps the chunk with broadcast
// shared-memory reads, four columns per 16-byte read. For all-pairs (b == a)
// only chunks that hold some j > i do work. The inner loop is one XOR and one
// POPC per pair on the low halves (see k_simhash_match), so the kernel is
// bound by the POPC issue rate (the index sweep is HBM-bound only when `a`
// has very few rows).
#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

constexpr int kRows = 256;
constexpr int kChunk = 512;

__device__ __forceinline__ void emit(int64_t i, int64_t j, int h, mrc_pair* pairs, unsigned long long* count,
                                     int64_t capacity) {
  const unsigned long long at = atomicAdd(count, 1ull);
  if (at < (unsigned long long)capacity) {
    mrc_pair pr;
    pr.i = (int32_t)i;
    pr.j = (int32_t)j;
    pr.score = (float)h;
    pairs[at] = pr;
  }
}

// The low 32 bits alone already decide almost every pair: popc(a ^ b) <= hmax needs
// popc(low(a) ^ low(b)) <= hmax, which random 32-bit words meet with probability ~1e-6 at
// hmax = 3. So the sweep costs one XOR and one POPC per pair; the high halves are read only
// for the rare pairs that pass.
__global__ void __launch_bounds__(kRows) k_simhash_match(const uint64_t* __restrict__ a, int64_t na,
                                                         const uint64_t* __restrict__ b, int64_t nb, int32_t tri,
                                                         int32_t hmax, mrc_pair* pairs, unsigned long long* count,
                                                         int64_t capacity) {
  __shared__ __align__(16) uint32_t slo[kChunk];
  __shared__ __align__(16) uint32_t shi[kChunk];
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  const int64_t c0 = (int64_t)blockIdx.y * kChunk;
  if (tri && c0 + kChunk <= r0 + 1) return;  // no column j > i anywhere in this block
  const int64_t i = r0 + threadIdx.x;
  const int m = (int)(nb - c0 < kChunk ? nb - c0 : kChunk);
  for (int x = threadIdx.x; x < kChunk; x += kRows) {
    // columns past the end are padding, rejected by the bounds check of the slow path
    const uint64_t v = x < m ? b[c0 + x] : ~0ull;
    slo[x] = (uint32_t)v;
    shi[x] = (uint32_t)(v >> 32);
  }
  __syncthreads();
  if (i >= na) return;
  const uint64_t ai = a[i];
  const uint32_t alo = (uint32_t)ai, ahi = (uint32_t)(ai >> 32);
#pragma unroll 4
  for (int x = 0; x < kChunk; x += 4) {
    const uint4 q = *reinterpret_cast<const uint4*>(&slo[x]);
    const int h0 = __popc(alo ^ q.x), h1 = __popc(alo ^ q.y), h2 = __popc(alo ^ q.z), h3 = __popc(alo ^ q.w);
    if (min(min(h0, h1), min(h2, h3)) <= hmax) {
      const int hl[4] = {h0, h1, h2, h3};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t j = c0 + x + e;
        if (hl[e] <= hmax && x + e < m && (!tri || j > i)) {
          const int h = hl[e] + __popc(ahi ^ shi[x + e]);
          if (h <= hmax) emit(i, j, h, pairs, count, capacity);
        }
      }
    }
  }
}

// Throughput probe of the all-pairs match's bounding unit: every thread keeps eight independent
// population counts of a rotating word in flight (XOR, POPC, add each), so the loop runs at the
// rate the SMs issue 32-bit POPC. The result is kept live through a data-dependent store that
// never happens for these inputs.
__global__ void __launch_bounds__(256) k_popc_rate(uint32_t seed, int32_t iters, unsigned long long* sink) {
  uint32_t x[8], acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    x[u] = seed * (threadIdx.x + 1u) + (uint32_t)u * 0x9E3779B9u + blockIdx.x;
    acc[u] = 0u;
  }
  uint32_t k = blockIdx.x * 0x85EBCA6Bu;
  for (int32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += (uint32_t)__popc(x[u] ^ k);
    k += 0x9E3779B9u;
  }
  uint32_t t = 0u;
#pragma unroll
  for (int u = 0; u < 8; ++u) t += acc[u];
  if (t == 0xFFFFFFFFu) *sink = t;  // at most 8 * 32 * iters < 2^32 - 1
}

}  // namespace

cudaError_t measure_popc_rate(mrc_ctx* ctx, double* popc_per_s) {
  constexpr int32_t kIters = 4096;
  const int64_t blocks = (int64_t)ctx->num_sms * 8;
  unsigned long long* sink = nullptr;
  cudaError_t e = cudaMallocAsync(&sink, sizeof(unsigned long long), ctx->stream);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 0.f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first run warms up
    e = cudaEventRecord(e0, ctx->stream);
    k_popc_rate<<<(unsigned)blocks, 256, 0, ctx->stream>>>(0x1810u + (uint32_t)rep, kIters, sink);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best_ms == 0.f || ms < best_ms)) best_ms = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sink, ctx->stream);
  if (e != cudaSuccess) return e;
  *popc_per_s = (double)blocks * 256.0 * 8.0 * kIters / (best_ms * 1e-3);
  return cudaStreamSynchronize(ctx->stream);
}

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
  // algorithmic bytes: both fingerprint arrays read once; ops: one POPC per pair
  timing_begin(ctx, "simhash_match", 8.0 * (double)(na + (tri ? 0 : nb)), pairs_eval, &ev);
  k_simhash_match<<<dim3((unsigned)gx, (unsigned)gy), kRows, 0, ctx->stream>>>(a, na, b, nb, tri, hmax, pairs, count,
                                                                              capacity);
  timing_end(ctx, ev);
  return cudaGetLastError();
}

}  // namespace mrc
