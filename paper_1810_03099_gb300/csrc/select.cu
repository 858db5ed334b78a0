// select.cu -- reference selection on the device (Section IV, REGION selection).
//
// Terms are ranked by df descending, ids ascending within equal df; the selection takes the
// ranks [start, start + L) and partition p holds selection positions
// [floor(pL/k), floor((p+1)L/k)). With cnt[v] terms of df v, the terms of df v hold the ranks
// [#{df > v}, #{df > v} + cnt[v]), so only the df values whose rank range meets the selection
// matter: a contiguous band of values [v_lo, v_hi]. The device pass
//   1. histograms df (k_df_hist),
//   2. turns the histogram into #{df > v} and finds start, L and the band (one CTA,
//      k_sel_band),
//   3. collects the band's terms (k_band_collect) and
//   4. sorts them by (df descending, id ascending) in shared memory, which gives their ranks,
//      writes the partition of every selected term and the reference norms |R_p| (one CTA,
//      k_band_place; each partition summed by one thread in rank order, in double).
// A band of more than kBandMax terms (a tie group larger than the buffer) is reported in the
// status word; the caller then selects on the host.
#include <cuda_bf16.h>

#include <climits>

#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

constexpr int kSelThreads = 1024;
constexpr int kBandMax = 8192;  // band terms sorted in shared memory (64 KB of keys)

// Selection state (int64 words): [0] start, [1] L, [2] v_lo, [3] v_hi, [4] rank of the
// band's first term, [5] band size, [6] status (0 ok, 1 band too large), [7] largest df.
enum { kSsStart = 0, kSsL, kSsVlo, kSsVhi, kSsRank0, kSsBand, kSsStatus, kSsMaxdf, kSsWords = 8 };

__global__ void k_df_hist(const int32_t* __restrict__ df, int32_t V, int32_t* __restrict__ hist,
                          long long* __restrict__ state) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  int32_t d = t < V ? df[t] : 0;
  if (d > 0) atomicAdd(&hist[d], 1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d = max(d, __shfl_xor_sync(kFull, d, o));
  if ((threadIdx.x & 31) == 0 && d > 0) atomicMax(&state[kSsMaxdf], (long long)d);
}

// One CTA. above[v] = #{terms with df > v} for v in [0, maxdf]; then the selection and the
// band of df values whose ranks meet it.
__global__ void __launch_bounds__(kSelThreads, 1) k_sel_band(const int32_t* __restrict__ hist, int32_t* __restrict__ above,
                                                         int64_t n_docs, int64_t L, int64_t region_start,
                                                         long long* __restrict__ state) {
  __shared__ long long part[kSelThreads];
  __shared__ long long s_lo, s_hi;
  const int64_t maxdf = state[kSsMaxdf];
  // values in descending order: thread i takes the contiguous run [hi_i - per, hi_i]
  const int64_t nv = maxdf;  // values 1..maxdf
  const int64_t per = (nv + kSelThreads - 1) / kSelThreads;
  const int64_t v_top = maxdf - (int64_t)threadIdx.x * per;  // this thread's largest value
  long long sum = 0;
  for (int64_t q = 0; q < per; ++q) {
    const int64_t v = v_top - q;
    if (v >= 1) sum += hist[v];
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  // exclusive scan (in descending-value order) by a single warp over the 1024 run sums
  if (threadIdx.x < 32) {
    long long carry = 0;
    for (int c = 0; c < kSelThreads; c += 32) {
      const long long x = part[c + threadIdx.x];
      long long incl = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, incl, o);
        if ((int)threadIdx.x >= o) incl += y;
      }
      part[c + threadIdx.x] = carry + incl - x;
      carry += __shfl_sync(kFull, incl, 31);
    }
  }
  __syncthreads();
  long long run = part[threadIdx.x];  // terms with df > v_top
  for (int64_t q = 0; q < per; ++q) {
    const int64_t v = v_top - q;
    if (v >= 1) {
      above[v] = (int32_t)run;
      run += hist[v];
    }
  }
  if (threadIdx.x == kSelThreads - 1) above[0] = (int32_t)run;  // every term with df >= 1
  if (threadIdx.x == 0) {
    s_lo = LLONG_MAX;
    s_hi = -1;
  }
  __syncthreads();
  const int64_t ranked = above[0];
  int64_t start = region_start;
  if (start < 0) {
    const int64_t vcap = n_docs / 100;  // first rank whose df <= N / 100
    start = vcap >= maxdf ? 0 : (vcap >= 1 ? above[vcap] : ranked);
  }
  start = min(start, ranked);
  const int64_t end = min(start + L, ranked);
  for (int64_t q = 0; q < per; ++q) {
    const int64_t v = v_top - q;
    if (v >= 1) {
      const int64_t lo_rank = above[v], cnt = (int64_t)(v > 1 ? above[v - 1] : ranked) - above[v];
      if (cnt > 0 && lo_rank < end && lo_rank + cnt > start) {
        atomicMin(&s_lo, (long long)v);
        atomicMax(&s_hi, (long long)v);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    state[kSsStart] = start;
    state[kSsL] = end - start;
    state[kSsVlo] = s_hi >= 0 ? s_lo : 1;
    state[kSsVhi] = s_hi;  // -1: empty selection
    state[kSsRank0] = s_hi >= 0 ? above[s_hi] : 0;
    state[kSsBand] = 0;
    state[kSsStatus] = 0;
  }
}

__global__ void k_band_collect(const int32_t* __restrict__ df, int32_t V, long long* __restrict__ state,
                               unsigned long long* __restrict__ keys) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= V) return;
  const int32_t d = df[t];
  if (d < state[kSsVlo] || d > state[kSsVhi]) return;
  const long long at = (long long)atomicAdd(reinterpret_cast<unsigned long long*>(&state[kSsBand]), 1ull);
  // ascending keys = df descending, then id ascending
  if (at < kBandMax) keys[at] = ((unsigned long long)(0xFFFFFFFFu - (uint32_t)d) << 32) | (uint32_t)t;
}

// One CTA: sorts the band, writes the partition of each selected term (part holds -1 for
// every term on entry) and the reference norms. idf NULL: count weighting (r = 1).
__global__ void __launch_bounds__(kSelThreads) k_band_place(const unsigned long long* __restrict__ keys,
                                                           long long* __restrict__ state, const float* __restrict__ idf,
                                                           int32_t bf16, int32_t k, int32_t* __restrict__ part,
                                                           double* __restrict__ rnorm, float* __restrict__ rinv) {
  extern __shared__ unsigned long long sk[];  // [kBandMax]
  const long long nb = state[kSsBand];
  if (nb > kBandMax) {
    if (threadIdx.x == 0) state[kSsStatus] = 1;
    return;
  }
  int n2 = 1;
  while (n2 < nb) n2 <<= 1;
  for (int x = threadIdx.x; x < n2; x += kSelThreads) sk[x] = x < nb ? keys[x] : ~0ull;
  __syncthreads();
  for (int kk = 2; kk <= n2; kk <<= 1) {
    for (int j = kk >> 1; j > 0; j >>= 1) {
      for (int x = threadIdx.x; x < n2; x += kSelThreads) {
        const int y = x ^ j;
        if (y > x) {
          const unsigned long long a = sk[x], b = sk[y];
          if ((a > b) == ((x & kk) == 0)) {
            sk[x] = b;
            sk[y] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  const long long start = state[kSsStart], L = state[kSsL], rank0 = state[kSsRank0];
  // band position x holds rank rank0 + x; selection position = rank - start
  for (int x = threadIdx.x; x < nb; x += kSelThreads) {
    const long long pos = rank0 + x - start;
    if (pos >= 0 && pos < L) part[(uint32_t)sk[x]] = (int32_t)(((pos + 1) * k - 1) / L);
  }
  // partition q: selection positions [floor(qL/k), floor((q+1)L/k)), summed in rank order
  for (int q = threadIdx.x; q < k; q += kSelThreads) {
    double s = 0.0;
    const long long p0 = q * L / k, p1 = (q + 1) * L / k;
    for (long long pos = p0; pos < p1; ++pos) {
      const uint32_t t = (uint32_t)sk[pos + start - rank0];
      double r = 1.0;
      if (idf) r = bf16 ? (double)__bfloat162float(__float2bfloat16_rn(idf[t])) : (double)idf[t];
      s += r * r;
    }
    const double nr = sqrt(s);
    rnorm[q] = nr;
    rinv[q] = nr > 0.0 ? (float)(1.0 / nr) : 0.f;
  }
}

}  // namespace

int64_t device_selection_words() { return kSsWords; }

cudaError_t launch_select_region(mrc_ctx* ctx, const int32_t* df, int32_t V, int64_t n_docs, int64_t L,
                                 int64_t region_start, const float* idf, int32_t bf16, int32_t k, int32_t* hist,
                                 int32_t* above, long long* state, unsigned long long* keys, int32_t* part,
                                 double* rnorm, float* rinv) {
  if (V <= 0 || k <= 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * ((size_t)n_docs + 2), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(state, 0, sizeof(long long) * kSsWords, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(part, 0xFF, sizeof(int32_t) * (size_t)V, ctx->stream);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(((int64_t)V + 255) / 256);
  {
    KernelTimer kt(ctx, "select_hist", 4.0 * V);
    k_df_hist<<<blocks, 256, 0, ctx->stream>>>(df, V, hist, state);
  }
  {
    KernelTimer kt(ctx, "select_band", 8.0 * (double)n_docs);
    k_sel_band<<<1, kSelThreads, 0, ctx->stream>>>(hist, above, n_docs, L, region_start, state);
  }
  {
    KernelTimer kt(ctx, "select_collect", 4.0 * V);
    k_band_collect<<<blocks, 256, 0, ctx->stream>>>(df, V, state, keys);
  }
  const size_t smem = sizeof(unsigned long long) * kBandMax;
  if (resident_ctas(k_band_place, kSelThreads, smem) <= 0) return cudaErrorInvalidConfiguration;
  KernelTimer kt(ctx, "select_place");
  k_band_place<<<1, kSelThreads, smem, ctx->stream>>>(keys, state, idf, bf16, k, part, rnorm, rinv);
  return cudaGetLastError();
}

}  // namespace mrc
