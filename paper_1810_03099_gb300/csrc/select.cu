// select.cu -- reference selection on the device (Section IV, REGION selection).
//
// Terms are ranked by df descending, ids ascending within equal df; the selection takes the
// ranks [start, start + L) and partition p holds selection positions
// [floor(pL/k), floor((p+1)L/k)). With cnt[v] terms of df v, the terms of df v hold the ranks
// [#{df > v}, #{df > v} + cnt[v]), so only the df values whose rank range meets the selection
// matter: a contiguous band of values [v_lo, v_hi]. The device pass
//   1. histograms df (k_df_hist),
//   2. turns the histogram into above[v] = #{df > v} and finds start, L and the band (one
//      CTA, k_sel_band); the terms of df v hold the ranks [above[v], above[v - 1]),
//   3. places each band term in its df group's rank range (k_band_group, order within a
//      group arbitrary),
//   4. sorts each group by id (one CTA per group, k_group_sort), which gives every band
//      term its rank, and writes the partition of every selected term and its reference
//      weight by selection position,
//   5. sums the reference norms |R_p| (one CTA, k_ref_norms; each partition summed by one
//      thread in rank order, in double).
// A band of more than kBandMax terms is reported in the status word; the caller then runs the
// general pass (launch_select_general), which ranks any number of band terms:
//   6. compacts the band terms in id order (k_band_compact),
//   7. sorts them by df, descending, with a stable least-significant-digit radix sort on
//      v_hi - df, 8 bits a pass (k_radix_hist, k_radix_scan, k_radix_scatter): ids stay
//      ascending within each df, which is the ranking,
//   8. assigns partitions and reference weights by selection position (k_select_assign) and
//      sums the reference norms as step 5 does (k_ref_norms_wide).
// All three selections (Section IV) are a contiguous range of that one ranking: REGION the
// ranks [start, start + L); ALL every ranked term; DF1 the first L terms of df 1, which are the
// last ranks, in id order.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

constexpr int kSelThreads = 1024;
constexpr int kBandMax = 8192;  // band terms (and selection positions) held on the device
constexpr int kGroupThreads = 256;

// Selection state (int64 words): [0] start, [1] L, [2] v_lo, [3] v_hi, [4] rank of the
// band's first term, [5] band size, [6] status (0 ok, 1 band too large), [7] largest df.
enum { kSsStart = 0, kSsL, kSsVlo, kSsVhi, kSsRank0, kSsBand, kSsStatus, kSsMaxdf, kSsWords = 8 };

// df histogram. The small df values hold most of the vocabulary (Zipf), so their counts are
// first summed per CTA in shared memory (one global atomic per CTA and value); larger values go
// straight to global memory, once per group of equal values in a warp.
constexpr int kHistSmall = 1024;
__global__ void __launch_bounds__(1024) k_df_hist(const int32_t* __restrict__ df, int32_t V,
                                                  int32_t* __restrict__ hist, long long* __restrict__ state) {
  __shared__ int32_t s_hist[kHistSmall];
  __shared__ int32_t s_max[32];
  for (int x = threadIdx.x; x < kHistSmall; x += blockDim.x) s_hist[x] = 0;
  __syncthreads();
  int32_t dmax = 0;
  for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t - (int32_t)threadIdx.x < V; t += gridDim.x * blockDim.x) {
    const int32_t d = t < V ? df[t] : 0;
    if (d > 0 && d < kHistSmall) atomicAdd(&s_hist[d], 1);
    const int32_t big = d >= kHistSmall ? d : -1;  // the loop is warp-uniform: every lane matches
    const unsigned same = __match_any_sync(kFull, big);
    if (big >= 0 && (threadIdx.x & 31) == __ffs(same) - 1) atomicAdd(&hist[big], __popc(same));
    dmax = max(dmax, d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(kFull, dmax, o));
  if ((threadIdx.x & 31) == 0) s_max[threadIdx.x >> 5] = dmax;
  __syncthreads();
  for (int x = threadIdx.x; x < kHistSmall; x += blockDim.x)
    if (s_hist[x]) atomicAdd(&hist[x], s_hist[x]);
  if (threadIdx.x < 32) {
    dmax = threadIdx.x < (blockDim.x >> 5) ? s_max[threadIdx.x] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = max(dmax, __shfl_xor_sync(kFull, dmax, o));
    if (threadIdx.x == 0 && dmax > 0) atomicMax(&state[kSsMaxdf], (long long)dmax);
  }
}

// One CTA. above[v] = #{terms with df > v} for v in [0, maxdf]; then the selection and the
// band of df values whose ranks meet it.
__global__ void __launch_bounds__(kSelThreads, 1) k_sel_band(const int32_t* __restrict__ hist, int32_t* __restrict__ above,
                                                         int64_t n_docs, int64_t L, int64_t region_start,
                                                         int32_t mode, long long* __restrict__ state) {
  __shared__ long long part[kSelThreads];
  __shared__ long long s_lo, s_hi;
  const int64_t maxdf = state[kSsMaxdf];
  // values in descending order: thread i takes the contiguous run [hi_i - per, hi_i]
  const int64_t nv = maxdf;  // values 1..maxdf
  const int64_t per = (nv + kSelThreads - 1) / kSelThreads;
  const int64_t v_top = maxdf - (int64_t)threadIdx.x * per;  // this thread's largest value
  long long sum = 0;
#pragma unroll 8
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
  int64_t start = 0, end = ranked;  // ALL: every ranked term
  if (mode == MRC_SELECT_REGION) {
    start = region_start;
    if (start < 0) {
      const int64_t vcap = n_docs / 100;  // first rank whose df <= N / 100
      start = vcap >= maxdf ? 0 : (vcap >= 1 ? above[vcap] : ranked);
    }
    start = min(start, ranked);
    end = min(start + L, ranked);
  } else if (mode == MRC_SELECT_DF1) {  // the terms of df 1 hold the last ranks, in id order
    start = maxdf >= 1 ? above[1] : ranked;
    end = min(start + L, ranked);
  }
#pragma unroll 4
  for (int64_t q = 0; q < per; ++q) {
    const int64_t v = v_top - q;
    if (v >= 1) {
      const int64_t lo_rank = above[v], cnt = (int64_t)above[v - 1] - above[v];
      if (cnt > 0 && lo_rank < end && lo_rank + cnt > start) {
        atomicMin(&s_lo, (long long)v);
        atomicMax(&s_hi, (long long)v);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long v_lo = s_hi >= 0 ? s_lo : 1, v_hi = s_hi;  // v_hi = -1: empty selection
    const long long rank0 = s_hi >= 0 ? above[s_hi] : 0;
    const long long nb = s_hi >= 0 ? (long long)above[v_lo - 1] - rank0 : 0;
    state[kSsStart] = start;
    state[kSsL] = end - start;
    state[kSsVlo] = v_lo;
    state[kSsVhi] = v_hi;
    state[kSsRank0] = rank0;
    state[kSsBand] = nb;
    state[kSsStatus] = nb > kBandMax ? 1 : 0;
  }
}

// Each band term goes to a free slot of its df group's band range [above[d], above[d - 1]) -
// rank0 (the group's histogram count is used up as the slot counter).
__global__ void k_band_group(const int32_t* __restrict__ df, int32_t V, const int32_t* __restrict__ above,
                             int32_t* __restrict__ hist, const long long* __restrict__ state,
                             uint32_t* __restrict__ ids) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= V || state[kSsStatus] != 0) return;
  const int32_t d = df[t];
  if (d < state[kSsVlo] || d > state[kSsVhi]) return;
  const int32_t slot = atomicSub(&hist[d], 1) - 1;
  ids[above[d] - state[kSsRank0] + slot] = (uint32_t)t;
}

// One CTA per df group of the band (grid-stride): sorts the group's ids ascending in shared
// memory (bitonic), which completes the ranking; writes the partition of each selected term
// (part holds -1 for every term on entry) and its reference weight at its selection
// position. idf NULL: count weighting (r = 1).
__global__ void __launch_bounds__(kGroupThreads) k_group_sort(const int32_t* __restrict__ above, long long* __restrict__ state,
                                                            const uint32_t* __restrict__ ids, const float* __restrict__ idf,
                                                            int32_t bf16, int32_t k, int32_t* __restrict__ part,
                                                            float* __restrict__ rsel) {
  extern __shared__ uint32_t sid[];  // [next power of two >= group size]
  if (state[kSsStatus] != 0 || state[kSsVhi] < 0) return;
  const long long v_lo = state[kSsVlo], v_hi = state[kSsVhi], rank0 = state[kSsRank0];
  const long long start = state[kSsStart], L = state[kSsL];
  for (long long v = v_lo + blockIdx.x; v <= v_hi; v += gridDim.x) {
    const int32_t g0 = above[v], m = above[v - 1] - g0;  // ranks [g0, g0 + m)
    if (m <= 0 || g0 + m <= start || g0 >= start + L) continue;  // block-uniform
    int n2 = 1;
    while (n2 < m) n2 <<= 1;
    const uint32_t* gi = ids + (g0 - rank0);
    __syncthreads();  // the previous group's reads of sid are done
    for (int x = threadIdx.x; x < n2; x += kGroupThreads) sid[x] = x < m ? gi[x] : 0xFFFFFFFFu;
    __syncthreads();
    for (int kk = 2; kk <= n2; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int x = threadIdx.x; x < n2; x += kGroupThreads) {
          const int y = x ^ j;
          if (y > x) {
            const uint32_t a = sid[x], b = sid[y];
            if ((a > b) == ((x & kk) == 0)) {
              sid[x] = b;
              sid[y] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int x = threadIdx.x; x < m; x += kGroupThreads) {
      const long long pos = (long long)g0 + x - start;  // selection position
      if (pos >= 0 && pos < L) {
        const uint32_t t = sid[x];
        part[t] = (int32_t)(((pos + 1) * k - 1) / L);
        float r = 1.f;
        if (idf) r = bf16 ? __bfloat162float(__float2bfloat16_rn(idf[t])) : idf[t];
        rsel[pos] = r;
      }
    }
  }
}

// One CTA: partition q holds selection positions [floor(qL/k), floor((q+1)L/k)); |R_q|^2 is
// summed by one thread in rank order, in double. With rinv16, the same norms of the
// bfloat16-rounded weights (the precision form's compare operands) as well.
__global__ void __launch_bounds__(kSelThreads) k_ref_norms(const long long* __restrict__ state,
                                                         const float* __restrict__ rsel, int32_t k,
                                                         double* __restrict__ rnorm, float* __restrict__ rinv,
                                                         float* __restrict__ rinv16) {
  __shared__ float sr[kBandMax];
  if (state[kSsStatus] != 0) return;
  const long long L = state[kSsVhi] < 0 ? 0 : state[kSsL];
  for (long long x = threadIdx.x; x < L; x += kSelThreads) sr[x] = rsel[x];
  __syncthreads();
  for (int q = threadIdx.x; q < k; q += kSelThreads) {
    double s = 0.0;
    const long long p0 = q * L / k, p1 = (q + 1) * L / k;
    for (long long pos = p0; pos < p1; ++pos) {
      const double r = (double)sr[pos];
      s += r * r;
    }
    const double nr = sqrt(s);
    rnorm[q] = nr;
    rinv[q] = nr > 0.0 ? (float)(1.0 / nr) : 0.f;
    if (rinv16) {
      double s16 = 0.0;
      for (long long pos = p0; pos < p1; ++pos) {
        const double r = (double)__bfloat162float(__float2bfloat16_rn(sr[pos]));
        s16 += r * r;
      }
      rinv16[q] = s16 > 0.0 ? (float)(1.0 / sqrt(s16)) : 0.f;
    }
  }
}

// ---------------------------------------------------------------- general pass (any band size)
constexpr int kRadixItems = 1024;  // items per CTA of the compaction and the radix passes
constexpr int kRadixBits = 8;
constexpr int kRadixDigits = 1 << kRadixBits;

__device__ __forceinline__ bool general_needed(const long long* state) { return state[kSsStatus] == 1; }

// Radix passes the band's keys v_hi - df need (0 when the band is one df value).
__device__ __forceinline__ int radix_passes(const long long* state) {
  const long long span = state[kSsVhi] - state[kSsVlo];
  int bits = 0;
  while (bits < 62 && (span >> bits) != 0) ++bits;
  return (bits + kRadixBits - 1) / kRadixBits;
}

// Step 6a: per CTA of kRadixItems terms, the number of band terms.
__global__ void __launch_bounds__(kRadixItems) k_band_count(const int32_t* __restrict__ df, int32_t V,
                                                            const long long* __restrict__ state,
                                                            int32_t* __restrict__ bcount) {
  __shared__ int32_t s_n;
  if (!general_needed(state)) return;
  const long long v_lo = state[kSsVlo], v_hi = state[kSsVhi];
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * kRadixItems + threadIdx.x;
  const bool in = t < V && df[t] >= v_lo && df[t] <= v_hi;
  const unsigned b = __ballot_sync(kFull, in);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(&s_n, __popc(b));
  __syncthreads();
  if (threadIdx.x == 0) bcount[blockIdx.x] = s_n;
}

// Exclusive scan of n int32 counts in place by one CTA (thread i sums a contiguous run, the runs
// are scanned by one warp, then written back); the total goes to *total.
__global__ void __launch_bounds__(kSelThreads, 1) k_scan_counts(int32_t* __restrict__ c, int64_t n,
                                                                const long long* __restrict__ state,
                                                                long long* __restrict__ total) {
  __shared__ long long part[kSelThreads];
  if (!general_needed(state)) return;
  const int64_t per = (n + kSelThreads - 1) / kSelThreads;
  const int64_t a = min(n, (int64_t)threadIdx.x * per), b = min(n, a + per);
  long long sum = 0;
  for (int64_t x = a; x < b; ++x) sum += c[x];
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x < 32) {
    long long carry = 0;
    for (int q = 0; q < kSelThreads; q += 32) {
      const long long x = part[q + threadIdx.x];
      long long incl = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, incl, o);
        if ((int)threadIdx.x >= o) incl += y;
      }
      part[q + threadIdx.x] = carry + incl - x;
      carry += __shfl_sync(kFull, incl, 31);
    }
    if (threadIdx.x == 0 && total) *total = carry;
  }
  __syncthreads();
  long long run = part[threadIdx.x];
  for (int64_t x = a; x < b; ++x) {
    const int32_t v = c[x];
    c[x] = (int32_t)run;
    run += v;
  }
}

// Step 6b: the band terms in id order: ids[pos] = t, keys[pos] = v_hi - df[t].
__global__ void __launch_bounds__(kRadixItems) k_band_compact(const int32_t* __restrict__ df, int32_t V,
                                                              const long long* __restrict__ state,
                                                              const int32_t* __restrict__ boff,
                                                              uint32_t* __restrict__ ids, uint32_t* __restrict__ keys) {
  __shared__ int32_t s_warp[kRadixItems / 32];
  if (!general_needed(state)) return;
  const long long v_lo = state[kSsVlo], v_hi = state[kSsVhi];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * kRadixItems + threadIdx.x;
  const int32_t d = t < V ? df[t] : 0;
  const bool in = t < V && d >= v_lo && d <= v_hi;
  const unsigned b = __ballot_sync(kFull, in);
  if (lane == 0) s_warp[warp] = __popc(b);
  __syncthreads();
  if (warp == 0) {  // exclusive scan of the 32 warp counts
    const int x = s_warp[lane];
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += y;
    }
    s_warp[lane] = incl - x;
  }
  __syncthreads();
  if (in) {
    const int64_t pos = (int64_t)boff[blockIdx.x] + s_warp[warp] + __popc(b & ((1u << lane) - 1u));
    if (pos < V) {  // a guard: the band holds at most V terms
      ids[pos] = (uint32_t)t;
      keys[pos] = (uint32_t)(v_hi - d);
    }
  }
}

// Step 7a: digit counts of one radix pass, digit-major: cnt[digit * nblk + block].
__global__ void __launch_bounds__(kRadixItems) k_radix_hist(const uint32_t* __restrict__ keys,
                                                            const long long* __restrict__ state,
                                                            const long long* __restrict__ nband, int pass,
                                                            int32_t* __restrict__ cnt, int64_t nblk) {
  __shared__ int32_t s_cnt[kRadixDigits];
  if (!general_needed(state) || pass >= radix_passes(state)) return;
  const int64_t n = *nband;  // CTAs past the band's end write zero counts (the scan reads them all)
  for (int x = threadIdx.x; x < kRadixDigits; x += kRadixItems) s_cnt[x] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kRadixItems + threadIdx.x;
  if (i < n) atomicAdd(&s_cnt[(keys[i] >> (kRadixBits * pass)) & (kRadixDigits - 1)], 1);
  __syncthreads();
  for (int x = threadIdx.x; x < kRadixDigits; x += kRadixItems) cnt[(int64_t)x * nblk + blockIdx.x] = s_cnt[x];
}

// Step 7b: one stable radix pass. An item's place is the digit's offset for its block, plus the
// items of the same digit in earlier warps of the block, plus those in earlier lanes of its warp.
__global__ void __launch_bounds__(kRadixItems) k_radix_scatter(const uint32_t* __restrict__ keys,
                                                               const uint32_t* __restrict__ ids,
                                                               const long long* __restrict__ state,
                                                               const long long* __restrict__ nband, int pass,
                                                               const int32_t* __restrict__ off, int64_t nblk,
                                                               uint32_t* __restrict__ keys_out,
                                                               uint32_t* __restrict__ ids_out) {
  __shared__ int32_t s_wc[kRadixItems / 32][kRadixDigits];  // per warp and digit: count, then prefix
  if (!general_needed(state) || pass >= radix_passes(state)) return;
  const int64_t n = *nband;
  if ((int64_t)blockIdx.x * kRadixItems >= n) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int x = threadIdx.x; x < (kRadixItems / 32) * kRadixDigits; x += kRadixItems) (&s_wc[0][0])[x] = 0;
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * kRadixItems + threadIdx.x;
  const bool valid = i < n;
  const uint32_t key = valid ? keys[i] : 0u;
  const uint32_t id = valid ? ids[i] : 0u;
  const int dg = valid ? (int)((key >> (kRadixBits * pass)) & (kRadixDigits - 1)) : kRadixDigits;  // sentinel
  const unsigned peers = __match_any_sync(kFull, dg);
  const int in_warp = __popc(peers & ((1u << lane) - 1u));
  if (valid && lane == __ffs(peers) - 1) s_wc[warp][dg] = __popc(peers);
  __syncthreads();
  for (int d = threadIdx.x; d < kRadixDigits; d += kRadixItems) {  // exclusive scan over the warps
    int run = 0;
    for (int w = 0; w < kRadixItems / 32; ++w) {
      const int c = s_wc[w][d];
      s_wc[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  if (valid) {
    const int64_t pos = (int64_t)off[(int64_t)dg * nblk + blockIdx.x] + s_wc[warp][dg] + in_warp;
    if (pos >= 0 && pos < n) {  // always so when the counts are consistent; a guard, not a branch taken
      keys_out[pos] = key;
      ids_out[pos] = id;
    }
  }
}

// Step 8a: the sorted band terms hold the ranks rank0, rank0 + 1, ...; those in [start, start + L)
// get their partition and, at their selection position, their reference weight. ids_sorted is
// buffer 0 or 1 of the ping-pong by the number of passes.
__global__ void k_select_assign(const uint32_t* __restrict__ ids0, const uint32_t* __restrict__ ids1, int32_t V,
                                const long long* __restrict__ state, const long long* __restrict__ nband,
                                const float* __restrict__ idf, int32_t bf16, int32_t k, int32_t* __restrict__ part,
                                float* __restrict__ rsel) {
  if (!general_needed(state)) return;
  const uint32_t* ids = (radix_passes(state) & 1) ? ids1 : ids0;
  const int64_t n = *nband;
  const long long rank0 = state[kSsRank0], start = state[kSsStart], L = state[kSsL];
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const long long pos = rank0 + r - start;
    if (pos < 0 || pos >= L) continue;
    const uint32_t t = ids[r];
    if (t >= (uint32_t)V) continue;  // a guard: every sorted id is a term
    part[t] = (int32_t)(((pos + 1) * k - 1) / L);
    float w = 1.f;
    if (idf) w = bf16 ? __bfloat162float(__float2bfloat16_rn(idf[t])) : idf[t];
    rsel[pos] = w;
  }
}

// Step 8b: k_ref_norms for a selection of any length (the weights read from global memory).
__global__ void __launch_bounds__(kSelThreads) k_ref_norms_wide(const long long* __restrict__ state,
                                                              const float* __restrict__ rsel, int32_t k,
                                                              double* __restrict__ rnorm, float* __restrict__ rinv,
                                                              float* __restrict__ rinv16) {
  if (!general_needed(state)) return;
  const long long L = state[kSsVhi] < 0 ? 0 : state[kSsL];
  for (int q = threadIdx.x; q < k; q += kSelThreads) {
    double s = 0.0, s16 = 0.0;
    const long long p0 = q * L / k, p1 = (q + 1) * L / k;
    for (long long pos = p0; pos < p1; ++pos) {
      const float w = rsel[pos];
      const double r = (double)w;
      s += r * r;
      const double r16 = (double)__bfloat162float(__float2bfloat16_rn(w));
      s16 += r16 * r16;
    }
    const double nr = sqrt(s);
    rnorm[q] = nr;
    rinv[q] = nr > 0.0 ? (float)(1.0 / nr) : 0.f;
    if (rinv16) rinv16[q] = s16 > 0.0 ? (float)(1.0 / sqrt(s16)) : 0.f;
  }
}

}  // namespace

int64_t device_selection_words() { return kSsWords; }

cudaError_t launch_select_region(mrc_ctx* ctx, const int32_t* df, int32_t V, int64_t n_docs, int64_t L,
                                 int64_t region_start, int32_t mode, const float* idf, int32_t bf16, int32_t k,
                                 int32_t* hist,
                                 int32_t* above, long long* state, unsigned long long* keys, int32_t* part,
                                 double* rnorm, float* rinv, float* rinv16) {
  if (V <= 0 || k <= 0) return cudaErrorInvalidValue;
  // keys: 64 KB of scratch = band ids [kBandMax] + reference weights by position [kBandMax]
  uint32_t* ids = reinterpret_cast<uint32_t*>(keys);
  float* rsel = reinterpret_cast<float*>(ids + kBandMax);
  cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(int32_t) * ((size_t)n_docs + 2), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(state, 0, sizeof(long long) * kSsWords, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(part, 0xFF, sizeof(int32_t) * (size_t)V, ctx->stream);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)(((int64_t)V + 255) / 256);
  {
    KernelTimer kt(ctx, "select_hist", 4.0 * V);
    const int64_t hb = std::min<int64_t>(((int64_t)V + 1023) / 1024, 2 * (int64_t)ctx->num_sms);
    k_df_hist<<<(unsigned)hb, 1024, 0, ctx->stream>>>(df, V, hist, state);
  }
  {
    KernelTimer kt(ctx, "select_band", 8.0 * (double)n_docs);
    k_sel_band<<<1, kSelThreads, 0, ctx->stream>>>(hist, above, n_docs, L, region_start, mode, state);
  }
  {
    KernelTimer kt(ctx, "select_group", 4.0 * V);
    k_band_group<<<blocks, 256, 0, ctx->stream>>>(df, V, above, hist, state, ids);
  }
  const size_t smem = sizeof(uint32_t) * kBandMax;
  if (resident_ctas(k_group_sort, kGroupThreads, smem) <= 0) return cudaErrorInvalidConfiguration;
  {
    KernelTimer kt(ctx, "select_sort");
    k_group_sort<<<(unsigned)(2 * ctx->num_sms), kGroupThreads, smem, ctx->stream>>>(above, state, ids, idf, bf16,
                                                                                       k, part, rsel);
  }
  KernelTimer kt(ctx, "select_norms");
  k_ref_norms<<<1, kSelThreads, 0, ctx->stream>>>(state, rsel, k, rnorm, rinv, rinv16);
  return cudaGetLastError();
}

size_t select_general_bytes(int32_t V) {
  const size_t nblk = ((size_t)std::max(V, 1) + kRadixItems - 1) / kRadixItems;
  return 5 * 4 * (size_t)std::max(V, 1) + 4 * (kRadixDigits + 1) * nblk + 256;
}

cudaError_t launch_select_general(mrc_ctx* ctx, const int32_t* df, int32_t V, const float* idf, int32_t bf16,
                                  int32_t k, long long* state, void* scratch, int32_t* part, double* rnorm,
                                  float* rinv, float* rinv16) {
  if (V <= 0 || k <= 0) return cudaErrorInvalidValue;
  const int64_t nblk = ((int64_t)V + kRadixItems - 1) / kRadixItems;
  // scratch: ids and keys twice [V] (ping-pong), reference weights [V], digit counts
  // [256 * nblk], per-CTA band counts [nblk], the band size
  uint32_t* ids0 = static_cast<uint32_t*>(scratch);
  uint32_t* keys0 = ids0 + V;
  uint32_t* ids1 = keys0 + V;
  uint32_t* keys1 = ids1 + V;
  float* rsel = reinterpret_cast<float*>(keys1 + V);
  int32_t* cnt = reinterpret_cast<int32_t*>(rsel + V);
  int32_t* bcount = cnt + kRadixDigits * nblk;
  long long* nband = reinterpret_cast<long long*>((reinterpret_cast<uintptr_t>(bcount + nblk) + 7) & ~uintptr_t(7));
  KernelTimer kt(ctx, "select_general", 24.0 * V);
  const unsigned g = (unsigned)nblk;
  k_band_count<<<g, kRadixItems, 0, ctx->stream>>>(df, V, state, bcount);
  k_scan_counts<<<1, kSelThreads, 0, ctx->stream>>>(bcount, nblk, state, nband);
  k_band_compact<<<g, kRadixItems, 0, ctx->stream>>>(df, V, state, bcount, ids0, keys0);
  // df < 2^31: at most four passes of 8 bits; each returns at once past the passes the band needs
  for (int pass = 0; pass < 4; ++pass) {
    const uint32_t* ki = (pass & 1) ? keys1 : keys0;
    const uint32_t* ii = (pass & 1) ? ids1 : ids0;
    uint32_t* ko = (pass & 1) ? keys0 : keys1;
    uint32_t* io = (pass & 1) ? ids0 : ids1;
    k_radix_hist<<<g, kRadixItems, 0, ctx->stream>>>(ki, state, nband, pass, cnt, nblk);
    k_scan_counts<<<1, kSelThreads, 0, ctx->stream>>>(cnt, kRadixDigits * nblk, state, nullptr);
    k_radix_scatter<<<g, kRadixItems, 0, ctx->stream>>>(ki, ii, state, nband, pass, cnt, nblk, ko, io);
  }
  k_select_assign<<<(unsigned)std::min<int64_t>(nblk * 4, 8 * ctx->num_sms), 256, 0, ctx->stream>>>(
      ids0, ids1, V, state, nband, idf, bf16, k, part, rsel);
  k_ref_norms_wide<<<1, kSelThreads, 0, ctx->stream>>>(state, rsel, k, rnorm, rinv, rinv16);
  return cudaGetLastError();
}

}  // namespace mrc
