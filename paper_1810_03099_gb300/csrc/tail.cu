// tail.cu -- sparse completion of the exact cosine, and FP32 rescoring of candidates.
//
// Exact cosine (Eq. 1) of unit TF-IDF vectors splits over the vocabulary:
// cos(i, j) = sum over frequent ("head") terms + sum over the other terms.
// The head sums come from a single-fp16 tensor-core GEMM as an fp16 matrix
// H16 (an approximation with a proven error bound). This kernel adds the
// remaining terms from postings lists, selects candidates against the
// threshold lowered by that bound, and recomputes each candidate's head
// exactly before the final test (see k_cosine_tail).
//
// Rescoring (reduced-precision forms): each candidate pair found with a
// lowered threshold in FP8 or FP16 is recomputed as an FP32 dot product of the
// two FP32 unit signatures and kept iff it reaches tau.
#include <cuda_fp16.h>

#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

constexpr int kTailThreads = 512;
constexpr int kTailWarps = kTailThreads / 32;
constexpr int kMaxWindow = 32768;                      // columns per work item (128 KB of accumulators)
constexpr float kTailFix = 1073741824.0f;              // 2^30: tail sums stay below 2^31
constexpr float kTailInv = 1.0f / 1073741824.0f;
constexpr int kSortMax = 4096;                         // postings per sorted group
constexpr int kSortThreads = 512;

// Sorts the postings of each group of consecutive tail terms by (term, document) with a
// bitonic sort of 64-bit keys in shared memory: key = term-in-group << 44 | doc << 12 |
// original slot. Segments keep their places, so each term's postings come out sorted by
// document. Then records row_pos[offsets[doc] + r] = sorted position of that posting.
__global__ void __launch_bounds__(kSortThreads) k_sort_postings(
    const int64_t* __restrict__ cstart, const int32_t* __restrict__ gterm, int32_t n_groups,
    const int32_t* __restrict__ post_doc, const float* __restrict__ post_w, const int32_t* __restrict__ post_r,
    const int64_t* __restrict__ doc_off, int32_t* __restrict__ sdoc, float* __restrict__ sw,
    int64_t* __restrict__ row_pos) {
  __shared__ unsigned long long keys[kSortMax];
  __shared__ int32_t tst[kSortMax / 2 + 1];
  for (int32_t g = blockIdx.x; g < n_groups; g += gridDim.x) {
    const int32_t t0 = gterm[g], t1 = gterm[g + 1];
    const int32_t nterm = t1 - t0;
    const int64_t p0 = cstart[t0];
    const int32_t P = (int32_t)(cstart[t1] - p0);
    __syncthreads();
    for (int x = threadIdx.x; x <= nterm; x += kSortThreads) tst[x] = (int32_t)(cstart[t0 + x] - p0);
    int n2 = 2;
    while (n2 < P) n2 <<= 1;
    __syncthreads();
    for (int x = threadIdx.x; x < n2; x += kSortThreads) {
      unsigned long long k = ~0ull;
      if (x < P) {
        int a = 0, b = nterm;  // last term start <= x
        while (b - a > 1) {
          const int m = (a + b) >> 1;
          if (tst[m] <= x) a = m; else b = m;
        }
        k = ((unsigned long long)a << 44) | ((unsigned long long)(uint32_t)post_doc[p0 + x] << 12) |
            (unsigned long long)x;
      }
      keys[x] = k;
    }
    __syncthreads();
    for (int k = 2; k <= n2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int x = threadIdx.x; x < n2; x += kSortThreads) {
          const int y = x ^ j;
          if (y > x) {
            const unsigned long long a = keys[x], b = keys[y];
            if ((a > b) == ((x & k) == 0)) {
              keys[x] = b;
              keys[y] = a;
            }
          }
        }
        __syncthreads();
      }
    }
    for (int x = threadIdx.x; x < P; x += kSortThreads) {
      const int64_t src = p0 + (int64_t)(keys[x] & 4095ull);
      const int64_t dst = p0 + x;
      const int32_t d = post_doc[src];
      sdoc[dst] = d;
      sw[dst] = post_w[src];
      row_pos[doc_off[d] + post_r[src]] = dst;
    }
  }
}

// Exact score of one candidate pair (i, j): the head part recomputed from the split head rows
// (w = hi + lo / 4096 is exact in FP32: 22 significant bits), FP32 products summed by the
// warp in a fixed order, plus the exact tail sum. Every lane returns the same value.
__device__ __forceinline__ float exact_head(const __half* __restrict__ hhi, const __half* __restrict__ hlo,
                                            int32_t kd, int64_t i, int64_t j, int lane) {
  const __half* ai = hhi + i * kd;
  const __half* bi = hlo + i * kd;
  const __half* aj = hhi + j * kd;
  const __half* bj = hlo + j * kd;
  float s = 0.f;
  for (int32_t c = 8 * lane; c < kd; c += 256) {
    const uint4 xa = __ldg(reinterpret_cast<const uint4*>(ai + c));
    const uint4 xb = __ldg(reinterpret_cast<const uint4*>(bi + c));
    const uint4 ya = __ldg(reinterpret_cast<const uint4*>(aj + c));
    const uint4 yb = __ldg(reinterpret_cast<const uint4*>(bj + c));
    const __half2* pa = reinterpret_cast<const __half2*>(&xa);
    const __half2* pb = reinterpret_cast<const __half2*>(&xb);
    const __half2* qa = reinterpret_cast<const __half2*>(&ya);
    const __half2* qb = reinterpret_cast<const __half2*>(&yb);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 h1 = __half22float2(pa[u]), l1 = __half22float2(pb[u]);
      const float2 h2 = __half22float2(qa[u]), l2 = __half22float2(qb[u]);
      const float x0 = fmaf(l1.x, 1.0f / kSplitLoScale, h1.x), x1 = fmaf(l1.y, 1.0f / kSplitLoScale, h1.y);
      const float y0 = fmaf(l2.x, 1.0f / kSplitLoScale, h2.x), y1 = fmaf(l2.y, 1.0f / kSplitLoScale, h2.y);
      s = fmaf(x0, y0, s);
      s = fmaf(x1, y1, s);
    }
  }
  return warp_sum(s);
}

// One CTA per (row i, column window) work item. The tail sums accumulate in a shared-memory
// row of 2^-30 fixed-point integers (each product is < 1: rounding <= 2^-31; integer sums do
// not depend on the order in which threads add them):
//  1. acc[j] = 0 over the window;
//  2. for every tail term t of document i, the postings after i's own position in t's
//     sorted list are exactly the documents j > i sharing t: acc[j] += w_it * w_jt. Each
//     warp takes 32 of the row's terms at a time (one lane per term holds its metadata),
//     flattens their postings into one index range (warp prefix sum; a shuffle binary
//     search maps an index back to its term) and walks it with four loads per lane in
//     flight, so short lists do not leave lanes idle;
//  3. scan: H16[i][j] (the fp16 head score from the tensor cores, eight columns per 16-byte
//     load) + tail >= tau - delta marks a candidate, where delta bounds the head's error;
//     each candidate's head is recomputed exactly (exact_head) and the pair is kept iff
//     head + tail >= tau.
__global__ void __launch_bounds__(kTailThreads) k_cosine_tail(
    int64_t n, const __half* __restrict__ H, int64_t ldh, const int64_t* __restrict__ row_off,
    const int32_t* __restrict__ row_cnt, const int32_t* __restrict__ row_term, const float* __restrict__ row_w,
    const int64_t* __restrict__ row_pos, const int64_t* __restrict__ tail_start, const int32_t* __restrict__ post_cnt,
    const int32_t* __restrict__ sdoc, const float* __restrict__ sw, const __half* __restrict__ hhi,
    const __half* __restrict__ hlo, int32_t kd, float tau, float delta, mrc_pair* pairs,
    unsigned long long* count, int64_t capacity, int64_t window, int64_t n_windows, int64_t n_items) {
  extern __shared__ int32_t acc[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float cand_tau = tau - delta;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int64_t i = item / n_windows;
    const int64_t w = item % n_windows;
    const int64_t base = w * window;  // a multiple of 8 (window is)
    const int64_t lo = max(i + 1, base), hi = min(n, base + window);
    if (lo >= hi) continue;  // block-uniform
    __syncthreads();  // the previous item's scan is done with acc
    const int64_t a0 = (lo - base) & ~7ll, a1 = hi - base;  // accumulator range touched, 8-aligned start
    for (int64_t x = a0 + 4 * threadIdx.x; x < a1; x += 4 * kTailThreads)
      *reinterpret_cast<int4*>(acc + x) = make_int4(0, 0, 0, 0);
    __syncthreads();
    const int32_t nt = row_cnt[i];
    const int64_t ro = row_off[i];
    for (int32_t b0 = warp; b0 < nt; b0 += 32 * kTailWarps) {
      // lane l holds term b0 + 16 l: its remaining postings [st, st + cnt) (documents > i)
      const int32_t r = b0 + kTailWarps * lane;
      int64_t st = 0;
      int32_t cnt = 0;
      float wi = 0.f;
      if (r < nt) {
        const int32_t t = row_term[ro + r];
        wi = row_w[ro + r];
        st = row_pos[ro + r] + 1;
        cnt = (int32_t)(tail_start[t] + post_cnt[t] - st);
      }
      // flatten the batch: posting f of the batch belongs to the last lane q with excl_q <= f
      int32_t incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
      }
      const int32_t excl = incl - cnt;
      const int32_t total = __shfl_sync(kFull, incl, 31);
      for (int32_t f0 = 0; f0 < total; f0 += 4 * 32) {
        int32_t jd[4];
        float wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int32_t f = f0 + 32 * u + lane;
          int q = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int cand = q + step;
            const int32_t ex = __shfl_sync(kFull, excl, cand & 31);
            if (cand < 32 && ex <= f) q = cand;
          }
          const int64_t sq = __shfl_sync(kFull, st, q);
          const int32_t eq = __shfl_sync(kFull, excl, q);
          const float wq = __shfl_sync(kFull, wi, q);
          jd[u] = -1;
          wv[u] = 0.f;
          if (f < total) {
            const int64_t x = sq + (f - eq);
            jd[u] = sdoc[x];
            wv[u] = wq * sw[x];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (jd[u] >= lo && jd[u] < hi) atomicAdd(&acc[jd[u] - base], __float2int_rn(wv[u] * kTailFix));
      }
    }
    __syncthreads();
    // scan: each lane takes eight consecutive columns (one 16-byte load of H16, in the row's
    // ldh >= round8(n) padding at the end, so never past the row)
    const __half* hrow = H + i * ldh;
    for (int64_t g0 = base + a0 + 8 * (int64_t)warp * 32; g0 < hi; g0 += 8 * kTailThreads) {
      const int64_t g = g0 + 8 * lane;
      uint32_t mask = 0;
      float sv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
      if (g < hi) {
        const uint4 raw = __ldcs(reinterpret_cast<const uint4*>(hrow + g));
        const __half2* h2 = reinterpret_cast<const __half2*>(&raw);
        const int4 t0 = *reinterpret_cast<const int4*>(acc + (g - base));
        const int4 t1 = *reinterpret_cast<const int4*>(acc + (g - base) + 4);
        const int32_t tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 hf = __half22float2(h2[u]);
          sv[2 * u] = (float)tv[2 * u] * kTailInv;
          sv[2 * u + 1] = (float)tv[2 * u + 1] * kTailInv;
          const int64_t ja = g + 2 * u, jb = ja + 1;
          if (ja >= lo && ja < hi && hf.x + sv[2 * u] >= cand_tau) mask |= 1u << (2 * u);
          if (jb >= lo && jb < hi && hf.y + sv[2 * u + 1] >= cand_tau) mask |= 1u << (2 * u + 1);
        }
      }
      unsigned todo = __ballot_sync(kFull, mask != 0);
      while (todo) {  // rare: candidates of one lane at a time, the whole warp per candidate
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        uint32_t m = __shfl_sync(kFull, mask, src);
        const int64_t gs = __shfl_sync(kFull, g, src);
        while (m) {
          const int e = __ffs(m) - 1;
          m &= m - 1;
          const int64_t j = gs + e;
          float tail = 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float y = __shfl_sync(kFull, sv[u], src);
            if (u == e) tail = y;
          }
          const float s = exact_head(hhi, hlo, kd, i, j, lane) + tail;
          if (lane == 0 && s >= tau) {
            const unsigned long long at = atomicAdd(count, 1ull);
            if (at < (unsigned long long)capacity) {
              mrc_pair pr;
              pr.i = (int32_t)i;
              pr.j = (int32_t)j;
              pr.score = s;
              pairs[at] = pr;
            }
          }
        }
      }
    }
  }
}

__global__ void k_rescore(const mrc_pair* __restrict__ cand, const unsigned long long* n_cand, int64_t cand_cap,
                          const float* __restrict__ qunit, const float* __restrict__ xunit, int32_t k, float tau,
                          mrc_pair* pairs, unsigned long long* count, int64_t capacity) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t nc0 = (int64_t)*n_cand;
  const int64_t nc = nc0 < cand_cap ? nc0 : cand_cap;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nc; c += nwarps) {
    const mrc_pair pc = cand[c];
    const float* qa = qunit + (int64_t)pc.i * k;
    const float* xb = xunit + (int64_t)pc.j * k;
    float s = 0.f;
    for (int q = lane; q < k; q += 32) s = fmaf(qa[q], xb[q], s);
    s = warp_sum(s);
    if (lane == 0 && s >= tau) {
      const unsigned long long at = atomicAdd(count, 1ull);
      if (at < (unsigned long long)capacity) {
        mrc_pair pr = pc;
        pr.score = s;
        pairs[at] = pr;
      }
    }
  }
}

}  // namespace

cudaError_t launch_sort_postings(mrc_ctx* ctx, const int64_t* cstart, const int32_t* gterm, int32_t n_groups,
                                 const int32_t* post_doc, const float* post_w, const int32_t* post_r,
                                 const int64_t* doc_off, int32_t* sdoc, float* sw, int64_t* row_pos) {
  if (n_groups <= 0) return cudaSuccess;
  int grid = ctx->num_sms * 3;
  if (n_groups < grid) grid = n_groups;
  cudaEvent_t ev = nullptr;
  timing_begin(ctx, "sort_postings", 0.0, 0.0, &ev);
  k_sort_postings<<<grid, kSortThreads, 0, ctx->stream>>>(cstart, gterm, n_groups, post_doc, post_w, post_r, doc_off,
                                                           sdoc, sw, row_pos);
  timing_end(ctx, ev);
  return cudaGetLastError();
}

cudaError_t launch_cosine_tail(mrc_ctx* ctx, int64_t n, const void* H16, int64_t ldh, const int64_t* row_off,
                               const int32_t* row_cnt, const int32_t* row_term, const float* row_w,
                               const int64_t* row_pos, const int64_t* tail_start, const int32_t* post_cnt,
                               const int32_t* sdoc, const float* sw, const void* head_hi, const void* head_lo,
                               int32_t kd, float tau, float delta, mrc_pair* pairs, unsigned long long* count,
                               int64_t capacity, double work_pairs) {
  if (n <= 1) return cudaSuccess;
  if ((ldh & 7) || ldh < (n + 7) / 8 * 8 || (kd & 63) || kd <= 0) return cudaErrorInvalidValue;
  const int64_t n8 = (n + 7) / 8 * 8;
  const int64_t window = n8 < kMaxWindow ? n8 : kMaxWindow;  // a multiple of 8
  const int64_t n_windows = (n + window - 1) / window;
  const int64_t n_items = n * n_windows;
  const size_t smem = sizeof(int32_t) * (size_t)window;
  cudaError_t e = cudaFuncSetAttribute(k_cosine_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cosine_tail, kTailThreads, smem);
  int64_t grid = (int64_t)ctx->num_sms * (per_sm > 0 ? per_sm : 1);
  if (n_items < grid) grid = n_items;
  cudaEvent_t ev = nullptr;
  // algorithmic bytes: the upper triangle of the fp16 head scores read once; flops: 2 per
  // tail posting product
  timing_begin(ctx, "cosine_tail", 2.0 * (double)n * (double)(n - 1) / 2.0, 2.0 * work_pairs, &ev);
  k_cosine_tail<<<(unsigned)grid, kTailThreads, smem, ctx->stream>>>(
      n, reinterpret_cast<const __half*>(H16), ldh, row_off, row_cnt, row_term, row_w, row_pos, tail_start, post_cnt,
      sdoc, sw, reinterpret_cast<const __half*>(head_hi), reinterpret_cast<const __half*>(head_lo), kd, tau, delta,
      pairs, count, capacity, window, n_windows, n_items);
  timing_end(ctx, ev);
  return cudaGetLastError();
}

cudaError_t launch_rescore(mrc_ctx* ctx, const mrc_pair* cand, const unsigned long long* n_cand, int64_t cand_cap,
                           const float* qunit, const float* xunit, int32_t k, float tau, mrc_pair* pairs,
                           unsigned long long* count, int64_t capacity) {
  int64_t grid = (int64_t)ctx->num_sms * 8;
  cudaEvent_t ev = nullptr;
  timing_begin(ctx, "rescore", 0.0, 0.0, &ev);
  k_rescore<<<(unsigned)grid, 256, 0, ctx->stream>>>(cand, n_cand, cand_cap, qunit, xunit, k, tau, pairs, count,
                                                     capacity);
  timing_end(ctx, ev);
  return cudaGetLastError();
}

}  // namespace mrc
