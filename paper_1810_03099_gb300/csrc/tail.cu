// tail.cu -- sparse completion of the exact cosine, and FP32 rescoring of candidates.
//
// Exact cosine (Eq. 1) of unit TF-IDF vectors splits over the vocabulary:
// cos(i, j) = sum over frequent ("head") terms + sum over the other terms.
// The head sums come from the tensor-core GEMM as an FP32 matrix H. This
// kernel adds the remaining terms from postings lists and applies the
// threshold (see k_cosine_tail).
//
// Rescoring (reduced-precision forms): each candidate pair found with a
// lowered threshold in FP8 or FP16 is recomputed as an FP32 dot product of the
// two FP32 unit signatures and kept iff it reaches tau.
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

// One CTA per (row i, column window) work item, accumulating in a shared-memory row of
// 2^-30 fixed-point integers (each product is < 1: rounding <= 2^-31; integer sums do not
// depend on the order in which threads add them):
//  1. acc[j] = H[i][j] for the window (independent loads, four per thread in flight);
//  2. for every tail term t of document i, the postings after i's own position in t's
//     sorted list are exactly the documents j > i sharing t: acc[j] += w_it * w_jt. Each
//     warp takes 32 of the row's terms at a time (one lane per term holds its metadata),
//     flattens their postings into one index range (warp prefix sum; a shuffle binary
//     search maps an index back to its term) and walks it with four loads per lane in
//     flight, so short lists do not leave lanes idle;
//  3. threshold and warp-aggregated compaction.
__global__ void __launch_bounds__(kTailThreads) k_cosine_tail(
    int64_t n, const float* __restrict__ H, int64_t ldh, const int64_t* __restrict__ row_off,
    const int32_t* __restrict__ row_cnt, const int32_t* __restrict__ row_term, const float* __restrict__ row_w,
    const int64_t* __restrict__ row_pos, const int64_t* __restrict__ tail_start, const int32_t* __restrict__ post_cnt,
    const int32_t* __restrict__ sdoc, const float* __restrict__ sw, float tau, mrc_pair* pairs,
    unsigned long long* count, int64_t capacity, int64_t window, int64_t n_windows, int64_t n_items) {
  extern __shared__ int32_t acc[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int64_t i = item / n_windows;
    const int64_t w = item % n_windows;
    const int64_t base = w * window;
    const int64_t lo = max(i + 1, base), hi = min(n, base + window);
    if (lo >= hi) continue;  // block-uniform
    const float* hrow = H + i * ldh;
    __syncthreads();  // the previous item's scan is done with acc
    for (int64_t j = lo + threadIdx.x; j < hi; j += 8 * kTailThreads) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t jj = j + u * kTailThreads;
        v[u] = jj < hi ? __ldcs(hrow + jj) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t jj = j + u * kTailThreads;
        if (jj < hi) acc[jj - base] = __float2int_rn(v[u] * kTailFix);
      }
    }
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
    for (int64_t x0 = lo; x0 < hi; x0 += kTailThreads) {
      const int64_t j = x0 + threadIdx.x;
      float s = 0.f;
      bool hit = false;
      if (j < hi) {
        s = (float)acc[j - base] * kTailInv;
        hit = s >= tau;
      }
      const unsigned bal = __ballot_sync(kFull, hit);
      if (bal) {
        unsigned long long at0 = 0;
        if (lane == 0) at0 = atomicAdd(count, (unsigned long long)__popc(bal));
        at0 = __shfl_sync(kFull, at0, 0);
        if (hit) {
          const unsigned long long at = at0 + __popc(bal & ((1u << lane) - 1u));
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

cudaError_t launch_cosine_tail(mrc_ctx* ctx, int64_t n, const float* H, int64_t ldh, const int64_t* row_off,
                               const int32_t* row_cnt, const int32_t* row_term, const float* row_w,
                               const int64_t* row_pos, const int64_t* tail_start, const int32_t* post_cnt,
                               const int32_t* sdoc, const float* sw, float tau, mrc_pair* pairs,
                               unsigned long long* count, int64_t capacity, double work_pairs) {
  if (n <= 1) return cudaSuccess;
  const int64_t window = n < kMaxWindow ? n : kMaxWindow;
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
  // algorithmic bytes: the upper triangle of H read once; flops: 2 per tail posting product
  timing_begin(ctx, "cosine_tail", 4.0 * (double)n * (double)(n - 1) / 2.0, 2.0 * work_pairs, &ev);
  k_cosine_tail<<<(unsigned)grid, kTailThreads, smem, ctx->stream>>>(n, H, ldh, row_off, row_cnt, row_term, row_w,
                                                                     row_pos, tail_start, post_cnt, sdoc, sw, tau,
                                                                     pairs, count, capacity, window, n_windows,
                                                                     n_items);
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
