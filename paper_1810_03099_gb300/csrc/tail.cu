// tail.cu -- sparse completion of the exact cosine, and FP32 rescoring of candidates.
//
// Exact cosine (Eq. 1) of unit TF-IDF vectors splits over the vocabulary:
// cos(i, j) = sum over frequent ("head") terms + sum over the other terms.
// The head sums come from the tensor-core GEMM as an FP32 matrix H. This
// kernel adds the remaining terms from postings lists and applies the
// threshold: one CTA per (row i, column window) work item accumulates, in a
// shared-memory row of 2^-40 fixed-point integers (order-free, hence
// deterministic), H[i][j] plus w_it * w_jt for every tail term t of document
// i and every later document j in t's postings; then it emits every j > i
// with cos(i, j) >= tau.
//
// Rescoring (reduced-precision forms): each candidate pair found with a
// lowered threshold in FP8 or FP16 is recomputed as an FP32 dot product of the
// two FP32 unit signatures and kept iff it reaches tau.
#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

constexpr int kTailThreads = 256;
constexpr int kWindow = 4096;  // columns per work item (32 KB of accumulators)
constexpr float kTailFix = 1099511627776.0f;  // 2^40
constexpr float kTailInv = 1.0f / 1099511627776.0f;

__global__ void __launch_bounds__(kTailThreads) k_cosine_tail(
    int64_t n, const float* __restrict__ H, int64_t ldh, const int64_t* __restrict__ row_off,
    const int32_t* __restrict__ row_cnt, const int32_t* __restrict__ row_term, const float* __restrict__ row_w,
    const int64_t* __restrict__ tail_start, const int32_t* __restrict__ post_cnt, const int32_t* __restrict__ post_doc,
    const float* __restrict__ post_w, float tau, mrc_pair* pairs, unsigned long long* count, int64_t capacity,
    int64_t n_windows, int64_t n_items) {
  __shared__ long long acc[kWindow];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t item = blockIdx.x; item < n_items; item += gridDim.x) {
    const int64_t i = item / n_windows;
    const int64_t w = item % n_windows;
    const int64_t lo = max(i + 1, w * kWindow), hi = min(n, (w + 1) * kWindow);
    if (lo >= hi) continue;  // block-uniform
    const int64_t base = w * kWindow;
    __syncthreads();
    for (int64_t j = lo + threadIdx.x; j < hi; j += kTailThreads)
      acc[j - base] = __float2ll_rn(H[i * ldh + j] * kTailFix);
    __syncthreads();
    const int32_t nt = row_cnt[i];
    const int64_t ro = row_off[i];
    for (int32_t r = warp; r < nt; r += kTailThreads / 32) {
      const int32_t t = row_term[ro + r];
      const float wi = row_w[ro + r];
      const int64_t s0 = tail_start[t], cnt = post_cnt[t];
      for (int64_t x = lane; x < cnt; x += 32) {
        const int64_t j = post_doc[s0 + x];
        if (j >= lo && j < hi) {
          const float prod = wi * post_w[s0 + x];
          atomicAdd(reinterpret_cast<unsigned long long*>(&acc[j - base]),
                    (unsigned long long)__float2ll_rn(prod * kTailFix));
        }
      }
    }
    __syncthreads();
    // threshold and warp-aggregated emission
    const int64_t span = hi - lo;
    for (int64_t x0 = 0; x0 < span; x0 += kTailThreads) {
      const int64_t j = lo + x0 + threadIdx.x;
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

cudaError_t launch_cosine_tail(mrc_ctx* ctx, int64_t n, const float* H, int64_t ldh, const int64_t* row_off,
                               const int32_t* row_cnt, const int32_t* row_term, const float* row_w,
                               const int64_t* tail_start, const int32_t* post_cnt, const int32_t* post_doc,
                               const float* post_w, float tau, mrc_pair* pairs, unsigned long long* count,
                               int64_t capacity, double work_pairs) {
  if (n <= 1) return cudaSuccess;
  const int64_t n_windows = (n + kWindow - 1) / kWindow;
  const int64_t n_items = n * n_windows;
  int64_t grid = (int64_t)ctx->num_sms * 6;
  if (n_items < grid) grid = n_items;
  cudaEvent_t ev = nullptr;
  // algorithmic bytes: the upper triangle of H read once; flops: 2 per tail posting product
  timing_begin(ctx, "cosine_tail", 4.0 * (double)n * (double)(n - 1) / 2.0, 2.0 * work_pairs, &ev);
  k_cosine_tail<<<(unsigned)grid, kTailThreads, 0, ctx->stream>>>(n, H, ldh, row_off, row_cnt, row_term, row_w,
                                                                  tail_start, post_cnt, post_doc, post_w, tau, pairs,
                                                                  count, capacity, n_windows, n_items);
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
