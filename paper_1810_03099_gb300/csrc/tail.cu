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

constexpr int kTailThreads = 768;                      // two CTAs per SM
constexpr int kTailWarps = kTailThreads / 32;
constexpr int kMaxWindow = 24576;                      // columns per work item (96 KB of accumulators)
constexpr int kTermBatch = kTailThreads;               // row terms whose postings are flattened together
constexpr float kTailFix = 1073741824.0f;              // 2^30: tail sums stay below 2^31
constexpr float kTailInv = 1.0f / 1073741824.0f;
constexpr int kRankWarps = 8;                          // warps per CTA of the long-list ranking
constexpr int kWalkChunks = 4;                        // 32-posting chunks per lane in flight

// Orders each tail term's postings by document: a posting's rank in its list is the number
// of postings of the same term with a smaller document id (ids in one list are distinct, so
// the ranks are a permutation). One warp per term. Then writes the sorted list and, for the
// posting of term t in slot r of document d, row_walk[offsets[d] + r] = [sorted position + 1,
// end of t's list): the postings of the documents after d that share t. Positions are 32-bit
// (fewer than 2^31 postings).
__device__ __forceinline__ void put_ranked(int32_t at, int32_t end, int32_t d, float w, int32_t r, int64_t off,
                                           int2* __restrict__ spost, int2* __restrict__ row_walk) {
  spost[at] = make_int2(d, __float_as_int(w));
  row_walk[off + r] = make_int2(at + 1, end);
}

// Lists of at most 32 postings: one posting per lane, ranks through shuffles. Every load of a
// posting (document, weight, slot, the document's offset) is issued before the ranking.
__global__ void __launch_bounds__(256) k_rank_small(const int64_t* __restrict__ cstart,
                                                    const int32_t* __restrict__ terms, int32_t n_terms,
                                                    const int4* __restrict__ post,
                                                    const int64_t* __restrict__ doc_off, int2* __restrict__ spost,
                                                    int2* __restrict__ row_walk) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; x < n_terms; x += nwarps) {
    const int32_t c = terms[x];
    const int32_t p0 = (int32_t)cstart[c];
    const int32_t m = (int32_t)cstart[c + 1] - p0;
    int32_t d = 0x7fffffff, r = 0;
    float w = 0.f;
    int64_t off = 0;
    if (lane < m) {
      const int4 pe = post[p0 + lane];
      d = pe.x;
      w = __int_as_float(pe.y);
      r = pe.z;
      off = doc_off[d];
    }
    int32_t rank = 0;
    for (int q = 0; q < m; ++q) rank += __shfl_sync(kFull, d, q) < d ? 1 : 0;
    if (lane < m) put_ranked(p0 + rank, p0 + m, d, w, r, off, spost, row_walk);
  }
}

// Longer lists (up to max_m postings): staged in the warp's shared-memory buffer; each
// posting counts the smaller ids there, four per 16-byte broadcast read.
__global__ void __launch_bounds__(kRankWarps * 32) k_rank_big(
    const int64_t* __restrict__ cstart, const int32_t* __restrict__ terms, int32_t n_terms, int32_t buf,
    const int4* __restrict__ post, const int64_t* __restrict__ doc_off, int2* __restrict__ spost,
    int2* __restrict__ row_walk) {
  extern __shared__ __align__(16) int32_t rbuf[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* sd = rbuf + warp * buf;
  const int64_t nwarps = (int64_t)gridDim.x * kRankWarps;
  for (int64_t x = (int64_t)blockIdx.x * kRankWarps + warp; x < n_terms; x += nwarps) {
    const int32_t c = terms[x];
    const int32_t p0 = (int32_t)cstart[c];
    const int32_t m = (int32_t)cstart[c + 1] - p0;
    const int32_t m4 = (m + 3) & ~3;
    if (m4 > buf) continue;  // excluded by the host
    for (int32_t y = lane; y < m4; y += 32) sd[y] = y < m ? post[p0 + y].x : 0x7fffffff;
    __syncwarp();
    for (int32_t e = lane; e < m; e += 32) {
      const int32_t d = sd[e];
      const int4 pe = post[p0 + e];
      const float w = __int_as_float(pe.y);
      const int32_t r = pe.z;
      const int64_t off = doc_off[d];
      int32_t rank = 0;
      for (int32_t y = 0; y < m4; y += 4) {
        const int4 v = *reinterpret_cast<const int4*>(sd + y);
        rank += (v.x < d) + (v.y < d) + (v.z < d) + (v.w < d);
      }
      put_ranked(p0 + rank, p0 + m, d, w, r, off, spost, row_walk);
    }
    __syncwarp();
  }
}

// ---- head/tail split of the vocabulary (exact cosine set-up) ----------------------------
// A term is a head term (a dense tensor-core column) when df >= cut, a tail term (sparse
// postings) when 2 <= df < cut, and ignored otherwise (a term in one document joins no
// pair). Head columns and tail lists follow term-id order. Three passes: per-block counts
// over 1024-term blocks, one CTA turning them into block offsets, per-term placement.
constexpr int kTermBlock = 1024;
enum { kTcHead = 0, kTcTail, kTcPost, kTcSmall, kTcMaxM, kTcWork, kTcFields };

struct TermFlags {
  int32_t head, tail, post, small;
};
__device__ __forceinline__ TermFlags term_class(int32_t d, int32_t cut) {
  TermFlags f;
  f.head = d >= cut;
  f.tail = d >= 2 && d < cut;
  f.post = f.tail ? d : 0;
  f.small = f.tail && d <= 32;
  return f;
}

// Exclusive scan of v over the CTA (kTermBlock threads); *total receives the sum.
// scratch: 33 words of shared memory.
__device__ __forceinline__ long long block_excl_scan(long long v, long long* scratch, long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();  // scratch is free (a previous scan may still read it)
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const long long w = scratch[lane];
    long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += y;
    }
    scratch[lane] = wi - w;
    if (lane == 31) scratch[32] = wi;
  }
  __syncthreads();
  *total = scratch[32];
  return scratch[warp] + incl - v;
}

__device__ __forceinline__ long long block_max(long long v, long long* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  __syncthreads();
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  if (warp == 0) {
    long long x = scratch[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(kFull, x, o));
    if (lane == 0) scratch[32] = x;
  }
  __syncthreads();
  return scratch[32];
}

__global__ void __launch_bounds__(kTermBlock) k_term_count(const int32_t* __restrict__ df, int32_t V, int32_t cut,
                                                           long long* __restrict__ part) {
  __shared__ long long scratch[33];
  const int64_t t = (int64_t)blockIdx.x * kTermBlock + threadIdx.x;
  const int32_t d = t < V ? df[t] : 0;
  const TermFlags f = term_class(d, cut);
  const long long v[kTcFields] = {f.head, f.tail, f.post, f.small, f.tail ? d : 0,
                                  f.tail ? (long long)d * (d - 1) / 2 : 0};
  long long out[kTcFields];
#pragma unroll
  for (int q = 0; q < kTcFields; ++q) {
    long long total = 0;
    if (q == kTcMaxM)
      total = block_max(v[q], scratch);
    else
      block_excl_scan(v[q], scratch, &total);
    out[q] = total;
  }
  if (threadIdx.x < kTcFields) part[(int64_t)blockIdx.x * kTcFields + threadIdx.x] = out[threadIdx.x];
}

// One CTA: per-block counts -> exclusive per-block offsets (in place, except the maximum
// field), and the totals into summary[kTcFields].
__global__ void __launch_bounds__(kTermBlock) k_term_scan(long long* __restrict__ part, int64_t nb,
                                                          long long* __restrict__ summary) {
  __shared__ long long scratch[33];
  const int64_t per = (nb + kTermBlock - 1) / kTermBlock;  // blocks per thread, contiguous
  const int64_t b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
#pragma unroll 1
  for (int q = 0; q < kTcFields; ++q) {
    long long sum = 0;
    for (int64_t b = b0; b < b1; ++b) {
      const long long x = part[b * kTcFields + q];
      sum = q == kTcMaxM ? max(sum, x) : sum + x;
    }
    if (q == kTcMaxM) {
      const long long m = block_max(sum, scratch);
      if (threadIdx.x == 0) summary[q] = m;
      continue;
    }
    long long total = 0;
    long long run = block_excl_scan(sum, scratch, &total);
    for (int64_t b = b0; b < b1; ++b) {
      const long long x = part[b * kTcFields + q];
      part[b * kTcFields + q] = run;
      run += x;
    }
    if (threadIdx.x == 0) summary[q] = total;
  }
}

// Per term: head column, or tail list start; the tail-list boundaries (cstart), and the tail
// lists split into those of at most 32 postings (rank_terms[0, n_small)) and the longer ones
// (rank_terms[n_small, n_tail)).
__global__ void __launch_bounds__(kTermBlock) k_term_place(const int32_t* __restrict__ df, int32_t V, int32_t cut,
                                                           const long long* __restrict__ part,
                                                           const long long* __restrict__ summary,
                                                           int32_t* __restrict__ colmap, int64_t* __restrict__ tstart,
                                                           int64_t* __restrict__ cstart,
                                                           int32_t* __restrict__ rank_terms) {
  __shared__ long long scratch[33];
  const int64_t t = (int64_t)blockIdx.x * kTermBlock + threadIdx.x;
  const int32_t d = t < V ? df[t] : 0;
  const TermFlags f = term_class(d, cut);
  const long long* off = part + (int64_t)blockIdx.x * kTcFields;
  long long total;
  const long long r_head = off[kTcHead] + block_excl_scan(f.head, scratch, &total);
  const long long r_tail = off[kTcTail] + block_excl_scan(f.tail, scratch, &total);
  const long long r_post = off[kTcPost] + block_excl_scan(f.post, scratch, &total);
  const long long r_small = off[kTcSmall] + block_excl_scan(f.small, scratch, &total);
  if (t >= V) return;
  colmap[t] = f.head ? (int32_t)r_head : (f.tail ? -2 : -1);
  tstart[t] = f.tail ? r_post : 0;
  if (f.tail) {
    cstart[r_tail] = r_post;
    cstart[r_tail + 1] = r_post + d;  // the same value the next tail term writes as its start
    if (f.small)
      rank_terms[r_small] = (int32_t)r_tail;
    else
      rank_terms[summary[kTcSmall] + (r_tail - r_small)] = (int32_t)r_tail;
  }
}

// Exclusive scan of v over the CTA with one barrier: each warp publishes its total, then every
// warp adds up the totals before it itself. scratch: kTailWarps words, not rewritten before
// the CTA's next barrier.
__device__ __forceinline__ int32_t cta_excl_scan1(int32_t v, int32_t* scratch, int32_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) scratch[warp] = incl;
  __syncthreads();
  const int32_t w = lane < kTailWarps ? scratch[lane] : 0;
  int32_t before = lane < warp ? w : 0, all = w;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    before += __shfl_xor_sync(kFull, before, o);
    all += __shfl_xor_sync(kFull, all, o);
  }
  *total = all;
  return before + incl - v;
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

// A work item is one or two segments; a segment is row `row`'s columns [c_lo, c_hi), their
// accumulators at acc[off + (j - cb)] (cb = c_lo rounded down to 8; off a multiple of 8).
struct TailSeg {
  int32_t row, c_lo, c_hi, cb, off;
};

// Work item -> segments (number of non-empty segments returned). With one window per row,
// rows pair up as (r, n-1-r): the pair's columns [r+1, n) and [n-r, n) fill one accumulator
// row of about n entries, so every item costs about the same and the per-item fixed work is
// halved. Otherwise an item is one row's columns within one window.
__device__ __forceinline__ int tail_segments(int64_t item, int32_t n, int32_t window, int32_t n_windows, bool paired,
                                             TailSeg& s0, TailSeg& s1) {
  if (paired) {
    const int32_t r0 = (int32_t)item, r1 = n - 1 - (int32_t)item;
    s0 = TailSeg{r0, r0 + 1, n, (r0 + 1) & ~7, 0};
    s1 = TailSeg{r1, r1 + 1, n, (r1 + 1) & ~7, (n - s0.cb + 7) & ~7};
    const int k0 = s0.c_lo < s0.c_hi, k1 = r1 > r0 && s1.c_lo < s1.c_hi;
    if (!k0) s0 = s1;  // (cannot happen for r0 < n - 1; kept for safety)
    return k0 + k1;
  }
  const int32_t i = (int32_t)(item / n_windows);
  const int32_t base = (int32_t)(item % n_windows) * window;  // a multiple of 8 (window is)
  s0 = TailSeg{i, max(i + 1, base), min(n, base + window), base, 0};
  s1 = s0;
  return s0.c_lo < s0.c_hi ? 1 : 0;
}

// One CTA per work item (see tail_segments). The tail sums accumulate in a shared-memory row
// of 2^-30 fixed-point integers (each product is < 1: rounding <= 2^-31; integer sums do not
// depend on the order in which threads add them):
//  1. acc = 0 over the item's segments;
//  2. for every tail term t of a segment's document i, the postings after i's own position in
//     t's sorted list are exactly the documents j > i sharing t: acc[j] += w_it * w_jt. The
//     CTA takes up to 768 of the item's terms at a time, flattens their postings into one
//     position range (CTA prefix sum of the list lengths, term tables in shared memory) and
//     gives every warp an equal slice of it, four loads per lane in flight, so neither short
//     lists nor uneven terms leave warps idle;
//  3. scan: H16[i][j] (the fp16 head score from the tensor cores, eight columns per 16-byte
//     load) + tail >= tau - delta marks a candidate, where delta bounds the head's error;
//     each candidate's head is recomputed exactly (exact_head) and the pair is kept iff
//     head + tail >= tau.
__global__ void __launch_bounds__(kTailThreads, 2) k_cosine_tail(
    int32_t n, const __half* __restrict__ H, int64_t ldh, const int64_t* __restrict__ row_off,
    const int32_t* __restrict__ row_cnt, const int2* __restrict__ row_walk, const float* __restrict__ row_w,
    const int2* __restrict__ spost, const __half* __restrict__ hhi,
    const __half* __restrict__ hlo, int32_t kd, float tau, float delta, mrc_pair* pairs,
    unsigned long long* count, int64_t capacity, int32_t window, int32_t acc_len, int32_t n_windows, int64_t n_items,
    int32_t paired, unsigned long long* next_item) {
  extern __shared__ int32_t acc[];  // [acc_len] accumulators, then the term table
  // per term of the batch, one 16-byte entry: x = end of its flattened range, y = posting
  // index - flattened position, z = 2^30 x the row's weight (float bits), w = accumulator shift
  int4* t_ent = reinterpret_cast<int4*>(acc + acc_len);  // [kTermBatch]
  __shared__ int32_t t_scan[33];
  __shared__ long long s_item[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float cand_tau = tau - delta;
  // Work items are taken in order as CTAs free up, one ahead: the index of the next item is
  // requested at the start of the current one and read after its first barrier.
  if (threadIdx.x == 0) s_item[0] = (long long)atomicAdd(next_item, 1ull);
  __syncthreads();
  for (int it = 0;; ++it) {
    const int64_t item = s_item[it & 1];
    if (item >= n_items) break;  // block-uniform
    __syncthreads();  // every thread has read s_item[it & 1] before it is requested again
    if (threadIdx.x == 0) s_item[(it + 1) & 1] = (long long)atomicAdd(next_item, 1ull);
    TailSeg sa, sb;
    const int nseg = tail_segments(item, n, window, n_windows, paired != 0, sa, sb);
    if (nseg == 0) {  // block-uniform
      __syncthreads();  // publishes s_item[(it + 1) & 1]
      continue;
    }
    // pull the segments' head scores toward L2 while the tail sums are built (one 128-byte
    // line per thread and segment covers 49,152 columns)
    {
      const int32_t at = (sa.c_lo & ~63) + 64 * (int32_t)threadIdx.x;
      if (at < sa.c_hi) asm volatile("prefetch.global.L2 [%0];" ::"l"(H + (int64_t)sa.row * ldh + at));
      const int32_t bt = (sb.c_lo & ~63) + 64 * (int32_t)threadIdx.x;
      if (nseg > 1 && bt < sb.c_hi) asm volatile("prefetch.global.L2 [%0];" ::"l"(H + (int64_t)sb.row * ldh + bt));
    }
    const TailSeg& sl = nseg > 1 ? sb : sa;
    const int32_t a1 = sl.off + (sl.c_hi - sl.cb);  // accumulators in use
    for (int32_t x = 4 * (int32_t)threadIdx.x; x < a1; x += 4 * kTailThreads)
      *reinterpret_cast<int4*>(acc + x) = make_int4(0, 0, 0, 0);
    __syncthreads();
    const int32_t nt0 = row_cnt[sa.row], nt = nt0 + (nseg > 1 ? row_cnt[sb.row] : 0);
    for (int32_t b0 = 0; b0 < nt; b0 += kTermBatch) {
      // term r = b0 + thread: its remaining postings [st, st + cnt) (documents > its row)
      const int32_t r = b0 + threadIdx.x;
      int32_t st = 0, cnt = 0, sh = 0;
      float wi = 0.f;
      if (r < nt) {
        const bool q = r >= nt0;
        const int64_t ro = row_off[q ? sb.row : sa.row] + (q ? r - nt0 : r);
        const int2 wk = row_walk[ro];
        st = wk.x;
        cnt = wk.y - wk.x;
        wi = row_w[ro];
        sh = q ? sb.off - sb.cb : sa.off - sa.cb;
      }
      int32_t total;
      const int32_t ex = cta_excl_scan1(cnt, t_scan, &total);  // synchronises the CTA
      const int32_t nterm = min(kTermBatch, nt - b0);
      // posting index = y + flattened position
      t_ent[threadIdx.x] = make_int4(ex + cnt, st - ex, __float_as_int(wi * kTailFix), sh);
      __syncthreads();
      // the batch's postings flattened into [0, total); each warp takes an equal slice. The
      // term of position f is the first whose range ends after f (empty terms end where they
      // start, so they are passed over): a lane finds it by binary search for its first
      // position and then only moves forward.
      const int32_t s0 = (int32_t)((int64_t)total * warp / kTailWarps);
      const int32_t s1 = (int32_t)((int64_t)total * (warp + 1) / kTailWarps);
      int32_t own = 0;
      {
        const int32_t f = s0 + lane;
        int32_t a = 0, c = nterm - 1;  // end[c] > f for f < total; find the first such term
        while (a < c) {
          const int32_t m = (a + c) >> 1;
          if (t_ent[m].x <= f) a = m + 1; else c = m;
        }
        own = a;
      }
      int32_t end = t_ent[own].x;  // end of the current term's range
      for (int32_t f0 = s0; f0 < s1; f0 += 32 * kWalkChunks) {
        int2 pv[kWalkChunks];
        float wv[kWalkChunks];
        int32_t shv[kWalkChunks];
#pragma unroll
        for (int u = 0; u < kWalkChunks; ++u) {
          const int32_t f = f0 + 32 * u + lane;
          pv[u] = make_int2(-1, 0);
          wv[u] = 0.f;
          shv[u] = 0;
          if (f < s1) {
            while (end <= f) end = t_ent[++own].x;
            const int4 te = t_ent[own];
            pv[u] = spost[te.y + f];  // (document, weight) of the posting
            wv[u] = __int_as_float(te.z);
            shv[u] = te.w;
          }
        }
        // with one window per row every posting after a segment's row lies in its columns
#pragma unroll
        for (int u = 0; u < kWalkChunks; ++u) {
          const int32_t j = pv[u].x;
          if (n_windows == 1 ? j >= 0 : (j >= sa.c_lo && j < sa.c_hi))
            atomicAdd(&acc[j + shv[u]], __float2int_rn(wv[u] * __int_as_float(pv[u].y)));
        }
      }
      __syncthreads();  // the next batch rewrites the term tables; the scan below reads acc
    }
    // scan: each lane takes eight consecutive columns of one segment (one 16-byte load of H16,
    // in the row's ldh >= round8(n) padding at the end, so never past the row)
    const int32_t g_a = (sa.c_hi - sa.cb + 7) >> 3;  // 8-column groups of the first segment
    const int32_t g_all = g_a + (nseg > 1 ? (sb.c_hi - sb.cb + 7) >> 3 : 0);
    for (int32_t q0 = 32 * warp; q0 < g_all; q0 += kTailThreads) {
      const int32_t q = q0 + lane;
      const bool sq = q >= g_a;
      const TailSeg& sg = sq ? sb : sa;
      const int32_t g = sg.cb + 8 * (sq ? q - g_a : q);
      const int32_t ai = sg.off + (g - sg.cb);
      uint32_t mask = 0;
      if (q < g_all) {
        const uint4 raw = __ldcs(reinterpret_cast<const uint4*>(H + (int64_t)sg.row * ldh + g));
        const __half2* h2 = reinterpret_cast<const __half2*>(&raw);
        const int4 t0 = *reinterpret_cast<const int4*>(acc + ai);
        const int4 t1 = *reinterpret_cast<const int4*>(acc + ai + 4);
        const int32_t tv[8] = {t0.x, t0.y, t0.z, t0.w, t1.x, t1.y, t1.z, t1.w};
        float sv[8];  // head + tail (the 2^-30 scaling is exact)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float2 hf = __half22float2(h2[u]);
          sv[2 * u] = fmaf((float)tv[2 * u], kTailInv, hf.x);
          sv[2 * u + 1] = fmaf((float)tv[2 * u + 1], kTailInv, hf.y);
        }
        // one comparison for the eight columns; the bounds only matter for the rare hits
        // (columns outside [c_lo, c_hi) hold stale values)
        const float mx = fmaxf(fmaxf(fmaxf(sv[0], sv[1]), fmaxf(sv[2], sv[3])),
                               fmaxf(fmaxf(sv[4], sv[5]), fmaxf(sv[6], sv[7])));
        if (mx >= cand_tau) {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (g + e >= sg.c_lo && g + e < sg.c_hi && sv[e] >= cand_tau) mask |= 1u << e;
        }
      }
      unsigned todo = __ballot_sync(kFull, mask != 0);
      while (todo) {  // rare: candidates of one lane at a time, the whole warp per candidate
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        uint32_t m = __shfl_sync(kFull, mask, src);
        const int32_t gs = __shfl_sync(kFull, g, src);
        const int32_t as = __shfl_sync(kFull, ai, src);
        const int32_t row = __shfl_sync(kFull, sg.row, src);
        while (m) {
          const int e = __ffs(m) - 1;
          m &= m - 1;
          const int32_t j = gs + e;
          const float s = exact_head(hhi, hlo, kd, row, j, lane) + (float)acc[as + e] * kTailInv;
          if (lane == 0 && s >= tau) {
            const unsigned long long at = atomicAdd(count, 1ull);
            if (at < (unsigned long long)capacity) {
              mrc_pair pr;
              pr.i = row;
              pr.j = j;
              pr.score = s;
              pairs[at] = pr;
            }
          }
        }
      }
    }
  }
}

// ---- bound-pruned exact cosine: verification of the candidates ---------------------------
// A pair (i, j) is a candidate when the tensor-core head score plus tn_i * tn_j reaches
// tau - delta' (Cauchy-Schwarz bounds the tail dot product by the tail norms). Each candidate
// gets the same score as the tail walk would give it: the head recomputed exactly from the
// split rows plus the tail sum of round((u_i 2^30) u_j) over the tail terms the two documents
// share, found by a hash join in the warp's shared-memory table (the shorter list inserted;
// lists beyond a quarter of the table are joined in hash-partitioned passes).
constexpr int kVerWarps = 8;
constexpr int kVerSlots = 1024;  // per-warp table: term ids and weights (load <= 1/4 per pass)
constexpr int kVerBatch = 8;     // list entries per lane loaded at once

// Exact head from the split rows with all of a lane's loads for two 256-column steps in flight;
// the same sum, in the same order, as exact_head.
// Columns [0, kd) of rows of stride ld.
__device__ __forceinline__ float exact_head_batched(const __half* __restrict__ hhi, const __half* __restrict__ hlo,
                                                    int32_t ld, int32_t kd, int64_t i, int64_t j, int lane) {
  const __half* ai = hhi + i * ld;
  const __half* bi = hlo + i * ld;
  const __half* aj = hhi + j * ld;
  const __half* bj = hlo + j * ld;
  float s = 0.f;
  for (int32_t c0 = 8 * lane; c0 < kd; c0 += 512) {
    uint4 xa[2], xb[2], ya[2], yb[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int32_t c = c0 + 256 * h;
      if (c < kd) {
        xa[h] = __ldg(reinterpret_cast<const uint4*>(ai + c));
        xb[h] = __ldg(reinterpret_cast<const uint4*>(bi + c));
        ya[h] = __ldg(reinterpret_cast<const uint4*>(aj + c));
        yb[h] = __ldg(reinterpret_cast<const uint4*>(bj + c));
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (c0 + 256 * h >= kd) break;
      const __half2* pa = reinterpret_cast<const __half2*>(&xa[h]);
      const __half2* pb = reinterpret_cast<const __half2*>(&xb[h]);
      const __half2* qa = reinterpret_cast<const __half2*>(&ya[h]);
      const __half2* qb = reinterpret_cast<const __half2*>(&yb[h]);
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
  }
  return warp_sum(s);
}

// One (term, weight) batch of a tail list: kVerBatch entries per thread, loads all in flight.
struct ListBatch {
  int32_t t[kVerBatch];
  float w[kVerBatch];
};
__device__ __forceinline__ void load_batch(ListBatch& b, const int32_t* __restrict__ row_term,
                                           const float* __restrict__ row_w, int64_t off, int32_t n, int32_t x0,
                                           int stride, int tid) {
#pragma unroll
  for (int u = 0; u < kVerBatch; ++u) {
    const int32_t x = x0 + stride * u + tid;
    b.t[u] = x < n ? __ldg(row_term + off + x) : -1;
    b.w[u] = x < n ? __ldg(row_w + off + x) : 0.f;
  }
}
// Inserts a batch's terms (of partition ps of 2^lp) into a table of `slots` entries (linear
// probing; a full table gives up and records kErrTable).
__device__ __forceinline__ void insert_batch(const ListBatch& b, int32_t* keys, float* vals, int slots, int lslots,
                                             int lp, int32_t ps, int32_t* err) {
#pragma unroll
  for (int u = 0; u < kVerBatch; ++u) {
    const int32_t t = b.t[u];
    if (t < 0 || (lp > 0 && (int32_t)(((uint32_t)t * 0x9E3779B1u) >> (32 - lp)) != ps)) continue;
    uint32_t slot = ((uint32_t)t * 0x85EBCA6Bu) >> (32 - lslots);
    for (int probes = 0;; ++probes) {
      if (atomicCAS(&keys[slot], -1, t) == -1) {
        vals[slot] = b.w[u];
        break;
      }
      slot = (slot + 1) & (slots - 1);
      if (probes + 1 == slots) {
        set_err(err, kErrTable);
        break;
      }
    }
  }
}
// Adds round((w_i 2^30) w_j) for the batch's terms found in the table (the table holds the
// weights of document i when i_small, else of document j).
__device__ __forceinline__ long long probe_batch(const ListBatch& b, const int32_t* keys, const float* vals, int slots,
                                                 int lslots, int lp, int32_t ps, bool i_small) {
  long long acc = 0;
#pragma unroll
  for (int u = 0; u < kVerBatch; ++u) {
    const int32_t t = b.t[u];
    if (t < 0 || (lp > 0 && (int32_t)(((uint32_t)t * 0x9E3779B1u) >> (32 - lp)) != ps)) continue;
    uint32_t slot = ((uint32_t)t * 0x85EBCA6Bu) >> (32 - lslots);
    for (int probes = 0; probes < slots; ++probes) {
      const int32_t k = keys[slot];
      if (k == t) {
        const float ws = vals[slot];
        const float wi = i_small ? ws : b.w[u], wj = i_small ? b.w[u] : ws;
        acc += __float2int_rn((wi * kTailFix) * wj);
        break;
      }
      if (k == -1) break;
      slot = (slot + 1) & (slots - 1);
    }
  }
  return acc;
}
__device__ __forceinline__ void emit_verified(float s, float tau, int32_t i, int32_t j, mrc_pair* pairs,
                                              unsigned long long* count, int64_t capacity) {
  if (s >= tau) {
    const unsigned long long at = atomicAdd(count, 1ull);
    if (at < (unsigned long long)capacity) {
      mrc_pair pr;
      pr.i = i;
      pr.j = j;
      pr.score = s;
      pairs[at] = pr;
    }
  }
}

// Warp per candidate whose shorter tail list fits a quarter of the warp's table (one pass) and
// whose longer list takes at most two probe batches; the others are appended to long_idx for
// k_cosine_verify_long.
__global__ void __launch_bounds__(kVerWarps * 32, 3) k_cosine_verify(
    const mrc_pair* __restrict__ cand, const unsigned long long* __restrict__ n_cand, int64_t cand_cap,
    const __half* __restrict__ hhi, const __half* __restrict__ hlo, int32_t ld, int32_t kd_arg,
    const int32_t* __restrict__ kd_dev, const int64_t* __restrict__ row_off, const int32_t* __restrict__ row_cnt,
    const int32_t* __restrict__ row_term, const float* __restrict__ row_w, float tau, mrc_pair* pairs,
    unsigned long long* count, int64_t capacity, int32_t* long_idx, unsigned long long* n_long, int32_t* err) {
  const int32_t kd = kd_dev ? *kd_dev : kd_arg;
  extern __shared__ __align__(16) int32_t vsm[];  // [kVerWarps][kVerSlots keys + kVerSlots weights]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* keys = vsm + warp * 2 * kVerSlots;
  float* vals = reinterpret_cast<float*>(keys + kVerSlots);
  const unsigned long long nc0 = *n_cand;
  const int64_t nc = nc0 < (unsigned long long)cand_cap ? (int64_t)nc0 : cand_cap;
  if (err && nc0 > (unsigned long long)cand_cap && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrOverflow);
  const int64_t nwarps = (int64_t)gridDim.x * kVerWarps;
  for (int64_t c = (int64_t)blockIdx.x * kVerWarps + warp; c < nc; c += nwarps) {
    const mrc_pair pc = cand[c];
    const int32_t i = pc.i, j = pc.j;
    const int32_t ni = row_cnt[i], nj = row_cnt[j];
    const bool i_small = ni <= nj;
    const int32_t ns = i_small ? ni : nj, nl = i_small ? nj : ni;
    if (ns > kVerSlots / 4 || nl > kVerSlots / 2) {  // more than one table pass or two probe batches
      if (lane == 0) long_idx[atomicAdd(n_long, 1ull)] = (int32_t)c;
      continue;
    }
    const int64_t os = row_off[i_small ? i : j], ol = row_off[i_small ? j : i];
    long long acc = 0;
    if (ns > 0) {
      ListBatch b;
      load_batch(b, row_term, row_w, os, ns, 0, 32, lane);  // ns <= 32 * kVerBatch
      for (int x = 4 * lane; x < kVerSlots; x += 128) *reinterpret_cast<int4*>(keys + x) = make_int4(-1, -1, -1, -1);
      __syncwarp();
      insert_batch(b, keys, vals, kVerSlots, 10, 0, 0, err);
      __syncwarp();
      for (int32_t y0 = 0; y0 < nl; y0 += 32 * kVerBatch) {
        load_batch(b, row_term, row_w, ol, nl, y0, 32, lane);
        acc += probe_batch(b, keys, vals, kVerSlots, 10, 0, 0, i_small);
      }
      __syncwarp();
    }
    const float head = exact_head_batched(hhi, hlo, ld, kd, i, j, lane);
    const long long tail = warp_sum(acc);
    if (lane == 0) emit_verified(head + (float)tail * kTailInv, tau, i, j, pairs, count, capacity);
  }
}

// CTA per candidate with a long shorter list: the CTA's whole table (kVerWarps * kVerSlots
// slots), a quarter of it per hash-partitioned pass. The head comes from warp 0 (the same sum
// as every other path).
__global__ void __launch_bounds__(kVerWarps * 32, 3) k_cosine_verify_long(
    const mrc_pair* __restrict__ cand, const int32_t* __restrict__ long_idx, const unsigned long long* __restrict__ n_long,
    const __half* __restrict__ hhi, const __half* __restrict__ hlo, int32_t ld, int32_t kd_arg,
    const int32_t* __restrict__ kd_dev, const int64_t* __restrict__ row_off, const int32_t* __restrict__ row_cnt,
    const int32_t* __restrict__ row_term, const float* __restrict__ row_w, float tau, mrc_pair* pairs,
    unsigned long long* count, int64_t capacity, int32_t* err) {
  const int32_t kd = kd_dev ? *kd_dev : kd_arg;
  constexpr int kSlots = kVerWarps * kVerSlots, kLog = 13;  // 8192 slots
  static_assert((1 << kLog) == kSlots, "table size");
  extern __shared__ __align__(16) int32_t vsm[];
  int32_t* keys = vsm;
  float* vals = reinterpret_cast<float*>(keys + kSlots);
  __shared__ unsigned long long s_tail;
  __shared__ float s_head;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nl_total = (int64_t)*n_long;
  for (int64_t q = blockIdx.x; q < nl_total; q += gridDim.x) {
    const mrc_pair pc = cand[long_idx[q]];
    const int32_t i = pc.i, j = pc.j;
    const int32_t ni = row_cnt[i], nj = row_cnt[j];
    const bool i_small = ni <= nj;
    const int64_t os = row_off[i_small ? i : j], ol = row_off[i_small ? j : i];
    const int32_t ns = i_small ? ni : nj, nl = i_small ? nj : ni;
    int lp = 0;
    while ((ns >> lp) > kSlots / 4) ++lp;
    const int32_t passes = 1 << lp;
    if (threadIdx.x == 0) s_tail = 0ull;
    long long acc = 0;
    for (int32_t ps = 0; ps < passes; ++ps) {
      __syncthreads();  // the previous pass's probes (and s_tail's reset) are done
      for (int x = 4 * (int)threadIdx.x; x < kSlots; x += 4 * kVerWarps * 32)
        *reinterpret_cast<int4*>(keys + x) = make_int4(-1, -1, -1, -1);
      __syncthreads();
      ListBatch b;
      for (int32_t x0 = 0; x0 < ns; x0 += kVerWarps * 32 * kVerBatch) {
        load_batch(b, row_term, row_w, os, ns, x0, kVerWarps * 32, threadIdx.x);
        insert_batch(b, keys, vals, kSlots, kLog, lp, ps, err);
      }
      __syncthreads();
      for (int32_t y0 = 0; y0 < nl; y0 += kVerWarps * 32 * kVerBatch) {
        load_batch(b, row_term, row_w, ol, nl, y0, kVerWarps * 32, threadIdx.x);
        acc += probe_batch(b, keys, vals, kSlots, kLog, lp, ps, i_small);
      }
    }
    const long long wsum = warp_sum(acc);
    if (lane == 0) atomicAdd(&s_tail, (unsigned long long)wsum);
    if (warp == 0) {
      const float h = exact_head_batched(hhi, hlo, ld, kd, i, j, lane);
      if (lane == 0) s_head = h;
    }
    __syncthreads();
    if (threadIdx.x == 0)
      emit_verified(s_head + (float)(long long)s_tail * kTailInv, tau, i, j, pairs, count, capacity);
    __syncthreads();  // s_tail, s_head and the table are reused by the next candidate
  }
}

// FP32 rescoring of candidates: one thread per candidate (unit_dot of its two unit signatures,
// so the loads of both rows are in flight together), kept iff the score is >= tau; the warp's
// kept pairs are appended with one atomic.
__global__ void k_rescore(const mrc_pair* __restrict__ cand, const unsigned long long* n_cand, int64_t cand_cap,
                          const float* __restrict__ qunit, const float* __restrict__ xunit, int32_t k, float tau,
                          mrc_pair* pairs, unsigned long long* count, int64_t capacity, int32_t* err) {
  const int lane = threadIdx.x & 31;
  const int64_t nc0 = (int64_t)*n_cand;
  const int64_t nc = nc0 < cand_cap ? nc0 : cand_cap;
  if (err && nc0 > cand_cap && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrOverflow);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < nc; w0 += stride) {
    const int64_t c = w0 + lane;
    mrc_pair pr{0, 0, 0.f};
    bool keep = false;
    if (c < nc) {
      pr = cand[c];
      pr.score = unit_dot(qunit + (int64_t)pr.i * k, xunit + (int64_t)pr.j * k, k);
      keep = pr.score >= tau;
    }
    const unsigned m = __ballot_sync(kFull, keep);
    if (m) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(count, (unsigned long long)__popc(m));
      b = __shfl_sync(kFull, b, 0) + (unsigned long long)__popc(m & ((1u << lane) - 1u));
      if (keep && b < (unsigned long long)capacity) pairs[b] = pr;
    }
  }
}

}  // namespace

cudaError_t launch_cosine_terms(mrc_ctx* ctx, const int32_t* df, int32_t V, int32_t cut, long long* part,
                                long long* summary, int32_t* colmap, int64_t* tstart, int64_t* cstart,
                                int32_t* rank_terms) {
  if (V <= 0) return cudaErrorInvalidValue;
  const int64_t nb = ((int64_t)V + kTermBlock - 1) / kTermBlock;
  if (nb > 0x7fffffff) return cudaErrorInvalidValue;
  {
    KernelTimer kt(ctx, "term_count", 4.0 * V);
    k_term_count<<<(unsigned)nb, kTermBlock, 0, ctx->stream>>>(df, V, cut, part);
  }
  {
    KernelTimer kt(ctx, "term_scan", 96.0 * nb);
    k_term_scan<<<1, kTermBlock, 0, ctx->stream>>>(part, nb, summary);
  }
  KernelTimer kt(ctx, "term_place", 28.0 * V);
  k_term_place<<<(unsigned)nb, kTermBlock, 0, ctx->stream>>>(df, V, cut, part, summary, colmap, tstart, cstart,
                                                             rank_terms);
  return cudaGetLastError();
}

cudaError_t launch_rank_postings(mrc_ctx* ctx, const int64_t* cstart, const int32_t* small_terms, int32_t n_small,
                                 const int32_t* big_terms, int32_t n_big, int32_t max_m, const int4* post,
                                 const int64_t* doc_off, void* spost,
                                 void* row_walk) {
  if (n_small > 0) {
    int64_t grid = (int64_t)ctx->num_sms * resident_ctas(k_rank_small, 256, 0);
    const int64_t need = ((int64_t)n_small + 7) / 8;
    if (need < grid) grid = need;
    KernelTimer kt(ctx, "rank_small");
    k_rank_small<<<(unsigned)grid, 256, 0, ctx->stream>>>(cstart, small_terms, n_small, post,
                                                           doc_off, reinterpret_cast<int2*>(spost),
                                                           reinterpret_cast<int2*>(row_walk));
  }
  if (n_big > 0) {
    const int32_t buf = (max_m + 3) & ~3;
    const size_t smem = sizeof(int32_t) * (size_t)kRankWarps * buf;
    const int per_sm = resident_ctas(k_rank_big, kRankWarps * 32, smem);
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    int64_t grid = (int64_t)ctx->num_sms * per_sm;
    const int64_t need = ((int64_t)n_big + kRankWarps - 1) / kRankWarps;
    if (need < grid) grid = need;
    KernelTimer kt(ctx, "rank_big");
    k_rank_big<<<(unsigned)grid, kRankWarps * 32, smem, ctx->stream>>>(cstart, big_terms, n_big, buf, post,
                                                                       doc_off,
                                                                       reinterpret_cast<int2*>(spost),
                                                                       reinterpret_cast<int2*>(row_walk));
  }
  return cudaGetLastError();
}

__global__ void k_cosine_dims(const long long* __restrict__ tsum, int32_t kd_h_max, int32_t* __restrict__ dims) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const long long h = tsum[kTcHead];
  int32_t kd_h = (int32_t)(((h < 0 ? 0 : h) + 63) / 64 * 64);
  if (kd_h > kd_h_max) kd_h = kd_h_max;  // cannot happen: the head has at most n_tokens / cut terms
  dims[0] = kd_h;
  dims[1] = (kd_h + kTailBuckets) / 64;
}

cudaError_t launch_cosine_dims(mrc_ctx* ctx, const long long* split_totals, int32_t kd_h_max, int32_t* dims) {
  KernelTimer kt(ctx, "cosine_dims");
  k_cosine_dims<<<1, 32, 0, ctx->stream>>>(split_totals, kd_h_max, dims);
  return cudaGetLastError();
}

// Rows of 16-byte chunks; hi: columns [0, kd_h + kTailBuckets), lo: [0, kd_h) (all multiples of 8).
__global__ void k_zero_head(uint4* __restrict__ hi, uint4* __restrict__ lo, int64_t n, int32_t ld,
                            const int32_t* __restrict__ dims) {
  const int32_t kd_h = dims[0];
  const int32_t chi = (kd_h + kTailBuckets) / 8, clo = kd_h / 8, cld = ld / 8;
  const int64_t total = n * (int64_t)chi;
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = x / chi;
    const int32_t c = (int32_t)(x - r * chi);
    hi[r * cld + c] = make_uint4(0u, 0u, 0u, 0u);
    if (c < clo) lo[r * cld + c] = make_uint4(0u, 0u, 0u, 0u);
  }
}

cudaError_t launch_zero_head(mrc_ctx* ctx, void* head_hi, void* head_lo, int64_t n, int32_t ld, const int32_t* dims) {
  if (ld % 8 != 0 || n <= 0) return cudaErrorInvalidValue;
  KernelTimer kt(ctx, "zero_head");
  k_zero_head<<<(unsigned)(4 * ctx->num_sms), 256, 0, ctx->stream>>>(reinterpret_cast<uint4*>(head_hi),
                                                                     reinterpret_cast<uint4*>(head_lo), n, ld, dims);
  return cudaGetLastError();
}

cudaError_t launch_cosine_verify(mrc_ctx* ctx, const mrc_pair* cand, const unsigned long long* n_cand,
                                 int64_t cand_cap, const void* head_hi, const void* head_lo, int32_t ld, int32_t kd,
                                 const int32_t* kd_dev, const int64_t* row_off, const int32_t* row_cnt, const int32_t* row_term,
                                 const float* row_w, float tau, mrc_pair* pairs, unsigned long long* count,
                                 int64_t capacity, int32_t* long_idx, unsigned long long* n_long, int32_t* err) {
  if ((kd & 63) || kd < 0 || (ld & 7) || ld < kd) return cudaErrorInvalidValue;
  const size_t smem = sizeof(int32_t) * 2 * kVerSlots * kVerWarps;
  const int per_sm = resident_ctas(k_cosine_verify, kVerWarps * 32, smem);
  const int per_sm_long = resident_ctas(k_cosine_verify_long, kVerWarps * 32, smem);
  if (per_sm <= 0 || per_sm_long <= 0) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaMemsetAsync(n_long, 0, sizeof(unsigned long long), ctx->stream);
  if (e != cudaSuccess) return e;
  const __half* hi = reinterpret_cast<const __half*>(head_hi);
  const __half* lo = reinterpret_cast<const __half*>(head_lo);
  {
    KernelTimer kt(ctx, "cosine_verify");
    k_cosine_verify<<<(unsigned)(ctx->num_sms * per_sm), kVerWarps * 32, smem, ctx->stream>>>(
        cand, n_cand, cand_cap, hi, lo, ld, kd, kd_dev, row_off, row_cnt, row_term, row_w, tau, pairs, count,
        capacity, long_idx, n_long, err);
  }
  KernelTimer kt(ctx, "cosine_verify_long");
  k_cosine_verify_long<<<(unsigned)(ctx->num_sms * per_sm_long), kVerWarps * 32, smem, ctx->stream>>>(
      cand, long_idx, n_long, hi, lo, ld, kd, kd_dev, row_off, row_cnt, row_term, row_w, tau, pairs, count, capacity,
      err);
  return cudaGetLastError();
}

cudaError_t launch_cosine_tail(mrc_ctx* ctx, int64_t n, const void* H16, int64_t ldh, const int64_t* row_off,
                               const int32_t* row_cnt, const void* row_walk, const float* row_w, const void* spost,
                               int64_t n_postings, const void* head_hi, const void* head_lo,
                               int32_t kd, float tau, float delta, mrc_pair* pairs, unsigned long long* count,
                               int64_t capacity, double work_pairs, unsigned long long* next_item) {
  if (n <= 1) return cudaSuccess;
  if (!next_item) return cudaErrorInvalidValue;
  // documents and postings are indexed in 32 bits
  if ((ldh & 7) || ldh < (n + 7) / 8 * 8 || (kd & 63) || kd <= 0 || n >= (1ll << 31) - 64 ||
      n_postings >= (1ll << 31) - 64)
    return cudaErrorInvalidValue;
  const int64_t n8 = (n + 7) / 8 * 8;
  const int32_t window = (int32_t)(n8 < kMaxWindow ? n8 : kMaxWindow);  // a multiple of 8
  const int32_t n_windows = (int32_t)((n + window - 1) / window);
  // one window per row: rows pair up, (n + 1) / 2 items over about n + 16 accumulators
  const int32_t paired = n_windows == 1 ? 1 : 0;
  const int64_t n_items = paired ? (n + 1) / 2 : n * n_windows;
  const int32_t acc_len = paired ? window + 32 : window;
  const size_t smem = sizeof(int32_t) * (size_t)acc_len + sizeof(int4) * kTermBatch;
  const int per_sm = resident_ctas(k_cosine_tail, kTailThreads, smem);
  if (per_sm <= 0) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)ctx->num_sms * per_sm;
  if (n_items < grid) grid = n_items;
  cudaError_t e = cudaMemsetAsync(next_item, 0, sizeof(unsigned long long), ctx->stream);
  if (e != cudaSuccess) return e;
  cudaEvent_t ev = nullptr;
  // algorithmic bytes: the upper triangle of the fp16 head scores read once; flops: 2 per
  // tail posting product
  timing_begin(ctx, "cosine_tail", 2.0 * (double)n * (double)(n - 1) / 2.0, 2.0 * work_pairs, &ev);
  k_cosine_tail<<<(unsigned)grid, kTailThreads, smem, ctx->stream>>>(
      (int32_t)n, reinterpret_cast<const __half*>(H16), ldh, row_off, row_cnt, reinterpret_cast<const int2*>(row_walk),
      row_w, reinterpret_cast<const int2*>(spost), reinterpret_cast<const __half*>(head_hi), reinterpret_cast<const __half*>(head_lo), kd, tau, delta,
      pairs, count, capacity, window, acc_len, n_windows, n_items, paired, next_item);
  timing_end(ctx, ev);
  return cudaGetLastError();
}

cudaError_t launch_rescore(mrc_ctx* ctx, const mrc_pair* cand, const unsigned long long* n_cand, int64_t cand_cap,
                           const float* qunit, const float* xunit, int32_t k, float tau, mrc_pair* pairs,
                           unsigned long long* count, int64_t capacity, int32_t* err) {
  const int64_t grid = (int64_t)ctx->num_sms * 8;
  cudaEvent_t ev = nullptr;
  timing_begin(ctx, "rescore", 0.0, 0.0, &ev);
  k_rescore<<<(unsigned)grid, 256, 0, ctx->stream>>>(cand, n_cand, cand_cap, qunit, xunit, k, tau, pairs, count,
                                                     capacity, err);
  timing_end(ctx, ev);
  return cudaGetLastError();
}

}  // namespace mrc
