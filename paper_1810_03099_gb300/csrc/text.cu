// text.cu -- character 3-grams of raw text (the front end of Section III's vector space model).
//
// A document is a byte range of one text buffer. Its terms are the 3-grams of the 26-letter
// alphabet (case folded): every window of three consecutive letters inside the document, with
// id 676 x + 26 y + z (letters numbered 0..25). Other bytes separate.
//
// The text is cut into 8,192-byte tiles, one CTA each, independent of document boundaries, so
// the work is balanced whatever the length mix. A thread holds 32 bytes of the tile (and the 4
// after them) in registers and tests four bytes per operation (letter masks and letter numbers
// by byte-parallel arithmetic on 32-bit words); the CTA marks the document starts that fall in
// its tile in shared memory. Position p starts a 3-gram iff bytes p, p+1, p+2 are letters and
// no document starts at p+1 or p+2. Two passes: the first counts each tile's 3-grams, a
// one-CTA scan turns the counts into tile offsets, and the second writes the ids (staged in
// shared memory in text order, stored coalesced) and every document's 3-gram offset.
#include <algorithm>
#include <cstdint>

#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

constexpr int kGramTile = 8192;             // bytes per CTA
constexpr int kGramThreads = 256;           // 8 warps x 1,024 bytes
constexpr int kGramWords = kGramTile / 32;  // 32-bit masks per tile

struct GramArgs {
  int64_t n_docs;
  const int64_t* text_offsets;  // [n_docs + 1]
  const uint8_t* text;          // [n_bytes]
  int64_t n_bytes;
  int64_t* gram_offsets;  // [n_docs + 1] (write pass)
  int32_t* grams;         // [capacity] (write pass)
  int64_t capacity;
  const int64_t* tile_doc;  // [n_tiles] first document starting at or after the tile's first byte
  int32_t* tile_cnt;    // [n_tiles] (count pass)
  unsigned long long* group_sum;  // [ceil(n_tiles / 1024)] 3-grams per group of 1,024 tiles
  int64_t* tile_base;   // [n_tiles + 1] exclusive offsets, then the total (write pass)
  int32_t* err;
  int vec16;  // text is 16-byte aligned: 16-byte loads
};

constexpr int64_t kNoDoc = 0x7FFFFFFFFFFFFFFFll;  // offset of a document past the last

// Byte k of letter_bytes4(w) is 1 iff byte k of w is an ASCII letter of either case (bit k of
// letter_bits4, packed). Four bytes at a time: bytes >= 0x80 are excluded by their top bit; for
// the others (low 7 bits z, case folded) the adds z + 0x1F and z + 0x05 reach the top bit
// exactly when z >= 'a' and z > 'z', and never carry into the next byte.
__device__ __forceinline__ uint32_t letter_bytes4(uint32_t w) {  // 0x01 in each letter byte
  const uint32_t y = w | 0x20202020u;
  const uint32_t z = y & 0x7F7F7F7Fu;
  const uint32_t ge = (z + 0x1F1F1F1Fu) & 0x80808080u;
  const uint32_t gt = (z + 0x05050505u) & 0x80808080u;
  return (ge & ~gt & ~(y & 0x80808080u)) >> 7;
}
__device__ __forceinline__ uint32_t letter_bits4(uint32_t m) {  // m = letter_bytes4(w)
  return (m | (m >> 7) | (m >> 14) | (m >> 21)) & 0xFu;
}

// Byte k of the result: the letter number 0..25 of byte k of w if that byte is a letter, else 0
// ((b | 0xA0) - 0x61 has its top bit set and never borrows; the low 7 bits are the number).
__device__ __forceinline__ uint32_t letter_nums4(uint32_t w, uint32_t m) {
  return ((w | 0xA0A0A0A0u) - 0x61616161u) & (m * 0x7Fu);
}

// The 36 text bytes [p, p + 36) as nine little-endian words (zeros past the end of the text).
__device__ __forceinline__ void load36(const GramArgs& a, int64_t p, uint32_t (&w)[9]) {
  if (a.vec16 && p + 36 <= a.n_bytes) {
    const uint4* g = reinterpret_cast<const uint4*>(a.text + p);
    const uint4 u0 = __ldg(g), u1 = __ldg(g + 1);
    w[0] = u0.x, w[1] = u0.y, w[2] = u0.z, w[3] = u0.w;
    w[4] = u1.x, w[5] = u1.y, w[6] = u1.z, w[7] = u1.w;
    w[8] = __ldg(reinterpret_cast<const uint32_t*>(a.text + p + 32));
    return;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    uint32_t x = 0u;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int64_t q = p + 4 * k + b;
      x |= (q < a.n_bytes ? (uint32_t)__ldg(a.text + q) : 0u) << (8 * b);
    }
    w[k] = x;
  }
}

__device__ __forceinline__ int64_t doc_start(const GramArgs& a, int64_t d) {
  return d <= a.n_docs ? __ldg(a.text_offsets + d) : kNoDoc;
}

// Thread i of the CTA owns bytes [32 i, 32 i + 32) of the tile and holds them in registers,
// with the 4 bytes after them.
template <bool WRITE>
__global__ void __launch_bounds__(kGramThreads) k_text_grams(GramArgs a) {
  __shared__ uint32_t starts[kGramWords + 1];             // bit q: a document starts at lo + q
  __shared__ uint32_t valid_s[WRITE ? kGramThreads : 1];  // 3-gram start masks, per thread
  __shared__ int32_t pre_s[WRITE ? kGramThreads : 1];     // exclusive 3-gram counts, per thread
  __shared__ int32_t warp_tot[kGramThreads / 32];
  __shared__ int32_t stage[WRITE ? kGramTile : 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t t = blockIdx.x;
  const int64_t lo = t * kGramTile;

  // 1. this thread's bytes; the document starts in [lo, lo + tile + 2)
  uint32_t w[9];
  load36(a, lo + 32 * tid, w);
  for (int x = tid; x <= kGramWords; x += kGramThreads) starts[x] = 0u;
  const int64_t first_doc = __ldg(a.tile_doc + t);
  const int64_t first_start = doc_start(a, first_doc + tid);
  const int64_t base = WRITE ? __ldg(a.tile_base + t) : 0;
  __syncthreads();
  const int64_t bound = lo + kGramTile + 2;
  for (int64_t d = first_doc + tid, s = first_start; s < bound;) {
    // (k_text_offsets validates the offsets; this guard only keeps invalid ones in bounds)
    if (s >= lo) atomicOr(&starts[(s - lo) >> 5], 1u << ((s - lo) & 31));
    d += kGramThreads;
    s = doc_start(a, d);
  }
  __syncthreads();

  // 2. position j starts a 3-gram iff bytes j, j+1, j+2 are letters and no document starts at
  //    j+1 or j+2
  uint32_t mb[9];
  uint64_t lm = 0ull;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    mb[k] = letter_bytes4(w[k]);
    lm |= (uint64_t)letter_bits4(mb[k]) << (4 * k);
  }
  const uint64_t sm = (uint64_t)starts[tid] | ((uint64_t)starts[tid + 1] << 32);
  const uint32_t valid = (uint32_t)(lm & (lm >> 1) & (lm >> 2) & ~(sm >> 1) & ~(sm >> 2));

  // 3. counts: thread prefix within the warp, warp prefix within the tile
  const int c = __popc(valid);
  int incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  int wbase = 0, total = 0;
#pragma unroll
  for (int x = 0; x < kGramThreads / 32; ++x) {
    const int tw = warp_tot[x];
    if (x < warp) wbase += tw;
    total += tw;
  }
  if (!WRITE) {
    if (tid == 0) {
      a.tile_cnt[t] = total;
      atomicAdd(a.group_sum + (t >> 10), (unsigned long long)total);
    }
    return;
  }
  const int pre = wbase + incl - c;
  pre_s[tid] = pre;
  valid_s[tid] = valid;

  // 4. ids into shared memory in text order, then one coalesced copy to the output
  uint32_t L[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) L[k] = letter_nums4(w[k], mb[k]);  // 0 for other bytes: lanes stay < 2^15
  // ids two at a time in 16-bit lanes (ids < 2^15, so the lanes never carry into each other):
  // for positions 4g + r, r = 0..3, with letter numbers n_0..n_5 of bytes 4g..4g+5,
  // even = 676 (n0, n2) + 26 (n1, n3) + (n2, n4) and odd = 676 (n1, n3) + 26 (n2, n4) + (n3, n5)
  int at = pre;
#pragma unroll
  for (int g = 0; g < 8; ++g) {
    const uint32_t a0 = __byte_perm(L[g], 0u, 0x4240);                   // (n0, n2)
    const uint32_t a1 = __byte_perm(L[g], 0u, 0x4341);                   // (n1, n3)
    const uint32_t a2 = __byte_perm(L[g], L[g + 1], 0x4442) & 0x00FF00FFu;  // (n2, n4)
    const uint32_t a3 = __byte_perm(L[g], L[g + 1], 0x4543) & 0x00FF00FFu;  // (n3, n5)
    const uint32_t ev = 676u * a0 + 26u * a1 + a2;
    const uint32_t od = 676u * a1 + 26u * a2 + a3;
    const uint32_t ids[4] = {ev & 0xFFFFu, od & 0xFFFFu, ev >> 16, od >> 16};
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if ((valid >> (4 * g + r)) & 1u) stage[at++] = (int32_t)ids[r];
  }
  __syncthreads();
  const int64_t lim = a.capacity - base;  // ids past the caller's capacity are dropped
  for (int x = tid; x < total && x < lim; x += kGramThreads) a.grams[base + x] = stage[x];

  // 5. 3-gram offset of every document that starts in this tile (the last tile also takes the
  //    documents that start at the end of the text)
  const int64_t hi = min(lo + (int64_t)kGramTile, a.n_bytes);
  const bool last = lo + kGramTile >= a.n_bytes;
  for (int64_t d = first_doc + tid, s = first_start; s < hi || (s == hi && last);) {
    if (s >= lo) {
      const int xq = (int)(s - lo);
      const int x = xq >> 5;
      const int64_t before = x >= kGramThreads ? total : pre_s[x] + __popc(valid_s[x] & ((1u << (xq & 31)) - 1u));
      a.gram_offsets[d] = base + before;
    }
    d += kGramThreads;
    s = doc_start(a, d);
  }
}

// Checks text_offsets (offsets[0] = 0, non-decreasing, offsets[n_docs] = n_bytes) and fills
// tile_doc[t] = the first document whose start is >= t * tile: document d takes the tiles whose
// first byte lies in (offsets[d-1], offsets[d]]. Entries stay 0 where invalid offsets leave gaps.
__global__ void k_text_offsets(const int64_t* off, int64_t n_docs, int64_t n_bytes, int64_t tiles,
                               int64_t* tile_doc, int32_t* err) {
  const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (d > n_docs) return;
  const int64_t s = off[d];
  if ((d == 0 && s != 0) || s < 0 || s > n_bytes || (d < n_docs && off[d + 1] < s)) atomicOr(err, kErrBadOffsets);
  const int64_t prev = d == 0 ? -1 : off[d - 1];
  if (s < 0 || prev >= s) return;
  const int64_t t1 = min(s / kGramTile, tiles - 1);
  for (int64_t t = (prev + kGramTile) / kGramTile; t <= t1; ++t) tile_doc[t] = d;  // (prev, s] holds t * tile
}

// Inclusive sum of v over the threads of a 1,024-thread CTA, in thread order (one barrier pair).
__device__ __forceinline__ int64_t cta_incl_scan_1024(int64_t v, int64_t* warp_sum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) warp_sum[warp] = v;
  __syncthreads();
  int64_t wb = 0;
  for (int x = 0; x < warp; ++x) wb += warp_sum[x];
  __syncthreads();
  return wb + v;
}

// CTA g scans the tile counts of group g (tiles [1024 g, 1024 g + 1024)), starting from the sum
// of the earlier groups' totals (group_sum, added by the count pass): base[t] = sum of
// cnt[0..t), base[n] = the total.
__global__ void __launch_bounds__(1024) k_tile_scan(const int32_t* cnt, int64_t n, const int64_t* group_sum,
                                                    int64_t* base) {
  __shared__ int64_t warp_sum[32];
  const int64_t g = blockIdx.x;
  int64_t before = 0;
  for (int64_t h = threadIdx.x; h < g; h += 1024) before += group_sum[h];
  const int64_t before_incl = cta_incl_scan_1024(before, warp_sum);
  __shared__ int64_t gbase;  // the CTA total of `before`: the last thread's inclusive sum
  if (threadIdx.x == 1023) gbase = before_incl;
  __syncthreads();
  const int64_t t = g * 1024 + threadIdx.x;
  const int64_t v = t < n ? cnt[t] : 0;
  const int64_t incl = cta_incl_scan_1024(v, warp_sum) + gbase;
  if (t < n) base[t] = incl - v;
  if (t == n - 1) base[n] = incl;
}

}  // namespace

int64_t text_gram_tiles(int64_t n_bytes) { return (n_bytes + kGramTile - 1) / kGramTile; }

cudaError_t launch_text_grams(mrc_ctx* ctx, int64_t n_docs, const int64_t* text_offsets, const uint8_t* text,
                              int64_t n_bytes, int64_t* gram_offsets, int32_t* grams, int64_t capacity,
                              int64_t* tile_doc, int32_t* tile_cnt, int64_t* group_sum, int64_t* tile_base,
                              int32_t* err) {
  const int64_t tiles = text_gram_tiles(n_bytes), groups = (tiles + 1023) / 1024;
  if (tiles > 0) {
    cudaError_t e = cudaMemsetAsync(tile_doc, 0, sizeof(int64_t) * (size_t)tiles, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(group_sum, 0, sizeof(int64_t) * (size_t)groups, ctx->stream);
    if (e != cudaSuccess) return e;
  }
  {
    KernelTimer kt(ctx, "text_offsets", 8.0 * (double)(n_docs + 1) + 8.0 * (double)tiles);
    k_text_offsets<<<(unsigned)((n_docs + 256) / 256), 256, 0, ctx->stream>>>(text_offsets, n_docs, n_bytes, tiles,
                                                                             tile_doc, err);
  }
  if (tiles == 0) {  // no text: every document has no 3-gram
    cudaError_t e = cudaMemsetAsync(gram_offsets, 0, sizeof(int64_t) * (size_t)(n_docs + 1), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(tile_base, 0, sizeof(int64_t), ctx->stream);
    return e;
  }
  if (tiles >= (1ll << 31)) return cudaErrorInvalidValue;
  GramArgs a{n_docs, text_offsets, text, n_bytes, gram_offsets, grams, capacity, tile_doc, tile_cnt,
             reinterpret_cast<unsigned long long*>(group_sum), tile_base, err,
             (reinterpret_cast<uintptr_t>(text) & 15u) == 0};
  {
    KernelTimer kt(ctx, "text_grams_count", (double)n_bytes + 4.0 * (double)tiles);
    k_text_grams<false><<<(unsigned)tiles, kGramThreads, 0, ctx->stream>>>(a);
  }
  {
    KernelTimer kt(ctx, "tile_scan", 12.0 * (double)tiles);
    k_tile_scan<<<(unsigned)groups, 1024, 0, ctx->stream>>>(tile_cnt, tiles, group_sum, tile_base);
  }
  // the write pass's algorithmic bytes: the text, 4 per 3-gram (at most one per byte, counted
  // as the bytes of the text here; the exact count is known only on the device), the offsets
  KernelTimer kt(ctx, "text_grams_write", 5.0 * (double)n_bytes + 16.0 * (double)(n_docs + 1));
  k_text_grams<true><<<(unsigned)tiles, kGramThreads, 0, ctx->stream>>>(a);
  return cudaGetLastError();
}

}  // namespace mrc
