// ingest.cu -- per-document passes over a token CSR (rows a1-a4 of the hot path).
//
// Every pass first turns a document's tokens into its bag of terms: the
// vector space model of Section III counts each term (3-gram id) of the
// document. The bag is built in shared memory as an open-addressing hash
// table (term -> count), by one warp for short documents and by one CTA for
// long ones; documents whose distinct terms could exceed half the CTA table
// are split into several passes by a second hash of the term id.
//
// Then, per distinct term t with count c, one of three things happens:
//   DF   : df[t] += 1                             (index build, Section IV ranking)
//   SIG  : w = c * idf(t);  |d|^2 += w^2;  num[part(t)] += w * r_t  (Eq. 1 against
//          each reference partition, Section IV), and the Simhash column sums of
//          Section III: sum over the term's occurrences of (+1 bit set, -1 clear)
//   DENSE: w/|d| goes to the exact-cosine operands (dense head columns or sparse
//          tail postings; see cosine_allpairs)
//
// Determinism: per-term contributions are computed in FP32 (a function of the
// term and its count only) and summed as 2^-22 fixed-point integers, so the
// result does not depend on the order in which threads meet the terms. Every
// contribution is >= 1 (counts >= 1, idf >= 1), so the rounding to the grid
// costs at most 2^-23 relative.
//
// Simhash column sums use a bit transpose: a warp holds 32 terms' 64-bit
// hashes, transposes them so that lane j holds bit j (and j+32) of all 32, and
// adds popc(bits & count-bit-plane) << plane. A column is positive iff
// 2 * (sum of counts whose hash bit is set) > document length.
#include <cuda_bf16.h>
#include <algorithm>
#include <string>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "device.cuh"
#include "ingest_dev.cuh"
#include "internal.h"

namespace mrc {
namespace {

// The paper's feature hashes (Section III hashes words with MD5 or SHA1): MD5 (RFC 1321) or
// SHA-1 (FIPS 180-4) of a 12-byte message, term t as a 32-bit little-endian word followed by
// the seed as a 64-bit little-endian word; the feature is the first 8 digest bytes read as a
// little-endian word. A 12-byte message is one padded block: the 0x80 byte follows it, then
// zeros, then the bit length 96 in the last 8 bytes (little-endian for MD5, big-endian for
// SHA-1). Computed once per vocabulary term (k_feature_table) and gathered per term.
__constant__ uint32_t kMd5Add[64] = {  // floor(2^32 |sin(i)|), i = 1..64
    0xD76AA478u, 0xE8C7B756u, 0x242070DBu, 0xC1BDCEEEu, 0xF57C0FAFu, 0x4787C62Au, 0xA8304613u, 0xFD469501u,
    0x698098D8u, 0x8B44F7AFu, 0xFFFF5BB1u, 0x895CD7BEu, 0x6B901122u, 0xFD987193u, 0xA679438Eu, 0x49B40821u,
    0xF61E2562u, 0xC040B340u, 0x265E5A51u, 0xE9B6C7AAu, 0xD62F105Du, 0x02441453u, 0xD8A1E681u, 0xE7D3FBC8u,
    0x21E1CDE6u, 0xC33707D6u, 0xF4D50D87u, 0x455A14EDu, 0xA9E3E905u, 0xFCEFA3F8u, 0x676F02D9u, 0x8D2A4C8Au,
    0xFFFA3942u, 0x8771F681u, 0x6D9D6122u, 0xFDE5380Cu, 0xA4BEEA44u, 0x4BDECFA9u, 0xF6BB4B60u, 0xBEBFBC70u,
    0x289B7EC6u, 0xEAA127FAu, 0xD4EF3085u, 0x04881D05u, 0xD9D4D039u, 0xE6DB99E5u, 0x1FA27CF8u, 0xC4AC5665u,
    0xF4292244u, 0x432AFF97u, 0xAB9423A7u, 0xFC93A039u, 0x655B59C3u, 0x8F0CCC92u, 0xFFEFF47Du, 0x85845DD1u,
    0x6FA87E4Fu, 0xFE2CE6E0u, 0xA3014314u, 0x4E0811A1u, 0xF7537E82u, 0xBD3AF235u, 0x2AD7D2BBu, 0xEB86D391u,
};

__device__ __forceinline__ uint32_t rotl32(uint32_t x, int s) { return __funnelshift_l(x, x, s); }
__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0u, 0x0123); }

__device__ uint64_t md5_feature(uint32_t t, uint64_t seed) {
  uint32_t X[16] = {t, (uint32_t)seed, (uint32_t)(seed >> 32), 0x80u, 0u, 0u, 0u, 0u,
                    0u, 0u, 0u, 0u, 0u, 0u, 96u, 0u};
  const int shift[16] = {7, 12, 17, 22, 5, 9, 14, 20, 4, 11, 16, 23, 6, 10, 15, 21};
  uint32_t a = 0x67452301u, b = 0xEFCDAB89u, c = 0x98BADCFEu, d = 0x10325476u;
#pragma unroll
  for (int i = 0; i < 64; ++i) {
    const int r = i >> 4;
    uint32_t f;
    int g;
    if (r == 0) {
      f = (b & c) | (~b & d);
      g = i;
    } else if (r == 1) {
      f = (b & d) | (c & ~d);
      g = (1 + 5 * i) & 15;
    } else if (r == 2) {
      f = b ^ c ^ d;
      g = (5 + 3 * i) & 15;
    } else {
      f = c ^ (b | ~d);
      g = (7 * i) & 15;
    }
    const uint32_t nb = b + rotl32(a + f + X[g] + kMd5Add[i], shift[4 * r + (i & 3)]);
    a = d;
    d = c;
    c = b;
    b = nb;
  }
  // digest bytes 0..7 are the first two state words, little-endian
  return (uint64_t)(0x67452301u + a) | ((uint64_t)(0xEFCDAB89u + b) << 32);
}

__device__ uint64_t sha1_feature(uint32_t t, uint64_t seed) {
  uint32_t W[16] = {bswap32(t), bswap32((uint32_t)seed), bswap32((uint32_t)(seed >> 32)), 0x80000000u,
                    0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 96u};
  uint32_t a = 0x67452301u, b = 0xEFCDAB89u, c = 0x98BADCFEu, d = 0x10325476u, e = 0xC3D2E1F0u;
#pragma unroll
  for (int i = 0; i < 80; ++i) {
    uint32_t w;
    if (i < 16) {
      w = W[i];
    } else {  // message schedule in a 16-word ring
      w = rotl32(W[(i - 3) & 15] ^ W[(i - 8) & 15] ^ W[(i - 14) & 15] ^ W[i & 15], 1);
      W[i & 15] = w;
    }
    uint32_t f, kc;
    if (i < 20) {
      f = (b & c) ^ (~b & d);
      kc = 0x5A827999u;
    } else if (i < 40) {
      f = b ^ c ^ d;
      kc = 0x6ED9EBA1u;
    } else if (i < 60) {
      f = (b & c) ^ (b & d) ^ (c & d);
      kc = 0x8F1BBCDCu;
    } else {
      f = b ^ c ^ d;
      kc = 0xCA62C1D6u;
    }
    const uint32_t tmp = rotl32(a, 5) + f + e + kc + w;
    e = d;
    d = c;
    c = rotl32(b, 30);
    b = a;
    a = tmp;
  }
  // digest bytes 0..7 are the first two state words, big-endian
  return (uint64_t)bswap32(0x67452301u + a) | ((uint64_t)bswap32(0xEFCDAB89u + b) << 32);
}

// One warp per document, documents taken one at a time from a device counter as warps free up
// (their lengths vary 100-fold). A pass that reads stored bags needs no table, so it takes
// every document here, the long-document list (longest first) before the short one; a hashing
// pass takes the short documents only (the long ones go to the group path).
// MINB: CTAs per SM the register budget is cut for (3 with 64-bit tables, 4 with 32-bit ones; 5
// for passes over stored bags, whose warps need little shared memory), so that as many
// documents as the shared memory holds are in flight. It also names the way the kernel takes
// (the one it is launched for): 5 stored bags, 4 32-bit tables, 3 64-bit tables.
template <int MODE, int MINB>
__global__ void __launch_bounds__(kWarpsShort * 32, MINB) k_ingest_short(IngestParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kq = ingest_kq<MODE>(p);
  uint8_t* base = smem + (p.bag_read ? bag_warp_bytes(kq) : short_warp_bytes(kq, p.narrow != 0)) * warp;
  const Transposer tr(lane);
  const int32_t n_short = p.list_counts[0];
  const int32_t n_long = p.bag_read ? p.list_counts[1] : 0;
  int32_t it = 0;
  if (lane == 0) it = atomicAdd(p.short_cursor, 1);
  it = __shfl_sync(kFull, it, 0);
  while (it < n_short + n_long) {
    int32_t next = 0;
    if (lane == 0) next = atomicAdd(p.short_cursor, 1);
    const int64_t d = it < n_long ? p.long_list[it] : p.short_list[it - n_long];
    warp_doc<MODE, MINB == 5 ? kVarBag : (MINB == 4 ? kVarNarrow : kVarWide)>(p, d, base, kq, lane, tr);
    it = __shfl_sync(kFull, next, 0);
  }
  // This grid may start while the long-document grid (launched just before it) is still
  // running; it completes only after that grid, so the next launch on the stream sees both.
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// G groups of kGroupThreads threads; NARROW: the groups' tables have 32-bit slots.
template <int MODE, int G, bool NARROW>
__global__ void __launch_bounds__(G * kGroupThreads, 1) k_ingest_long(IngestParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int32_t s_next, s_huge;
  constexpr int kThreads = G * kGroupThreads;
  const int g = threadIdx.x / kGroupThreads, gt = threadIdx.x % kGroupThreads;
  const int lane = threadIdx.x & 31;
  const int kq = ingest_kq<MODE>(p);
  const Transposer tr(lane);
  const int32_t n_long = p.list_counts[1];
  if (threadIdx.x == 0) {  // documents of kHugeMin tokens or more: length classes 2 and up, listed first
    int32_t h = 0;
    for (int c = 2; c < kLenClasses; ++c) h += p.list_counts[kCntClass + c];
    s_huge = h;
  }
  __syncthreads();
  const int32_t n_huge = s_huge;
  // the warp path's grid may start on SMs this grid leaves (the two touch disjoint documents)
  asm volatile("griddepcontrol.launch_dependents;");
  // The huge documents go to the groups (32-bit group tables only) when there are at least
  // four per CTA: then the pass is bound by throughput, and a whole CTA per document would leave
  // most of its warps waiting on one document's chain (half the groups' tokens per second).
  // With fewer, the longest document's latency bounds the pass, and a whole CTA takes it in
  // one hashing pass where a group would need up to ten.
  const bool huge_groups = NARROW && n_huge >= 4 * (int32_t)gridDim.x;
  // phase 1: the huge documents, one per CTA at a time
  while (!huge_groups) {
    if (threadIdx.x == 0) s_next = atomicAdd(p.huge_cursor, 1);
    __syncthreads();
    const int32_t it = s_next;
    __syncthreads();
    if (it >= n_huge) break;
    team_doc<MODE>(p, p.long_list[it], smem, kq, kHugeSlots, kThreads, 0, threadIdx.x, tr);
  }
  // phase 2: the other long documents, one per group at a time (the huge ones first when the
  // groups take them)
  uint8_t* base = smem + long_group_bytes(kq, NARROW) * g;
  int32_t* slot = reinterpret_cast<int32_t*>(base + (size_t)kq * 8 + 16 + 64 * 4);  // misc[0] of the group
  while (true) {
    if (gt == 0) *slot = (huge_groups ? 0 : n_huge) + atomicAdd(p.long_cursor, 1);
    team_sync(1 + g, kGroupThreads);
    const int32_t it = *slot;
    if (it >= n_long) break;
    if (huge_groups && it < n_huge)
      team_doc<MODE, unsigned long long>(p, p.long_list[it], base, kq, kHugeGroupSlots, kGroupThreads, 1 + g, gt,
                                         tr);
    else
      team_doc<MODE, typename std::conditional<NARROW, uint32_t, unsigned long long>::type>(
          p, p.long_list[it], base, kq, kLongSlots, kGroupThreads, 1 + g, gt, tr);
  }
}

// (length classes: see the long-document path)
__device__ __forceinline__ int len_class(int64_t len) {
  int c = 0;
  while (c < kLenClasses - 1 && len >= (2ll << (9 + c))) ++c;
  return c;
}



// Splits documents into the warp path (appended to short_list) and the CTA path (counted per
// length class); validates offsets.
__global__ void k_classify(const int64_t* off, int64_t n, int32_t* short_list, int32_t* counts, int32_t* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  if (i == 0 && off[0] != 0) set_err(err, kErrBadOffsets);
  int64_t len = i < n ? off[i + 1] - off[i] : 0;
  if (i < n && len < 0) set_err(err, kErrBadOffsets);
  if (i < n && len > MRC_MAX_DOC_TOKENS) set_err(err, kErrTooLong);
  const bool ok = i < n && len >= 0 && len <= MRC_MAX_DOC_TOKENS;
  if (!ok) len = 0;
  // one atomic per warp for the longest length and for the short-list appends
  int32_t mx = (int32_t)len;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(kFull, mx, o));
  if (lane == 0 && mx > 0) atomicMax(&counts[kCntMaxLen], mx);
  const bool is_short = ok && len <= kShortMax;
  const unsigned sm = __ballot_sync(kFull, is_short);
  int32_t base = 0;
  if (lane == 0 && sm) base = atomicAdd(&counts[kCntShort], __popc(sm));
  base = __shfl_sync(kFull, base, 0);
  if (is_short) short_list[base + __popc(sm & ((1u << lane) - 1u))] = (int32_t)i;
  if (ok && !is_short) {
    atomicAdd(&counts[kCntLong], 1);
    atomicAdd(&counts[kCntClass + len_class(len)], 1);
  }
}

// Places the CTA-path documents in long_list, longer length classes first, so that the
// longest documents start first and the short ones fill in behind them.
__global__ void k_place_long(const int64_t* off, int64_t n, int32_t* long_list, int32_t* counts) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t len = off[i + 1] - off[i];
  if (len <= kShortMax || len > MRC_MAX_DOC_TOKENS) return;
  const int c = len_class(len);
  int32_t base = 0;
  for (int q = kLenClasses - 1; q > c; --q) base += counts[kCntClass + q];
  long_list[base + atomicAdd(&counts[kCntClassFill + c], 1)] = (int32_t)i;
}

void launch_classify(mrc_ctx* ctx, const int64_t* off, int64_t n, int32_t* short_list, int32_t* long_list,
                     int32_t* counts, int32_t* err) {
  const unsigned blocks = (unsigned)((n + 255) / 256);
  {
    KernelTimer kt(ctx, "classify", 8.0 * (double)(n + 1));
    k_classify<<<blocks, 256, 0, ctx->stream>>>(off, n, short_list, counts, err);
  }
  KernelTimer kt(ctx, "place_long", 8.0 * (double)(n + 1));
  k_place_long<<<blocks, 256, 0, ctx->stream>>>(off, n, long_list, counts);
}

__global__ void k_idf(int64_t n_docs, const int32_t* df, int32_t vocab, int32_t weighting, float* idf,
                      TermInfo* tinfo) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= vocab) return;
  // idf(t) = ln((1 + N) / (1 + df(t))) + 1, evaluated in double
  const double v = log((1.0 + (double)n_docs) / (1.0 + (double)df[t])) + 1.0;
  idf[t] = (float)v;
  if (tinfo) {
    tinfo[t].idf = weighting == MRC_WEIGHT_TFIDF ? (float)v : 1.0f;
    tinfo[t].code = -1;
  }
}

// Unit-length packing of raw signatures (query signatures handed to mrc_match).
__global__ void k_pack(const float* sig, int64_t n, int32_t k, int32_t normalize, void* hi, void* lo, void* e4m3,
                       float* qnorm, float* unit, int32_t kp, int32_t kp8) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int64_t d = warp;
  float ss = 0.f;
  for (int q = lane; q < k; q += 32) {
    const float v = sig[d * k + q];
    ss += v * v;
  }
  ss = warp_sum(ss);
  const float nrm = sqrtf(ss);
  const int width = max(k, max(kp, kp8));
  float q2 = 0.f;
  for (int q = lane; q < width; q += 32) {
    const float u = q < k ? (normalize ? (nrm > 0.f ? sig[d * k + q] / nrm : 0.f) : sig[d * k + q]) : 0.f;
    if (unit && q < k) unit[d * k + q] = u;
    if (hi && q < kp) {
      const __half h = __float2half_rn(u);
      reinterpret_cast<__half*>(hi)[d * kp + q] = h;
      if (lo) reinterpret_cast<__half*>(lo)[d * kp + q] = __float2half_rn((u - __half2float(h)) * kSplitLoScale);
    }
    if (e4m3 && q < kp8) {
      const __nv_fp8_storage_t e = __nv_cvt_float_to_fp8(u * kE4M3Scale, __NV_SATFINITE, __NV_E4M3);
      reinterpret_cast<uint8_t*>(e4m3)[d * kp8 + q] = (uint8_t)e;
      const float v = __half2float(__half(__nv_cvt_fp8_to_halfraw(e, __NV_E4M3))) * (1.0f / kE4M3Scale);
      q2 += v * v;
    }
  }
  if (qnorm) {
    q2 = warp_sum(q2);
    if (lane == 0) qnorm[d] = sqrtf(q2);
  }
}

// Persistent grids: as many CTAs as fit on every SM at once (0: the shared memory limit could
// not be raised).
template <int MODE, int MINB>
int short_grid(const mrc_ctx* ctx, size_t smem) {
  return ctx->num_sms * resident_ctas(k_ingest_short<MODE, MINB>, kWarpsShort * 32, smem);
}
template <int MODE, bool NARROW>
int long_grid(const mrc_ctx* ctx, size_t smem) {
  constexpr int G = long_groups(MODE, NARROW);
  return ctx->num_sms * resident_ctas(k_ingest_long<MODE, G, NARROW>, G * kGroupThreads, smem);
}

size_t short_smem(int kq, bool bag, bool narrow) {
  return (size_t)kWarpsShort * (bag ? bag_warp_bytes(kq) : short_warp_bytes(kq, narrow));
}
template <int MODE, bool NARROW>
size_t long_smem(int kq) {
  return std::max((size_t)long_groups(MODE, NARROW) * long_group_bytes(kq, NARROW), long_huge_bytes(kq));
}

// The long-document grid (persistent: as many CTAs as fit, at most `cap`), narrow or wide tables.
template <int MODE, bool NARROW>
cudaError_t launch_long_as(mrc_ctx* ctx, const IngestParams& p, int kq, int64_t cap) {
  constexpr int G = long_groups(MODE, NARROW);
  const size_t smem = long_smem<MODE, NARROW>(kq);
  int grid = long_grid<MODE, NARROW>(ctx, smem);
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  if (cap < grid) grid = (int)cap;
  k_ingest_long<MODE, G, NARROW><<<grid, G * kGroupThreads, smem, ctx->stream>>>(p);
  return cudaGetLastError();
}
template <int MODE>
cudaError_t launch_long(mrc_ctx* ctx, const IngestParams& p, int kq, int64_t cap) {
  return p.narrow ? launch_long_as<MODE, true>(ctx, p, kq, cap) : launch_long_as<MODE, false>(ctx, p, kq, cap);
}

template <int MODE>
cudaError_t run_ingest(mrc_ctx* ctx, const DocsDev& d, IngestParams p, const char* name, double bytes_per_token,
                       double bytes_per_doc) {
  // Lists and counters stay on the device: both paths read their list sizes there, so no
  // host round trip is needed. Offsets/length errors land in the call's error word.
  mrc_status st = MRC_OK;
  const size_t list_bytes = sizeof(int32_t) * (size_t)std::max<int64_t>(d.n_docs, 1);
  int32_t* short_list = (int32_t*)ws_get(ctx, "ingest.short", list_bytes, &st);
  int32_t* long_list = (int32_t*)ws_get(ctx, "ingest.long", list_bytes, &st);
  int32_t* counts = (int32_t*)ws_get(ctx, "ingest.counts", sizeof(int32_t) * kCntWords, &st);
  if (st != MRC_OK) return cudaErrorMemoryAllocation;
  if (d.n_docs <= 0) return cudaSuccess;
  cudaError_t e;
  if (d.lists_ready) {  // the lists of the previous pass over these documents: reset the cursors
    e = cudaMemsetAsync(counts + kCntLongCursor, 0, sizeof(int32_t) * 3, ctx->stream);
    if (e != cudaSuccess) return e;
  } else {
    e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * kCntWords, ctx->stream);
    if (e != cudaSuccess) return e;
    launch_classify(ctx, d.offsets, d.n_docs, short_list, long_list, counts, d.err);
  }
  p.short_list = short_list;
  p.long_list = long_list;
  p.list_counts = counts;
  p.long_cursor = counts + kCntLongCursor;
  p.short_cursor = counts + kCntShortCursor;
  p.huge_cursor = counts + kCntHugeCursor;
  p.err = d.err;
  p.narrow = narrow_slots(p.vocab) ? 1 : 0;
  const int kq = ingest_kq<MODE>(p);
  const size_t s_smem = short_smem(kq, p.bag_read != 0, p.narrow != 0);
  const double tokens = (double)d.n_tokens;
  cudaEvent_t ev = nullptr;
  // The CTA path (longest documents first) is launched first; the warp path follows as a
  // programmatic dependent launch, so its CTAs fill SMs as the CTA path's grid drains instead
  // of waiting for the whole grid. Not while the stream is being captured into a graph.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(ctx->stream, &cap);
  const bool overlap = cap == cudaStreamCaptureStatusNone && !ctx->timing;
  if (!p.bag_read) {  // a pass over stored bags takes every document in the warp path
    std::string nm = std::string(name) + ".long";
    timing_begin(ctx, nm.c_str(), 0.0, 0.0, &ev);
    e = launch_long<MODE>(ctx, p, kq, d.n_docs);
    timing_end(ctx, ev);
    if (e != cudaSuccess) return e;
  }
  {
    // CTAs per SM: five over stored bags, four with 32-bit tables, three with 64-bit ones
    int grid = p.bag_read ? short_grid<MODE, 5>(ctx, s_smem)
                          : (p.narrow ? short_grid<MODE, 4>(ctx, s_smem) : short_grid<MODE, 3>(ctx, s_smem));
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    const int64_t need = (d.n_docs + kWarpsShort - 1) / kWarpsShort;
    if (need < grid) grid = (int)need;
    std::string nm = std::string(name) + ".short";
    timing_begin(ctx, nm.c_str(), tokens * bytes_per_token + bytes_per_doc * d.n_docs, 0.0, &ev);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kWarpsShort * 32);
    cfg.dynamicSmemBytes = s_smem;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap && !p.bag_read ? 1 : 0;
    e = p.bag_read ? cudaLaunchKernelEx(&cfg, k_ingest_short<MODE, 5>, p)
                   : (p.narrow ? cudaLaunchKernelEx(&cfg, k_ingest_short<MODE, 4>, p)
                               : cudaLaunchKernelEx(&cfg, k_ingest_short<MODE, 3>, p));
    timing_end(ctx, ev);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

IngestParams base_params(const DocsDev& d) {
  IngestParams p{};
  p.offsets = d.offsets;
  p.tokens = d.tokens;
  if (d.bag_terms && d.bag_cnts && d.bag_n) {
    p.bag_terms = d.bag_terms;
    p.bag_cnts = d.bag_cnts;
    p.bag_n = d.bag_n;
    p.bag_write = d.bag_write;
    p.bag_read = d.bag_read && !d.bag_write;
  }
  return p;
}

}  // namespace

cudaError_t launch_df(mrc_ctx* ctx, const DocsDev& d, int32_t* df, int32_t vocab) {
  IngestParams p = base_params(d);
  p.vocab = vocab;
  p.df = df;
  return run_ingest<kDF>(ctx, d, p, "ingest_df", 4.0, 8.0);
}

cudaError_t launch_df_norm(mrc_ctx* ctx, const DocsDev& d, int32_t* df, int32_t vocab, const float* idf,
                           unsigned long long* norm) {
  IngestParams p = base_params(d);
  p.vocab = vocab;
  p.df = df;
  p.norm_idf = idf;
  p.norm_out = norm;
  return run_ingest<kDFN>(ctx, d, p, "ingest_df_norm", 4.0, 16.0);
}

__global__ void k_term_info(const float* idf, const int32_t* part, int32_t vocab, int32_t tfidf, int32_t bf16,
                            TermInfo* tinfo) {
  const int32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= vocab) return;
  float w = 1.0f;
  if (tfidf) w = bf16 ? __bfloat162float(__float2bfloat16_rn(idf[t])) : idf[t];
  tinfo[t].idf = w;
  tinfo[t].code = part[t];
}

cudaError_t launch_term_info(mrc_ctx* ctx, const float* idf, const int32_t* part, int32_t vocab, int32_t tfidf,
                             int32_t bf16, TermInfo* tinfo) {
  KernelTimer kt(ctx, "term_info", 16.0 * vocab);
  k_term_info<<<(vocab + 255) / 256, 256, 0, ctx->stream>>>(idf, part, vocab, tfidf, bf16, tinfo);
  return cudaGetLastError();
}

__global__ void k_feature_table(int32_t vocab, uint64_t seed, int32_t mode, uint64_t* out) {
  const int32_t t = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
  if (t >= vocab) return;
  out[t] = mode == MRC_HASH_SHA1 ? sha1_feature((uint32_t)t, seed) : md5_feature((uint32_t)t, seed);
}

cudaError_t launch_feature_table(mrc_ctx* ctx, int32_t vocab, uint64_t seed, int32_t mode, uint64_t* out) {
  if (vocab <= 0) return cudaSuccess;
  KernelTimer kt(ctx, "feature_table", 8.0 * vocab);
  k_feature_table<<<(vocab + 255) / 256, 256, 0, ctx->stream>>>(vocab, seed, mode, out);
  return cudaGetLastError();
}

cudaError_t launch_idf(mrc_ctx* ctx, int64_t n_docs, const int32_t* df, int32_t vocab, int32_t weighting, float* idf,
                       TermInfo* tinfo) {
  KernelTimer kt(ctx, "idf", 8.0 * vocab);
  k_idf<<<(vocab + 255) / 256, 256, 0, ctx->stream>>>(n_docs, df, vocab, weighting, idf, tinfo);
  return cudaGetLastError();
}

cudaError_t launch_signature(mrc_ctx* ctx, const DocsDev& d, int32_t vocab, const TermInfo* tinfo,
                             const float* rinv, const float* rinv16, int32_t k, uint64_t seed, const uint64_t* fhash,
                             const SigOut& out) {
  IngestParams p = base_params(d);
  p.vocab = vocab;
  p.tinfo = tinfo;
  p.rinv = rinv;
  p.k = k;
  p.bf16w = rinv16 && out.op_e4m3 ? 1 : 0;
  p.rinv16 = rinv16;
  p.seed = seed;
  p.fhash = fhash;
  p.sig = out;
  return run_ingest<kSIG>(ctx, d, p, "signature", 4.0, 8.0 + 4.0 * k + 8.0);
}

cudaError_t launch_pack(mrc_ctx* ctx, const float* sig, int64_t n, int32_t k, int32_t normalize, void* hi, void* lo,
                        void* e4m3, float* qnorm, float* unit, int32_t kp, int32_t kp8) {
  if (n <= 0) return cudaSuccess;
  const int64_t threads = n * 32;
  KernelTimer kt(ctx, "pack", 8.0 * (double)n * k);
  k_pack<<<(unsigned)((threads + 255) / 256), 256, 0, ctx->stream>>>(sig, n, k, normalize, hi, lo, e4m3, qnorm,
                                                                      unit, kp, kp8);
  return cudaGetLastError();
}

__global__ void k_block_min(const float* norm, int64_t n, float* out) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b * 128 >= n) return;
  float m = __int_as_float(0x7f800000);
  for (int x = lane; x < 128; x += 32) {
    const int64_t j = b * 128 + x;
    if (j < n && norm[j] > 0.f) m = fminf(m, norm[j]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(kFull, m, o));
  if (lane == 0) out[b] = m == __int_as_float(0x7f800000) ? 1.0f : m;
}

cudaError_t launch_block_min(mrc_ctx* ctx, const float* norm, int64_t n, float* out) {
  const int64_t blocks = (n + 127) / 128;
  if (blocks <= 0) return cudaSuccess;
  KernelTimer kt(ctx, "block_min", 4.0 * (double)n);
  k_block_min<<<(unsigned)((blocks * 32 + 255) / 256), 256, 0, ctx->stream>>>(norm, n, out);
  return cudaGetLastError();
}

cudaError_t launch_densify(mrc_ctx* ctx, const DocsDev& d, int32_t vocab, const TermInfo* tinfo,
                           const DenseOut& out) {
  IngestParams p = base_params(d);
  p.vocab = vocab;
  p.tinfo = tinfo;
  p.dense = out;
  return run_ingest<kDENSE>(ctx, d, p, "densify", 4.0, 8.0);
}

}  // namespace mrc

namespace mrc {

// Signature pass whose scratch (document lists, counters, error word) is supplied by the
// caller instead of the context's workspace. lists: [2 * cap] int32; counts: [32] int32;
// err: [1] int32; all device memory, n_docs <= cap. *host_err receives the error word.
cudaError_t launch_signature_scratch(mrc_ctx* ctx, const DocsDev& d, int32_t vocab, const TermInfo* tinfo,
                                     const float* rinv, int32_t k, uint64_t seed,
                                     const uint64_t* fhash,
                                     const SigOut& out, int32_t* lists, int64_t cap, int32_t* counts, int32_t* err,
                                     int32_t* host_err) {
  *host_err = 0;
  if (d.n_docs > cap || d.n_docs < 0) return cudaErrorInvalidValue;
  IngestParams p = base_params(d);
  p.vocab = vocab;
  p.tinfo = tinfo;
  p.rinv = rinv;
  p.k = k;
  p.bf16w = 0;
  p.seed = seed;
  p.fhash = fhash;
  p.sig = out;
  int32_t* short_list = lists;
  int32_t* long_list = lists + cap;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * kCntWords, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), ctx->stream);
  if (e != cudaSuccess) return e;
  if (d.n_docs > 0) launch_classify(ctx, d.offsets, d.n_docs, short_list, long_list, counts, err);
  int32_t h[5] = {0, 0, 0, 0, 0};
  e = cudaMemcpyAsync(h, counts, sizeof(int32_t) * 4, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h + 4, err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (h[4] != 0) {
    *host_err = h[4];
    return cudaSuccess;
  }
  p.short_list = short_list;
  p.long_list = long_list;
  p.list_counts = counts;
  p.long_cursor = counts + kCntLongCursor;
  p.short_cursor = counts + kCntShortCursor;
  p.huge_cursor = counts + kCntHugeCursor;
  p.err = err;
  p.narrow = narrow_slots(p.vocab) ? 1 : 0;
  const size_t s_smem = short_smem(k, false, p.narrow != 0);
  if (h[0] > 0) {
    int grid = p.narrow ? short_grid<kSIG, 4>(ctx, s_smem) : short_grid<kSIG, 3>(ctx, s_smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    const int need = (h[0] + kWarpsShort - 1) / kWarpsShort;
    if (need < grid) grid = need;
    if (p.narrow)
      k_ingest_short<kSIG, 4><<<grid, kWarpsShort * 32, s_smem, ctx->stream>>>(p);
    else
      k_ingest_short<kSIG, 3><<<grid, kWarpsShort * 32, s_smem, ctx->stream>>>(p);
  }
  if (h[1] > 0) {
    e = launch_long<kSIG>(ctx, p, k, h[1]);
    if (e != cudaSuccess) return e;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(h + 4, err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return e;
  *host_err = h[4];
  return cudaSuccess;
}

}  // namespace mrc

namespace mrc {
namespace {

// Throughput probe of the bag-of-terms tables' bounding operation: every thread keeps eight
// 64-bit shared-memory atomic adds to distinct slots of a 4,096-slot table in flight, so the
// loop runs at the rate the SMs complete shared-memory 64-bit atomics. Hashing a token takes at
// least one such atomic (a claim or an increment). The table's sum is kept live through a
// store that never happens for these inputs.
constexpr int kAtomSlots = 4096;
__global__ void __launch_bounds__(256) k_smem_atomic_rate(int32_t iters, unsigned long long* sink) {
  __shared__ unsigned long long tab[kAtomSlots];
  for (int s = threadIdx.x; s < kAtomSlots; s += blockDim.x) tab[s] = 0ull;
  __syncthreads();
  for (int32_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 8; ++u) atomicAdd(&tab[(threadIdx.x + 256 * u + 2048 * (it & 1)) & (kAtomSlots - 1)], 1ull);
  }
  __syncthreads();
  if (tab[threadIdx.x] == 0xFFFFFFFFFFFFFFFFull) *sink = tab[threadIdx.x];  // each slot ends at iters
}

}  // namespace

cudaError_t measure_smem_atomic_rate(mrc_ctx* ctx, double* atomics_per_s) {
  constexpr int32_t kIters = 2048;
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
    k_smem_atomic_rate<<<(unsigned)blocks, 256, 0, ctx->stream>>>(kIters, sink);
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
  *atomics_per_s = (double)blocks * 256.0 * 8.0 * kIters / (best_ms * 1e-3);
  return cudaStreamSynchronize(ctx->stream);
}

}  // namespace mrc
