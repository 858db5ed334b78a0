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
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

constexpr uint32_t kEmpty = 0xFFFFFFFFu;
constexpr int kShortMax = 512;      // documents up to this length take the warp path
constexpr int kShortSlots = 1024;   // per-warp table (load <= 1/2)
constexpr int kWarpsShort = 7;      // warps per CTA in the warp path (three CTAs per SM)
constexpr int kShortRegs = kShortMax / 32;  // tokens (then terms) per lane held in registers (warp path)
constexpr int kGroupWarps = 4;      // warps per document group of the long-document path
constexpr int kGroupThreads = kGroupWarps * 32;
constexpr int kGroupsLong = 5;      // groups per CTA (one CTA per SM: five tables fill shared memory)
constexpr int kLongThreads = kGroupsLong * kGroupThreads;
constexpr int kLongSlots = 4096;    // per-group table: documents with > 2048 tokens take several passes
constexpr int kLongUnroll = 4;      // token loads per thread in flight (long-document path)
constexpr float kFix = 4194304.0f;  // 2^22
constexpr float kInvFix = 1.0f / 4194304.0f;

enum Mode { kDF = 0, kSIG = 1, kDENSE = 2, kDFN = 3 };

__device__ __forceinline__ uint32_t slot_of(uint32_t t, int log2ts) { return (t * 0x9E3779B1u) >> (32 - log2ts); }
__device__ __forceinline__ uint32_t pass_of(uint32_t t, uint32_t passes) {
  return ((t * 0x85EBCA77u) >> 7) % passes;
}

// SplitMix64 (Steele, Lea, Flood 2014), one step from state (t XOR seed).
__device__ __forceinline__ uint64_t feature_hash(uint32_t t, uint64_t seed) {
  uint64_t z = ((uint64_t)t ^ seed) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

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

// 32x32 bit-matrix transpose across a warp: on entry lane r holds row r (bit c = element
// (r, c)); on exit lane r holds column r of the input. Five exchange steps of distance
// s = 16, 8, 4, 2, 1: the lane whose bit s is clear keeps the bits of mask m_s and takes its
// partner's other bits shifted up by s; the other lane keeps ~m_s and takes its partner's bits
// shifted down. Both shifts are one rotation (by s or 32 - s; the bits that wrap around fall
// outside the taken mask), so a step is a shuffle, a funnel rotation and one three-input
// logic operation with per-lane constants computed once.
struct Transposer {
  uint32_t keep[5], rot[5];
  __device__ __forceinline__ explicit Transposer(int lane) {
    const uint32_t masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const uint32_t st = 16u >> i;
      const bool up = (lane & st) != 0;
      keep[i] = up ? ~masks[i] : masks[i];
      rot[i] = up ? 32u - st : st;
    }
  }
  __device__ __forceinline__ uint32_t operator()(uint32_t x) const {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      const uint32_t y = __shfl_xor_sync(kFull, x, 16 >> i);
      const uint32_t t = __funnelshift_l(y, y, rot[i]);
      x = (x & keep[i]) | (t & ~keep[i]);
    }
    return x;
  }
};

__device__ __forceinline__ unsigned long long to_fix(float x) { return __float2ull_rn(x * kFix); }

// 1 / |w| from the fixed-point squared norm (0 for an empty document).
// u^2 in 2^-31 fixed point, rounded up: FP32 with directed rounding (the power-of-two scaling
// is exact), so the bucket norms bound from above. A document's tail has sum u^2 <= 1, so a
// bucket's sum stays below 2^31 + 65,536 < 2^32.
__device__ __forceinline__ uint32_t to_fix31_up(float u) { return __float2uint_ru(__fmul_ru(u, u) * 2147483648.0f); }
__device__ __forceinline__ float inv_norm_of(unsigned long long norm_q) {
  const float n2 = (float)norm_q * kInvFix;
  return n2 > 0.f ? 1.0f / sqrtf(n2) : 0.f;
}

// Open-addressing table of a document's bag of terms: 64-bit slots, term id in the high word
// and its count in the low word (kEmpty64: free). Inserts up to B tokens per lane (those whose
// bit is set in pend) with all of a round's compare-and-swaps in flight: a token whose slot is
// free claims it with count 1; a token that finds its own term adds 1 to the slot; otherwise
// it moves to the next slot (linear probing from the same start slot keeps concurrent inserts
// consistent, and slots are never freed). A token that claimed a slot is its term's first
// occurrence in the document: the slot goes to the document's list of occupied slots (one
// shared-memory counter, so later passes walk only occupied slots) and, with df, the term's
// document frequency gets its 1. Returns false if a term found no slot.
constexpr unsigned long long kEmpty64 = 0xFFFFFFFF00000000ull;
template <int B>
__device__ __forceinline__ bool insert_batch(unsigned long long* tab, uint16_t* list, int32_t* list_n, int log2ts,
                                             const int32_t (&tk)[B], uint32_t pend, int32_t* df) {
  const uint32_t mask = (1u << log2ts) - 1u;
  uint32_t slot[B];
#pragma unroll
  for (int u = 0; u < B; ++u) slot[u] = slot_of((uint32_t)tk[u], log2ts);
  uint32_t fresh = 0u;
  for (uint32_t round = 0; pend != 0u && round <= mask; ++round) {
    unsigned long long prev[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if ((pend >> u) & 1u) prev[u] = atomicCAS(&tab[slot[u]], kEmpty64, ((unsigned long long)(uint32_t)tk[u] << 32) | 1ull);
#pragma unroll
    for (int u = 0; u < B; ++u)
      if ((pend >> u) & 1u) {
        if (prev[u] == kEmpty64) {
          fresh |= 1u << u;
          pend &= ~(1u << u);
        } else if ((uint32_t)(prev[u] >> 32) == (uint32_t)tk[u]) {
          atomicAdd(&tab[slot[u]], 1ull);
          pend &= ~(1u << u);
        } else {
          slot[u] = (slot[u] + 1u) & mask;
        }
      }
  }
  if (fresh) {
    int at = atomicAdd(list_n, __popc(fresh));
#pragma unroll
    for (int u = 0; u < B; ++u)
      if ((fresh >> u) & 1u) {
        list[at++] = (uint16_t)slot[u];
        if (df) atomicAdd(&df[tk[u]], 1);
      }
  }
  return pend == 0u;
}

__device__ __forceinline__ int log2_slots(int64_t len, int max_log2) {
  int l = 6;  // at least 64 slots
  while (l < max_log2 && (1ll << l) < 2 * len) ++l;
  return l;
}

struct IngestParams {
  const int64_t* offsets;
  const int32_t* tokens;
  int32_t vocab;
  const int32_t* short_list;
  const int32_t* long_list;
  const int32_t* list_counts;  // [0] short, [1] long
  int32_t* long_cursor;        // dynamic grab of long documents (group path)
  int32_t* huge_cursor;        // dynamic grab of the longest documents (CTA-wide)
  int32_t* short_cursor;       // dynamic grab of short documents (one warp each)
  int32_t* err;
  // DF (and DFN: df plus squared norms)
  int32_t* df;
  const float* norm_idf;
  unsigned long long* norm_out;
  // SIG
  const TermInfo* tinfo;
  const float* rinv;
  int32_t k;
  int32_t bf16w;         // precision form: also the signature of bfloat16 weights, for the E4M3 operand
  const float* rinv16;   // [k] 1 / |R_p| of the bfloat16 reference weights (with bf16w)
  uint64_t seed;
  const uint64_t* fhash;  // [vocab] feature hashes (MD5 / SHA-1 modes); NULL: SplitMix64 of (t ^ seed)
  SigOut sig;
  // DENSE
  DenseOut dense;
  // Bag of terms of every document, (term, count) pairs at the document's token offsets and
  // the number of pairs per document: a pass with bag_write stores the bag it builds, a later
  // pass over the same documents with bag_read takes it instead of hashing the tokens again.
  int32_t* bag_terms;
  int32_t* bag_cnts;
  int32_t* bag_n;
  int32_t bag_write, bag_read;
};

// Shared-memory 64-bit accumulator words per document: SIG, one per reference partition; DENSE
// in the bound-pruned mode, one 32-bit sum per tail bucket (two per word).
template <int MODE>
__host__ __device__ __forceinline__ int ingest_kq(const IngestParams& p) {
  return MODE == kSIG ? (p.bf16w ? 2 * p.k : p.k) : (MODE == kDENSE && !p.dense.postings ? kTailBuckets / 2 : 0);
}

// Per-group accumulators of the SIG and DENSE modes.
struct Acc {
  unsigned long long norm, norm16;  // norm16: squared norm of the bfloat16-weight vector (bf16w)
  uint32_t plo, phi;
};

// Per-term table values a mode needs besides the term's count: SIG (reference weight, reference
// partition), DENSE (idf or 1, head column / -1 / for a tail term -3 - its posting slot), DFN
// (idf or 1). Loading them is the only global-memory access per term, so the warp path gathers
// them for a whole document at once and the CTA path one chunk ahead.
struct TermAux {
  float w;
  int32_t code;
  uint64_t h;  // feature hash from the table (signature pass with a hash table only)
};

// The Simhash feature of `key` from the hash table (signature pass with MD5 / SHA-1 features).
template <int MODE>
__device__ __forceinline__ uint64_t load_hash(const IngestParams& p, uint32_t key) {
  return (MODE == kSIG && p.fhash && key != kEmpty) ? __ldg(reinterpret_cast<const unsigned long long*>(p.fhash) + key)
                                                    : 0ull;
}

template <int MODE>
__device__ __forceinline__ TermAux load_aux(const IngestParams& p, uint32_t key) {
  TermAux x{1.0f, 0, 0ull};
  if (MODE == kSIG) {
    const int2 ti = __ldg(reinterpret_cast<const int2*>(p.tinfo) + key);
    x.w = __int_as_float(ti.x);
    x.code = ti.y;
  } else if (MODE == kDENSE) {
    if (p.dense.idf) x.w = __ldg(p.dense.idf + key);
    x.code = __ldg(p.dense.colmap + key);
    if (x.code == -2 && p.dense.postings) {  // a tail term: claim its posting slot now (slots < 2^31 - 64)
      const int64_t pos = p.dense.tail_start[key] + atomicAdd(&p.dense.tail_fill[key], 1);
      x.code = -3 - (int32_t)pos;
    }
  } else if (MODE == kDFN) {
    if (p.norm_idf) x.w = __ldg(p.norm_idf + key);
  }
  return x;
}

// The work of one warp-chunk of 32 terms (key == kEmpty: no term in this lane).
template <int MODE>
__device__ __forceinline__ void chunk(const IngestParams& p, uint32_t key, uint32_t c, TermAux aux,
                                      const Transposer& tr, unsigned long long* num_q, Acc& a, int64_t doc,
                                      float inv_norm, int32_t* row_cnt_s, int64_t row_base) {
  const bool valid = key != kEmpty;
  if (MODE == kDF || MODE == kDFN) {
    if (valid) {
      if (p.bag_read) atomicAdd(&p.df[key], 1);  // hashing passes count df at insertion
      if (MODE == kDFN) {
        const float w = (float)c * aux.w;
        a.norm += to_fix(w * w);
      }
    }
    return;
  }
  if (MODE == kSIG) {
    if (p.sig.simhash) {
      const uint64_t h = !valid ? 0ull : p.fhash ? aux.h : feature_hash(key, p.seed);
      const uint32_t hl = tr((uint32_t)h);
      const uint32_t hh = tr((uint32_t)(h >> 32));
      const uint32_t cmax = __reduce_max_sync(kFull, c);
      for (uint32_t b = 0; (cmax >> b) != 0u; ++b) {
        const uint32_t plane = __ballot_sync(kFull, (c >> b) & 1u);
        a.plo += (uint32_t)__popc(hl & plane) << b;
        a.phi += (uint32_t)__popc(hh & plane) << b;
      }
    }
    if (valid) {
      // the term table holds idf (or 1 under count weighting)
      const float r = aux.w;
      const float w = (float)c * r;
      a.norm += to_fix(w * w);
      if (aux.code >= 0) atomicAdd(&num_q[aux.code], to_fix(w * r));
      if (p.bf16w) {  // the same with the weight rounded to bfloat16 (c * r16 is exact in FP32)
        const float r16 = __bfloat162float(__float2bfloat16_rn(r));
        const float w16 = (float)c * r16;
        a.norm16 += to_fix(w16 * w16);
        if (aux.code >= 0) atomicAdd(&num_q[p.k + aux.code], to_fix(w16 * r16));
      }
    }
    return;
  }
  // DENSE
  if (!valid) return;
  const float w = (float)c * aux.w;
  const float u = w * inv_norm;
  const int32_t code = aux.code;
  if (code >= 0) {
    const __half hi = __float2half_rn(u);
    const __half lo = __float2half_rn((u - __half2float(hi)) * kSplitLoScale);
    const int64_t at = doc * (int64_t)p.dense.kd + code;
    reinterpret_cast<__half*>(p.dense.head_hi)[at] = hi;
    reinterpret_cast<__half*>(p.dense.head_lo)[at] = lo;
  } else if (code <= -2) {  // a tail term (-2: no posting slot, bound-pruned mode)
    const int32_t r = atomicAdd(row_cnt_s, 1);
    p.dense.row_w[row_base + r] = u;
    if (code <= -3) {
      const int64_t pos = -3 - (int64_t)code;
      p.dense.post[pos] = make_int4((int32_t)doc, __float_as_int(u), r, 0);
    } else {
      p.dense.row_term[row_base + r] = (int32_t)key;
      // bucket |t|^2 in 32-bit 2^-31 fixed point (the accumulator area holds two per 8 bytes)
      atomicAdd(reinterpret_cast<uint32_t*>(num_q) + tail_bucket((int32_t)key), to_fix31_up(u));
    }
  }
}

// Bound-pruned exact cosine: the document's tail-bucket norms (sqrt of the 2^-31 fixed-point
// sums) as fp16 head columns kd_h .. kd_h + kTailBuckets - 1 (the split low part stays 0).
// Threads tid, tid + stride, ... of the document's group write.
__device__ __forceinline__ void write_bucket_norms(const IngestParams& p, int64_t d, const unsigned long long* num_q,
                                                   int tid, int stride) {
  const uint32_t* sums = reinterpret_cast<const uint32_t*>(num_q);
  const int32_t kd_h = p.dense.kd_h_dev ? *p.dense.kd_h_dev : p.dense.kd_h;
  __half* row = reinterpret_cast<__half*>(p.dense.head_hi) + d * (int64_t)p.dense.kd + kd_h;
  for (int q = tid; q < kTailBuckets; q += stride)
    row[q] = __float2half_rn(__fsqrt_ru(__uint2float_ru(sums[q]) * (1.0f / 2147483648.0f)));
}

// Writes the SIG outputs of one document; called by one full warp. With bf16w, the E4M3
// operand and its norm come from the unit signature of the bfloat16-weight vector (numerators
// num_q[k + p], squared norm norm16_q, reference norms rinv16); everything else from FP32 weights.
__device__ void finalize_sig(const IngestParams& p, int64_t d, int64_t len, unsigned long long norm_q,
                             unsigned long long norm16_q, const unsigned long long* num_q, uint32_t plo, uint32_t phi,
                             int lane) {
  const float nrm = sqrtf((float)norm_q * kInvFix);
  const float nrm16 = p.bf16w ? sqrtf((float)norm16_q * kInvFix) : 0.f;
  // raw signature s_p = t_p / |d|, t_p = num_p / |R_p|; the unit signature is s / |s|,
  // computed exactly as the packing of stored raw signatures computes it
  float ss = 0.f, ss16 = 0.f;
  for (int q = lane; q < p.k; q += 32) {
    const float t = (float)num_q[q] * kInvFix * p.rinv[q];
    const float sv = nrm > 0.f ? t / nrm : 0.f;
    ss += sv * sv;
    if (p.bf16w) {
      const float t16 = (float)num_q[p.k + q] * kInvFix * p.rinv16[q];
      const float sv16 = nrm16 > 0.f ? t16 / nrm16 : 0.f;
      ss16 += sv16 * sv16;
    }
  }
  ss = warp_sum(ss);
  const float sn = sqrtf(ss);
  float sn16 = 0.f;
  if (p.bf16w) sn16 = sqrtf(warp_sum(ss16));
  const int width = max(p.k, max(p.sig.kp, p.sig.kp8));
  float q2 = 0.f;  // squared norm of the E4M3-quantized unit signature
  for (int q = lane; q < width; q += 32) {
    const float t = q < p.k ? (float)num_q[q] * kInvFix * p.rinv[q] : 0.f;
    const float sv = nrm > 0.f ? t / nrm : 0.f;
    const float u = (q < p.k && sn > 0.f) ? sv / sn : 0.f;
    if (q < p.k) {
      if (p.sig.sig) p.sig.sig[d * p.k + q] = sv;
      if (p.sig.sig_unit) p.sig.sig_unit[d * p.k + q] = u;
    }
    if (q < p.sig.kp && p.sig.op_hi) {
      const __half hi = __float2half_rn(u);
      reinterpret_cast<__half*>(p.sig.op_hi)[d * p.sig.kp + q] = hi;
      if (p.sig.op_lo)
        reinterpret_cast<__half*>(p.sig.op_lo)[d * p.sig.kp + q] =
            __float2half_rn((u - __half2float(hi)) * kSplitLoScale);
    }
    if (q < p.sig.kp8 && p.sig.op_e4m3) {
      float u8 = u;
      if (p.bf16w) {
        const float t16 = q < p.k ? (float)num_q[p.k + q] * kInvFix * p.rinv16[q] : 0.f;
        const float sv16 = nrm16 > 0.f ? t16 / nrm16 : 0.f;
        u8 = (q < p.k && sn16 > 0.f) ? sv16 / sn16 : 0.f;
      }
      const __nv_fp8_storage_t e = __nv_cvt_float_to_fp8(u8 * kE4M3Scale, __NV_SATFINITE, __NV_E4M3);
      reinterpret_cast<uint8_t*>(p.sig.op_e4m3)[d * p.sig.kp8 + q] = (uint8_t)e;
      const float v = __half2float(__half(__nv_cvt_fp8_to_halfraw(e, __NV_E4M3))) * (1.0f / kE4M3Scale);
      q2 += v * v;
    }
  }
  if (p.sig.qnorm) {
    q2 = warp_sum(q2);
    if (lane == 0) p.sig.qnorm[d] = sqrtf(q2);
  }
  if (p.sig.simhash) {
    const unsigned lo = __ballot_sync(kFull, 2ll * (long long)plo > len);
    const unsigned hi = __ballot_sync(kFull, 2ll * (long long)phi > len);
    if (lane == 0) p.sig.simhash[d] = (uint64_t)lo | ((uint64_t)hi << 32);
  }
}

// ---------------------------------------------------------------- warp path
// Shared memory of one warp of the warp path: partition accumulators, the table, the list of
// occupied slots and two counters.
__host__ __device__ __forceinline__ size_t short_warp_bytes(int kq) {
  return (size_t)kq * 8 + (size_t)kShortSlots * 8 + (size_t)kShortMax * 2 + 16;
}

// One warp per document of <= kShortMax tokens, documents taken one at a time from a device
// counter as warps free up (their lengths vary 100-fold). The document's terms are either
// read from the stored bag into the table area (all loads in flight at once), or built by
// hashing the tokens (all token loads in flight at once, inserts in batches of 8) and found
// through the list of occupied slots. They are then walked 32 at a time, each chunk's table
// values gathered while the previous chunk is worked on.
template <int MODE>
__global__ void __launch_bounds__(kWarpsShort * 32, 3) k_ingest_short(IngestParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int kq = ingest_kq<MODE>(p);
  uint8_t* base = smem + short_warp_bytes(kq) * warp;
  unsigned long long* num_q = reinterpret_cast<unsigned long long*>(base);
  unsigned long long* tab = num_q + kq;
  uint16_t* list = reinterpret_cast<uint16_t*>(tab + kShortSlots);
  int32_t* misc = reinterpret_cast<int32_t*>(list + kShortMax);  // [0] list size, [1] row count
  const Transposer tr(lane);

  // A pass that reads stored bags needs no table, so it takes every document here, the
  // long-document list (longest first) before the short one; a hashing pass takes the short
  // documents only (the long ones go to the group path).
  const int32_t n_short = p.list_counts[0];
  const int32_t n_long = p.bag_read ? p.list_counts[1] : 0;
  int32_t it = 0;
  if (lane == 0) it = atomicAdd(p.short_cursor, 1);
  it = __shfl_sync(kFull, it, 0);
  while (it < n_short + n_long) {
    int32_t next = 0;
    if (lane == 0) next = atomicAdd(p.short_cursor, 1);
    const int64_t d = it < n_long ? p.long_list[it] : p.short_list[it - n_long];
    const int64_t o0 = p.offsets[d], len = p.offsets[d + 1] - o0;
    for (int q = lane; q < kq; q += 32) num_q[q] = 0ull;
    if (lane == 0) {
      misc[0] = 0;
      misc[1] = 0;
    }
    int nnz = 0;
    if (p.bag_read) {
      nnz = p.bag_n[d];  // the document's bag, built by an earlier pass, read as it is walked
    } else {
      const int l2 = log2_slots(len, 10);
      const int ts = 1 << l2;
      for (int s = lane; s < ts; s += 32) tab[s] = kEmpty64;
      int32_t tk[kShortRegs];
#pragma unroll
      for (int u = 0; u < kShortRegs; ++u) tk[u] = lane + 32 * u < len ? __ldcs(p.tokens + o0 + lane + 32 * u) : -1;
      __syncwarp();
      int32_t* df = (MODE == kDF || MODE == kDFN) ? p.df : nullptr;
#pragma unroll
      for (int h = 0; h < kShortRegs; h += 8) {
        if (32 * h >= len) break;  // warp-uniform
        int32_t tb[8];
        uint32_t pend = 0u;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          tb[u] = tk[h + u];
          if (lane + 32 * (h + u) < len) {
            if ((uint32_t)tb[u] >= (uint32_t)p.vocab)
              set_err(p.err, kErrBadToken);
            else
              pend |= 1u << u;
          }
        }
        if (!insert_batch<8>(tab, list, &misc[0], l2, tb, pend, df)) set_err(p.err, kErrTable);
      }
      __syncwarp();
      nnz = misc[0];
      if (p.bag_write) {
        for (int x = lane; x < nnz; x += 32) {
          const unsigned long long v = tab[list[x]];
          p.bag_terms[o0 + x] = (int32_t)(uint32_t)(v >> 32);
          p.bag_cnts[o0 + x] = (int32_t)(uint32_t)v;
        }
        if (lane == 0) p.bag_n[d] = nnz;
      }
    }
    Acc a{0ull, 0ull, 0u, 0u};
    float inv_norm = 0.f;
    if (MODE == kDENSE) inv_norm = inv_norm_of(p.dense.norm[d]);
    if (MODE != kDF || p.bag_read) {
      // term x: the bag's entry x, or the table slot the list's entry x names
      const bool bag = p.bag_read != 0;
      auto term = [&](int x, uint32_t& key, uint32_t& c) {
        if (x >= nnz) {
          key = kEmpty;
          c = 0u;
        } else if (bag) {
          key = (uint32_t)__ldcs(p.bag_terms + o0 + x);
          c = (uint32_t)__ldcs(p.bag_cnts + o0 + x);
        } else {
          const unsigned long long v = tab[list[x]];
          key = (uint32_t)(v >> 32);
          c = (uint32_t)v;
        }
      };
      uint32_t key, c;
      term(lane, key, c);
      TermAux ax{1.0f, 0, 0ull};
      if (MODE != kDF && key != kEmpty) ax = load_aux<MODE>(p, key);
      ax.h = load_hash<MODE>(p, key);
      for (int x0 = 0; x0 < nnz; x0 += 32) {
        uint32_t key1 = kEmpty, c1 = 0u;
        if (x0 + 32 < nnz) term(x0 + 32 + lane, key1, c1);  // the next chunk's table values, in flight
        TermAux ax1{1.0f, 0, 0ull};
        if (MODE != kDF && key1 != kEmpty) ax1 = load_aux<MODE>(p, key1);
        ax1.h = load_hash<MODE>(p, key1);
        chunk<MODE>(p, key, c, ax, tr, num_q, a, d, inv_norm, &misc[1], o0);
        key = key1;
        c = c1;
        ax = ax1;
      }
    }
    __syncwarp();
    if (MODE == kSIG) finalize_sig(p, d, len, warp_sum(a.norm), warp_sum(a.norm16), num_q, a.plo, a.phi, lane);
    if (MODE == kDFN) {
      const unsigned long long nq = warp_sum(a.norm);
      if (lane == 0) p.norm_out[d] = nq;
    }
    if (MODE == kDENSE) {
      if (!p.dense.postings) write_bucket_norms(p, d, num_q, lane, 32);
      if (lane == 0) p.dense.row_cnt[d] = misc[1];
    }
    __syncwarp();
    it = __shfl_sync(kFull, next, 0);
  }
  // This grid may start while the long-document grid (launched just before it) is still
  // running; it completes only after that grid, so the next launch on the stream sees both.
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Length classes of the long-document path: class c holds lengths in [2^(9+c), 2^(10+c)),
// c = 0..7.
constexpr int kLenClasses = 8;
// Counter words of one ingest call (int32).
constexpr int kCntShort = 0, kCntLong = 1, kCntMaxLen = 2, kCntLongCursor = 3, kCntShortCursor = 4,
              kCntHugeCursor = 5;
constexpr int kCntClass = 8, kCntClassFill = 16, kCntWords = 32;

// ---------------------------------------------------------------- long-document path
// Documents longer than kShortMax go to groups of kGroupWarps warps (kGroupsLong groups per
// CTA, each with its own table and named barrier), one document per group at a time, longest
// length class first. Documents of kHugeMin tokens or more are taken first, each by a whole
// CTA with one table in all of its shared memory (kHugeSlots slots). A document with more
// tokens than half its table is hashed in several passes, each keeping the terms of one hash
// partition (a second hash of the term id), so the table runs about half full. The list of
// occupied slots has room for every slot.
constexpr int kHugeMin = 2048;       // documents this long take a whole CTA
constexpr int kHugeSlots = 16384;    // the CTA-wide table
static_assert(kHugeMin == (2 << (9 + 1)), "length classes 2 and up are the documents of kHugeMin tokens or more");
__host__ __device__ __forceinline__ size_t long_group_bytes(int kq) {
  return (size_t)kq * 8 + 16 + 64 * 4 + 16 + (size_t)kLongSlots * 8 + (size_t)kLongSlots * 2;
}
__host__ __device__ __forceinline__ size_t long_huge_bytes(int kq) {
  return (size_t)kq * 8 + 16 + 64 * 4 + 16 + (size_t)kHugeSlots * 8 + (size_t)kHugeSlots * 2;
}

// Barrier `id` over `n` threads (id 0 with the whole CTA).
__device__ __forceinline__ void team_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// The team's warps walk the terms [0, n) of one document, warp tw taking chunks tw, tw + W, ...
// of 32 terms; term x is (key, count) = at(x) (kEmpty for x >= n). Each chunk's table values
// are gathered while the previous chunk is worked on. With bag_cursor, the terms are also
// appended to the document's bag (coalesced; no pass depends on the bag's order, every sum
// over it being an integer sum).
template <int MODE, typename At>
__device__ __forceinline__ void team_walk(const IngestParams& p, int n, int tw, int nwarps, int lane, const At& at,
                                          const Transposer& tr, unsigned long long* num_q, Acc& a, int64_t d,
                                          float inv_norm, int32_t* row_cnt_s, int64_t o0, int32_t* bag_cursor) {
  int x0 = tw * 32;
  uint32_t key = kEmpty, c = 0u;
  at(x0 + lane, key, c);
  TermAux ax{1.0f, 0, 0ull};
  if (MODE != kDF && key != kEmpty) ax = load_aux<MODE>(p, key);
  ax.h = load_hash<MODE>(p, key);
  while (x0 < n) {
    const int x1 = x0 + nwarps * 32;
    uint32_t key1 = kEmpty, c1 = 0u;
    if (x1 < n) at(x1 + lane, key1, c1);
    TermAux ax1{1.0f, 0, 0ull};
    if (MODE != kDF && key1 != kEmpty) ax1 = load_aux<MODE>(p, key1);
    ax1.h = load_hash<MODE>(p, key1);
    if (bag_cursor) {
      const unsigned occ = __ballot_sync(kFull, key != kEmpty);
      int32_t b = 0;
      if (lane == 0) b = atomicAdd(bag_cursor, __popc(occ));
      b = __shfl_sync(kFull, b, 0) + __popc(occ & ((1u << lane) - 1u));
      if (key != kEmpty) {
        p.bag_terms[o0 + b] = (int32_t)key;
        p.bag_cnts[o0 + b] = (int32_t)c;
      }
    }
    if (MODE != kDF || p.bag_read) chunk<MODE>(p, key, c, ax, tr, num_q, a, d, inv_norm, row_cnt_s, o0);
    x0 = x1;
    key = key1;
    c = c1;
    ax = ax1;
  }
}

// One long document by a team of `nthreads` threads (barrier `bar`) with a table of `slots`
// 64-bit entries in `base`: accumulators, then hashing passes (or the stored bag) and the
// walks, then the document's outputs. Called by every thread of the team.
template <int MODE>
__device__ void team_doc(const IngestParams& p, int64_t d, uint8_t* base, int kq, int slots, int nthreads, int bar,
                         int tt, const Transposer& tr) {
  const int tw = tt >> 5, lane = tt & 31, nwarps = nthreads >> 5;
  unsigned long long* num_q = reinterpret_cast<unsigned long long*>(base);
  unsigned long long* norm_s = num_q + kq;  // [0] |d|^2, [1] of the bfloat16 weights
  uint32_t* P = reinterpret_cast<uint32_t*>(norm_s + 2);  // [64] Simhash column sums
  int32_t* misc = reinterpret_cast<int32_t*>(P + 64);     // [1] row count, [2] bag size, [3] list size
  unsigned long long* tab = reinterpret_cast<unsigned long long*>(misc + 4);
  uint16_t* list = reinterpret_cast<uint16_t*>(tab + slots);
  const int64_t o0 = p.offsets[d], len = p.offsets[d + 1] - o0;
  for (int q = tt; q < kq; q += nthreads) num_q[q] = 0ull;
  if (tt < 64) P[tt] = 0u;
  if (tt == 0) {
    norm_s[0] = 0ull;
    norm_s[1] = 0ull;
    misc[1] = 0;
    misc[2] = 0;
  }
  Acc a{0ull, 0ull, 0u, 0u};
  float inv_norm = 0.f;
  if (MODE == kDENSE) inv_norm = inv_norm_of(p.dense.norm[d]);
  if (p.bag_read) {
    const int32_t nb = p.bag_n[d];
    team_sync(bar, nthreads);
    const int32_t* bt = p.bag_terms + o0;
    const int32_t* bcn = p.bag_cnts + o0;
    auto at = [&](int x, uint32_t& key, uint32_t& c) {
      if (x < nb) {
        key = (uint32_t)__ldcs(bt + x);
        c = (uint32_t)__ldcs(bcn + x);
      } else {
        key = kEmpty;
        c = 0u;
      }
    };
    team_walk<MODE>(p, nb, tw, nwarps, lane, at, tr, num_q, a, d, inv_norm, &misc[1], o0, nullptr);
  } else {
    int max_l2 = 6;
    while ((1 << (max_l2 + 1)) <= slots) ++max_l2;
    const int l2 = log2_slots(len, max_l2);
    const int ts = 1 << l2;
    const uint32_t passes = (uint32_t)((len + (slots / 2) - 1) / (slots / 2));
    int32_t* df = (MODE == kDF || MODE == kDFN) ? p.df : nullptr;
    const bool walk = MODE != kDF || p.bag_write;
    for (uint32_t pass = 0; pass < passes; ++pass) {
      team_sync(bar, nthreads);
      for (int sl = tt; sl < ts; sl += nthreads) tab[sl] = kEmpty64;
      if (tt == 0) misc[3] = 0;
      team_sync(bar, nthreads);
      for (int64_t x0 = tt; x0 < len; x0 += kLongUnroll * nthreads) {
        int32_t tk[kLongUnroll];  // kLongUnroll token loads in flight per thread
#pragma unroll
        for (int u = 0; u < kLongUnroll; ++u) {
          const int64_t x = x0 + u * nthreads;
          tk[u] = x < len ? __ldcs(p.tokens + o0 + x) : -1;
        }
        uint32_t pend = 0u;
#pragma unroll
        for (int u = 0; u < kLongUnroll; ++u) {
          if (x0 + u * nthreads >= len) break;
          const int32_t t = tk[u];
          if ((uint32_t)t >= (uint32_t)p.vocab) {
            if (pass == 0) set_err(p.err, kErrBadToken);
            continue;
          }
          if (passes > 1 && pass_of((uint32_t)t, passes) != pass) continue;
          pend |= 1u << u;
        }
        if (!insert_batch<kLongUnroll>(tab, list, &misc[3], l2, tk, pend, df)) set_err(p.err, kErrTable);
      }
      team_sync(bar, nthreads);
      if (walk) {
        const int n = misc[3];
        auto at = [&](int x, uint32_t& key, uint32_t& c) {
          const unsigned long long v = x < n ? tab[list[x]] : kEmpty64;
          key = (uint32_t)(v >> 32);
          c = (uint32_t)v;
        };
        team_walk<MODE>(p, n, tw, nwarps, lane, at, tr, num_q, a, d, inv_norm, &misc[1], o0,
                        p.bag_write ? &misc[2] : nullptr);
      }
    }
  }
  if (MODE == kDFN || MODE == kSIG) {
    const unsigned long long nq = warp_sum(a.norm);
    if (lane == 0 && nq) atomicAdd(norm_s, nq);
  }
  if (MODE == kSIG && p.bf16w) {
    const unsigned long long nq = warp_sum(a.norm16);
    if (lane == 0 && nq) atomicAdd(norm_s + 1, nq);
  }
  if (MODE == kSIG) {
    atomicAdd(&P[lane], a.plo);
    atomicAdd(&P[lane + 32], a.phi);
  }
  team_sync(bar, nthreads);
  if (MODE == kSIG && tw == 0) finalize_sig(p, d, len, norm_s[0], norm_s[1], num_q, P[lane], P[lane + 32], lane);
  if (MODE == kDENSE) {
    if (tt == 0) p.dense.row_cnt[d] = misc[1];
    if (!p.dense.postings) write_bucket_norms(p, d, num_q, tt, nthreads);
  }
  if (MODE == kDFN && tt == 0) p.norm_out[d] = norm_s[0];
  if (p.bag_write && tt == 0) p.bag_n[d] = misc[2];
  team_sync(bar, nthreads);
}

template <int MODE>
__global__ void __launch_bounds__(kLongThreads, 1) k_ingest_long(IngestParams p) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ int32_t s_next, s_huge;
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
  // phase 1: the huge documents, one per CTA at a time
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(p.huge_cursor, 1);
    __syncthreads();
    const int32_t it = s_next;
    __syncthreads();
    if (it >= n_huge) break;
    team_doc<MODE>(p, p.long_list[it], smem, kq, kHugeSlots, kLongThreads, 0, threadIdx.x, tr);
  }
  // phase 2: the other long documents, one per group at a time
  uint8_t* base = smem + long_group_bytes(kq) * g;
  int32_t* slot = reinterpret_cast<int32_t*>(base + (size_t)kq * 8 + 16 + 64 * 4);  // misc[0] of the group
  while (true) {
    if (gt == 0) *slot = n_huge + atomicAdd(p.long_cursor, 1);
    team_sync(1 + g, kGroupThreads);
    const int32_t it = *slot;
    if (it >= n_long) break;
    team_doc<MODE>(p, p.long_list[it], base, kq, kLongSlots, kGroupThreads, 1 + g, gt, tr);
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
template <int MODE>
int short_grid(const mrc_ctx* ctx, size_t smem) {
  return ctx->num_sms * resident_ctas(k_ingest_short<MODE>, kWarpsShort * 32, smem);
}
template <int MODE>
int long_grid(const mrc_ctx* ctx, size_t smem) {
  return ctx->num_sms * resident_ctas(k_ingest_long<MODE>, kLongThreads, smem);
}

size_t short_smem(int kq) { return (size_t)kWarpsShort * short_warp_bytes(kq); }
size_t long_smem(int kq) { return std::max((size_t)kGroupsLong * long_group_bytes(kq), long_huge_bytes(kq)); }

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
  const int kq = ingest_kq<MODE>(p);
  const size_t s_smem = short_smem(kq), l_smem = long_smem(kq);
  const double tokens = (double)d.n_tokens;
  cudaEvent_t ev = nullptr;
  // The CTA path (longest documents first) is launched first; the warp path follows as a
  // programmatic dependent launch, so its CTAs fill SMs as the CTA path's grid drains instead
  // of waiting for the whole grid. Not while the stream is being captured into a graph.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(ctx->stream, &cap);
  const bool overlap = cap == cudaStreamCaptureStatusNone && !ctx->timing;
  if (!p.bag_read) {  // a pass over stored bags takes every document in the warp path
    int grid = long_grid<MODE>(ctx, l_smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    if (d.n_docs < grid) grid = (int)d.n_docs;
    std::string nm = std::string(name) + ".long";
    timing_begin(ctx, nm.c_str(), 0.0, 0.0, &ev);
    k_ingest_long<MODE><<<grid, kLongThreads, l_smem, ctx->stream>>>(p);
    timing_end(ctx, ev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  {
    int grid = short_grid<MODE>(ctx, s_smem);
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
    e = cudaLaunchKernelEx(&cfg, k_ingest_short<MODE>, p);
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
  const size_t s_smem = short_smem(k), l_smem = long_smem(k);
  if (h[0] > 0) {
    int grid = short_grid<kSIG>(ctx, s_smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    const int need = (h[0] + kWarpsShort - 1) / kWarpsShort;
    if (need < grid) grid = need;
    k_ingest_short<kSIG><<<grid, kWarpsShort * 32, s_smem, ctx->stream>>>(p);
  }
  if (h[1] > 0) {
    int grid = long_grid<kSIG>(ctx, l_smem);
    if (grid <= 0) return cudaErrorInvalidConfiguration;
    if (h[1] < grid) grid = h[1];
    k_ingest_long<kSIG><<<grid, kLongThreads, l_smem, ctx->stream>>>(p);
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
