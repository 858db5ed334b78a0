// ingest_dev.cuh -- device code of the per-document passes (rows a1-a4), shared by the ingest
// kernels (ingest.cu) and the persistent batch kernel (compare_tc.cu). See ingest.cu for the
// design of the passes.
#pragma once

#include <cuda_bf16.h>
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
constexpr int kGroupsLong = 5;      // groups per CTA with 64-bit tables (one CTA per SM: five fill shared memory)
constexpr int kLongSlots = 4096;    // per-group table: documents with > 2048 tokens take several passes
constexpr int kLongUnroll = 4;      // token loads per thread in flight (long-document path)
constexpr float kFix = 4194304.0f;  // 2^22
constexpr float kInvFix = 1.0f / 4194304.0f;

enum Mode { kDF = 0, kSIG = 1, kDENSE = 2, kDFN = 3 };

__device__ __forceinline__ uint32_t slot_of(uint32_t t, int log2ts) { return (t * 0x9E3779B1u) >> (32 - log2ts); }
// The hashing pass [0, passes) of term t (a document hashed in several passes keeps one hash
// partition per pass): the high word of a second hash times passes, so no division.
__device__ __forceinline__ uint32_t pass_of(uint32_t t, uint32_t passes) { return __umulhi(t * 0x85EBCA77u, passes); }

// SplitMix64 (Steele, Lea, Flood 2014), one step from state (t XOR seed).
__device__ __forceinline__ uint64_t feature_hash(uint32_t t, uint64_t seed) {
  uint64_t z = ((uint64_t)t ^ seed) + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
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

// Conversions between FP32 and 64-bit integers with integer operations only: the hardware
// conversions of 64-bit integers run on the FP64 units, which are few on this part. Both round to
// nearest, ties to even, exactly as the 64-bit conversion instructions do.
// x >= 0 finite -> the nearest integer.
__device__ __forceinline__ unsigned long long f32_to_u64_rn(float x) {
  if (x < 4294967296.0f) return (unsigned long long)__float2uint_rn(x);
  const uint32_t b = __float_as_uint(x);  // >= 2^32: an integer, mantissa << (exponent - 23)
  const int e = (int)((b >> 23) & 0xFFu) - 127;
  return (unsigned long long)((b & 0x7FFFFFu) | 0x800000u) << (e - 23);
}
// v -> the nearest float.
__device__ __forceinline__ float u64_to_f32_rn(unsigned long long v) {
  if ((v >> 32) == 0ull) return __uint2float_rn((uint32_t)v);
  const int sh = 40 - __clzll((long long)v);  // bits below the 24 kept (v >= 2^32: sh >= 8)
  unsigned long long m = v >> sh;
  const unsigned long long rem = v & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  if (rem > half || (rem == half && (m & 1ull))) ++m;
  int ex = sh + 23;
  if (m == (1ull << 24)) {
    m >>= 1;
    ++ex;
  }
  return __uint_as_float(((uint32_t)(ex + 127) << 23) | ((uint32_t)m & 0x7FFFFFu));
}

__device__ __forceinline__ unsigned long long to_fix(float x) { return f32_to_u64_rn(x * kFix); }

// 1 / |w| from the fixed-point squared norm (0 for an empty document).
// u^2 in 2^-31 fixed point, rounded up: FP32 with directed rounding (the power-of-two scaling
// is exact), so the bucket norms bound from above. A document's tail has sum u^2 <= 1, so a
// bucket's sum stays below 2^31 + 65,536 < 2^32.
__device__ __forceinline__ uint32_t to_fix31_up(float u) { return __float2uint_ru(__fmul_ru(u, u) * 2147483648.0f); }
__device__ __forceinline__ float inv_norm_of(unsigned long long norm_q) {
  const float n2 = u64_to_f32_rn(norm_q) * kInvFix;
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
// The tables of the warp path and of the four-warp groups use 32-bit slots when the vocabulary has
// fewer than kNarrowVocab term ids: the term id above kSlotCountBits bits of count (those
// documents have fewer than kHugeMin tokens, so no count reaches 2^11), and all ones for a free
// slot (no term id reaches it). Half the shared memory per table, so more documents are in
// flight per SM. The CTA-wide table of the longest documents keeps 64-bit slots.
constexpr int kSlotCountBits = 11;
constexpr uint32_t kEmpty32 = 0xFFFFFFFFu;
constexpr int32_t kNarrowVocab = (1 << (32 - kSlotCountBits)) - 1;
template <typename S>
struct Slot;
template <>
struct Slot<unsigned long long> {
  static constexpr unsigned long long kFree = kEmpty64, kOne = 1ull;
  __device__ static unsigned long long make(uint32_t t) { return ((unsigned long long)t << 32) | 1ull; }
  __device__ static uint32_t term(unsigned long long v) { return (uint32_t)(v >> 32); }
  __device__ static uint32_t count(unsigned long long v) { return (uint32_t)v; }
};
template <>
struct Slot<uint32_t> {
  static constexpr uint32_t kFree = kEmpty32, kOne = 1u;
  __device__ static uint32_t make(uint32_t t) { return (t << kSlotCountBits) | 1u; }
  __device__ static uint32_t term(uint32_t v) { return v >> kSlotCountBits; }
  __device__ static uint32_t count(uint32_t v) { return v & ((1u << kSlotCountBits) - 1u); }
};
template <int B, typename S>
__device__ __forceinline__ bool insert_batch(S* tab, uint16_t* list, int32_t* list_n, int log2ts,
                                             const int32_t (&tk)[B], uint32_t pend, int32_t* df) {
  using T = Slot<S>;
  const uint32_t mask = (1u << log2ts) - 1u;
  uint32_t slot[B];
#pragma unroll
  for (int u = 0; u < B; ++u) slot[u] = slot_of((uint32_t)tk[u], log2ts);
  uint32_t fresh = 0u;
  for (uint32_t round = 0; pend != 0u && round <= mask; ++round) {
    S prev[B];
#pragma unroll
    for (int u = 0; u < B; ++u)
      if ((pend >> u) & 1u) prev[u] = atomicCAS(&tab[slot[u]], T::kFree, T::make((uint32_t)tk[u]));
#pragma unroll
    for (int u = 0; u < B; ++u)
      if ((pend >> u) & 1u) {
        if (prev[u] == T::kFree) {
          fresh |= 1u << u;
          pend &= ~(1u << u);
        } else if (T::term(prev[u]) == (uint32_t)tk[u]) {
          atomicAdd(&tab[slot[u]], T::kOne);
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
  // Persistent batch kernel: the number of real documents, read on the device; documents from
  // *n_live on are empty (their offsets are not read), and so is a document whose tokens do
  // not lie in [0, n_tokens). NULL elsewhere.
  const int64_t* n_live;
  int64_t n_tokens;
  int32_t narrow;  // warp-path tables with 32-bit slots (vocab < kNarrowVocab)
};

// Token range of document d. A document past *n_live, or with a length outside
// [0, MRC_MAX_DOC_TOKENS] (reported by the pass that lists the documents), is empty.
__device__ __forceinline__ void doc_span(const IngestParams& p, int64_t d, int64_t& o0, int64_t& len) {
  if (p.n_live && d >= *p.n_live) {
    o0 = 0;
    len = 0;
    return;
  }
  o0 = p.offsets[d];
  len = p.offsets[d + 1] - o0;
  if (len < 0 || len > MRC_MAX_DOC_TOKENS) len = 0;
  if (p.n_live && (o0 < 0 || o0 + len > p.n_tokens)) {
    o0 = 0;
    len = 0;
  }
}

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
  const float nrm = sqrtf(u64_to_f32_rn(norm_q) * kInvFix);
  const float nrm16 = p.bf16w ? sqrtf(u64_to_f32_rn(norm16_q) * kInvFix) : 0.f;
  // raw signature s_p = t_p / |d|, t_p = num_p / |R_p|; the unit signature is s / |s|,
  // computed exactly as the packing of stored raw signatures computes it. The raw entries of
  // the first kFinCache rounds (k <= 64) stay in registers for the second loop.
  constexpr int kFinCache = 2;
  auto raw = [&](int q) {
    const float t = u64_to_f32_rn(num_q[q]) * kInvFix * p.rinv[q];
    return nrm > 0.f ? t / nrm : 0.f;
  };
  auto raw16 = [&](int q) {
    const float t16 = u64_to_f32_rn(num_q[p.k + q]) * kInvFix * p.rinv16[q];
    return nrm16 > 0.f ? t16 / nrm16 : 0.f;
  };
  float svc[kFinCache], sv16c[kFinCache];
  float ss = 0.f, ss16 = 0.f;
#pragma unroll
  for (int r = 0; r < kFinCache; ++r) {
    const int q = lane + 32 * r;
    svc[r] = sv16c[r] = 0.f;
    if (q < p.k) {
      svc[r] = raw(q);
      ss += svc[r] * svc[r];
      if (p.bf16w) {
        sv16c[r] = raw16(q);
        ss16 += sv16c[r] * sv16c[r];
      }
    }
  }
  for (int q = lane + 32 * kFinCache; q < p.k; q += 32) {
    const float sv = raw(q);
    ss += sv * sv;
    if (p.bf16w) {
      const float sv16 = raw16(q);
      ss16 += sv16 * sv16;
    }
  }
  ss = warp_sum(ss);
  const float sn = sqrtf(ss);
  float sn16 = 0.f;
  if (p.bf16w) sn16 = sqrtf(warp_sum(ss16));
  const int width = max(p.k, max(p.sig.kp, p.sig.kp8));
  float q2 = 0.f;  // squared norm of the E4M3-quantized unit signature
  for (int q = lane, r = 0; q < width; q += 32, ++r) {
    float sv = 0.f;
    if (q < p.k) {
      if (r < kFinCache) {
#pragma unroll
        for (int x = 0; x < kFinCache; ++x)
          if (x == r) sv = svc[x];
      } else {
        sv = raw(q);
      }
    }
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
        float sv16 = 0.f;
        if (q < p.k) {
          if (r < kFinCache) {
#pragma unroll
            for (int x = 0; x < kFinCache; ++x)
              if (x == r) sv16 = sv16c[x];
          } else {
            sv16 = raw16(q);
          }
        }
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
// A pass over stored bags uses no table: its warps need only the accumulators and counters.
__host__ __device__ __forceinline__ size_t bag_warp_bytes(int kq) { return (size_t)kq * 8 + 16; }
__host__ __device__ __forceinline__ size_t short_warp_bytes(int kq, bool narrow) {
  return (size_t)kq * 8 + (size_t)kShortSlots * (narrow ? 4 : 8) + (size_t)kShortMax * 2 + 16;
}
__host__ __device__ __forceinline__ bool narrow_slots(int32_t vocab) { return vocab > 0 && vocab <= kNarrowVocab; }

// The hashing part of warp_doc: the document's tokens into the warp's table of S slots, the
// occupied slots listed; with bag_write the bag is stored. Returns the number of distinct terms.
template <int MODE, typename S>
__device__ __forceinline__ int hash_doc(const IngestParams& p, int64_t d, S* tab, uint16_t* list, int32_t* misc,
                                        int64_t o0, int64_t len, int lane) {
  using T = Slot<S>;
  const int l2 = log2_slots(len, 10);
  const int ts = 1 << l2;
  for (int s = lane; s < ts; s += 32) tab[s] = T::kFree;
  int32_t tk[kShortRegs];
#pragma unroll
  for (int u = 0; u < kShortRegs; ++u) tk[u] = lane + 32 * u < len ? __ldcs(p.tokens + o0 + lane + 32 * u) : -1;
  __syncwarp();
  int32_t* df = (MODE == kDF || MODE == kDFN) ? p.df : nullptr;
  // one copy of the batch insert for both batches (the tokens are selected, so they stay in
  // registers): the loop body is large, and two copies of it cost instruction-cache misses
  static_assert(kShortRegs == 16, "two batches of 8 tokens per lane");
#pragma unroll 1
  for (int h = 0; h < kShortRegs; h += 8) {
    if (32 * h >= len) break;  // warp-uniform
    int32_t tb[8];
    uint32_t pend = 0u;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      tb[u] = h == 0 ? tk[u] : tk[8 + u];
      if (lane + 32 * (h + u) < len) {
        if ((uint32_t)tb[u] >= (uint32_t)p.vocab)
          set_err(p.err, kErrBadToken);
        else
          pend |= 1u << u;
      }
    }
    if (!insert_batch<8, S>(tab, list, &misc[0], l2, tb, pend, df)) set_err(p.err, kErrTable);
  }
  __syncwarp();
  const int nnz = misc[0];
  if (p.bag_write) {
    for (int x = lane; x < nnz; x += 32) {
      const S v = tab[list[x]];
      p.bag_terms[o0 + x] = (int32_t)T::term(v);
      p.bag_cnts[o0 + x] = (int32_t)T::count(v);
    }
    if (lane == 0) p.bag_n[d] = nnz;
  }
  return nnz;
}

// One document of <= kShortMax tokens (or any stored bag) by one warp, in the warp's shared
// memory `base` (short_warp_bytes(kq, p.narrow), or bag_warp_bytes(kq) for a pass over stored
// bags). The document's terms are either read from the stored bag as they are walked, or built
// by hashing the tokens (all token loads in flight at once, inserts in batches of 8) and found
// through the list of occupied slots. They are then walked 32 at a time, each chunk's table
// values gathered while the previous chunk is worked on.
// V fixes at compile time which of the three ways the kernel takes (stored bags, 32-bit table,
// 64-bit table), so that each kernel holds the code of one and its loops stay in the
// instruction cache; kVarAny decides from p at run time.
constexpr int kVarAny = 0, kVarBag = 1, kVarNarrow = 2, kVarWide = 3;
template <int MODE, int V = kVarAny>
__device__ void warp_doc(const IngestParams& p, int64_t d, uint8_t* base, int kq, int lane, const Transposer& tr) {
  unsigned long long* num_q = reinterpret_cast<unsigned long long*>(base);
  uint8_t* tab = reinterpret_cast<uint8_t*>(num_q + kq);
  const bool bag_read = V == kVarAny ? p.bag_read != 0 : V == kVarBag;
  const bool narrow = V == kVarAny ? p.narrow != 0 : V == kVarNarrow;
  uint16_t* list = reinterpret_cast<uint16_t*>(tab + (size_t)kShortSlots * (narrow ? 4 : 8));
  // [0] list size, [1] row count (right after the accumulators in a pass over stored bags)
  int32_t* misc = bag_read ? reinterpret_cast<int32_t*>(tab) : reinterpret_cast<int32_t*>(list + kShortMax);
  int64_t o0, len;
  doc_span(p, d, o0, len);
  for (int q = lane; q < kq; q += 32) num_q[q] = 0ull;
  if (lane == 0) {
    misc[0] = 0;
    misc[1] = 0;
  }
  int nnz = 0;
  if (bag_read)
    nnz = p.bag_n[d];  // the document's bag, built by an earlier pass, read as it is walked
  else if (narrow)
    nnz = hash_doc<MODE, uint32_t>(p, d, reinterpret_cast<uint32_t*>(tab), list, misc, o0, len, lane);
  else
    nnz = hash_doc<MODE, unsigned long long>(p, d, reinterpret_cast<unsigned long long*>(tab), list, misc, o0, len,
                                             lane);
  Acc a{0ull, 0ull, 0u, 0u};
  float inv_norm = 0.f;
  if (MODE == kDENSE) inv_norm = inv_norm_of(p.dense.norm[d]);
  if (MODE != kDF || bag_read) {
    // term x: the bag's entry x, or the table slot the list's entry x names
    const bool bag = bag_read;
    auto term = [&](int x, uint32_t& key, uint32_t& c) {
      if (x >= nnz) {
        key = kEmpty;
        c = 0u;
      } else if (bag) {
        key = (uint32_t)__ldcs(p.bag_terms + o0 + x);
        c = (uint32_t)__ldcs(p.bag_cnts + o0 + x);
      } else if (narrow) {
        const uint32_t v = reinterpret_cast<const uint32_t*>(tab)[list[x]];
        key = Slot<uint32_t>::term(v);
        c = Slot<uint32_t>::count(v);
      } else {
        const unsigned long long v = reinterpret_cast<const unsigned long long*>(tab)[list[x]];
        key = Slot<unsigned long long>::term(v);
        c = Slot<unsigned long long>::count(v);
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
constexpr int kHugeMin = 2048;       // documents this long take a whole CTA (64-bit tables)
constexpr int kHugeSlots = 16384;    // the CTA-wide table
// With 32-bit group tables the documents of kHugeMin tokens or more go to the groups too, each
// into a table of kHugeGroupSlots 64-bit slots (their counts may need more than 11 bits) in the
// same bytes as the group's 32-bit table, hashed in passes of kHugeGroupSlots / 2 terms.
constexpr int kHugeGroupSlots = 2048;
static_assert(kHugeMin == (2 << (9 + 1)), "length classes 2 and up are the documents of kHugeMin tokens or more");
static_assert(kHugeMin <= (1 << kSlotCountBits), "a group-path document's counts fit a 32-bit slot");
static_assert(kHugeGroupSlots * (8 + 2) <= kLongSlots * (4 + 2) && kHugeGroupSlots <= kLongSlots,
              "a huge document's 64-bit table and slot list fit a 32-bit group's");
__host__ __device__ __forceinline__ size_t long_group_bytes(int kq, bool narrow) {
  return (size_t)kq * 8 + 16 + 64 * 4 + 16 + (size_t)kLongSlots * (narrow ? 4 : 8) + (size_t)kLongSlots * 2;
}
// Groups per CTA of the long-document path (one CTA per SM): five with 64-bit tables (shared
// memory), with 32-bit ones eight (1,024 threads) in the passes that need at most 64 registers a
// thread and seven (72 registers) in the signature pass.
__host__ __device__ constexpr int long_groups(int mode, bool narrow) {
  return !narrow ? kGroupsLong : (mode == kSIG ? 7 : 8);
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
// entries of type S (64-bit, or 32-bit for documents of fewer than kHugeMin tokens of a
// narrow vocabulary) in `base`: accumulators, then hashing passes (or the stored bag) and the
// walks, then the document's outputs. Called by every thread of the team.
template <int MODE, typename S = unsigned long long>
__device__ void team_doc(const IngestParams& p, int64_t d, uint8_t* base, int kq, int slots, int nthreads, int bar,
                         int tt, const Transposer& tr) {
  const int tw = tt >> 5, lane = tt & 31, nwarps = nthreads >> 5;
  unsigned long long* num_q = reinterpret_cast<unsigned long long*>(base);
  unsigned long long* norm_s = num_q + kq;  // [0] |d|^2, [1] of the bfloat16 weights
  uint32_t* P = reinterpret_cast<uint32_t*>(norm_s + 2);  // [64] Simhash column sums
  int32_t* misc = reinterpret_cast<int32_t*>(P + 64);     // [1] row count, [2] bag size, [3] list size
  S* tab = reinterpret_cast<S*>(misc + 4);
  uint16_t* list = reinterpret_cast<uint16_t*>(tab + slots);
  int64_t o0, len;
  doc_span(p, d, o0, len);
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
      for (int sl = tt; sl < ts; sl += nthreads) tab[sl] = Slot<S>::kFree;
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
          if (x < n) {
            const S v = tab[list[x]];
            key = Slot<S>::term(v);
            c = Slot<S>::count(v);
          } else {
            key = kEmpty;
            c = 0u;
          }
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

}  // namespace
}  // namespace mrc
