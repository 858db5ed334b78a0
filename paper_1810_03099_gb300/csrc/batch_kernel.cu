// batch_kernel.cu -- a query batch as one persistent, cooperative kernel (row a9).
//
// New documents are signatured and compared with the resident signature index (Section I:
// each new page against the stored signatures; Section IV: the signature pass and the compare),
// and their Simhash fingerprints are looked up in a block-table index (Section III). One launch
// runs every step; its CTAs (one per SM, all resident: cooperative launch) pass through six
// phases separated by grid-wide barriers:
//   0  list the batch's long documents, check the offsets, clear the per-query counters;
//   1  signature pass (Eq. 3 per reference partition, the Simhash columns, the unit signature and
//      the compare operand): documents longer than kShortMax by a whole CTA (one table in all of
//      its shared memory), the others by one warp each, both taken from atomic cursors;
//   2  tensor-core compare of the batch rows with every index row (the resident compare: TMA
//      producer warp, tcgen05 MMA warp, eight thresholding epilogue warps, accumulators in
//      TMEM), candidates above the lowered threshold into a list;
//   3  FP32 rescoring of the candidates (kept iff the unit-signature dot product, in the
//      library's one fixed order, reaches tau) and the Hamming probe (one CTA per
//      (query, table) bucket, its warps splitting the bucket), with per-query counts;
//   4  exclusive scans of the per-query counts (one CTA);
//   5  pairs scattered into query order.
// The signature pass and the compare reuse the device code of the separate kernels, so the
// results are those of the eager calls. Every wait (the grid barriers and the compare's
// pipeline) is bounded by the context's wait limit.
#include "ingest_dev.cuh"
#include "tc_dev.cuh"

namespace mrc {
namespace {

constexpr int kCtlLongN = 0, kCtlLongCur = 1, kCtlShortCur = 2, kCtlProbeCur = 3, kCtlBarrier = 4, kCtlAbort = 5;
static_assert(kCtlAbort < kBatchCtlWords, "control words");

struct BatchParams {
  IngestParams ing;
  GemmParams g;
  int64_t max_docs;
  const int64_t* n_live;
  int32_t* ctl;
  int32_t* long_list;
  int32_t team_slots;  // table of a CTA-wide document (power of two)
  // rescoring
  const mrc_pair* cand;
  const unsigned long long* n_cand;
  int64_t cand_cap;
  const float* q_unit;
  const float* x_unit;
  int32_t k;
  float tau;
  mrc_pair* pairs;
  unsigned long long* n_pairs;
  int64_t capacity;
  // grouping
  int32_t qstride;
  int32_t* qcnt;
  int32_t* qfill;
  int64_t* qoff;
  mrc_pair* grouped;
  // Hamming leg (hmax < 0: none)
  int32_t hmax;
  SimhashLayout L;
  int64_t hn;
  const uint64_t* hfp;
  const int32_t* hid;
  const int32_t* hoff;
  const uint64_t* qfp;
  mrc_pair* hpairs;
  unsigned long long* n_hpairs;
  int64_t hcapacity;
  int32_t* hqcnt;
  int32_t* hqfill;
  int64_t* hqoff;
  mrc_pair* hgrouped;
  int32_t* err;
  uint64_t timeout_ns;
  unsigned long long* stamps;  // [kBatchStamps] CTA 0's global timer at the start and after each phase
};

__device__ __forceinline__ uint32_t ld_acquire(const unsigned* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier of the cooperative launch: the k-th barrier of a launch waits until the
// counter reaches k * gridDim.x. Bounded: past the wait limit it records kErrTimeout and sets
// the abort word; a CTA that sees the abort word gives up too. Returns false then.
__device__ bool grid_sync(const BatchParams& bp, unsigned& target, int32_t* ok_s) {
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* ctr = reinterpret_cast<unsigned*>(bp.ctl + kCtlBarrier);
    volatile int32_t* abort_g = bp.ctl + kCtlAbort;
    int ok = 1;
    __threadfence();
    atomicAdd(ctr, 1u);
    const uint64_t t0 = gtime();
    while (ld_acquire(ctr) < target) {
      if (*abort_g) {
        ok = 0;
        break;
      }
      if (gtime() - t0 > bp.timeout_ns) {
        *abort_g = 1;
        set_err(bp.err, kErrTimeout);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    *ok_s = ok;
  }
  __syncthreads();
  return *ok_s != 0;
}

// The next item of an atomic cursor, for the whole CTA.
__device__ __forceinline__ int32_t cta_grab(int32_t* cursor, int32_t* slot) {
  if (threadIdx.x == 0) *slot = atomicAdd(cursor, 1);
  __syncthreads();
  const int32_t x = *slot;
  __syncthreads();
  return x;
}

// A batch of at most one document per CTA hashes every document with a whole CTA (a shorter
// latency than one warp per document); a larger one uses warps for documents of up to kShortMax
// tokens.
__device__ __forceinline__ bool team_all(int64_t n) { return n <= (int64_t)gridDim.x; }

// Phase 0: documents for the CTA-wide path go to the long list; offset errors are recorded
// (the documents concerned are then empty); per-query counters are cleared.
__device__ void phase_list(const BatchParams& bp, int64_t n) {
  const IngestParams& ing = bp.ing;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; d < bp.max_docs; d += stride) {
    bp.qcnt[d * bp.qstride] = 0;
    bp.qfill[d * bp.qstride] = 0;
    if (bp.hmax >= 0) {
      bp.hqcnt[d * bp.qstride] = 0;
      bp.hqfill[d * bp.qstride] = 0;
    }
    if (d >= n) continue;
    const int64_t o0 = ing.offsets[d], raw = ing.offsets[d + 1] - o0;
    if ((d == 0 && o0 != 0) || raw < 0 || o0 < 0 || o0 + raw > ing.n_tokens) set_err(bp.err, kErrBadOffsets);
    else if (raw > MRC_MAX_DOC_TOKENS) set_err(bp.err, kErrTooLong);
    int64_t s, len;
    doc_span(ing, d, s, len);
    if (len > kShortMax || (team_all(n) && len > 0)) bp.long_list[atomicAdd(&bp.ctl[kCtlLongN], 1)] = (int32_t)d;
  }
}

// Phase 1: the signature pass of the batch's documents (documents past n are written as empty
// ones: zero signature and operand, Simhash 0).
__device__ void phase_signature(const BatchParams& bp, int64_t n, uint8_t* smem, int32_t* slot) {
  const IngestParams& ing = bp.ing;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const Transposer tr(lane);
  const int kq = ingest_kq<kSIG>(ing);
  const int32_t n_long = __ldcg(bp.ctl + kCtlLongN);
  while (true) {
    const int32_t x = cta_grab(bp.ctl + kCtlLongCur, slot);
    if (x >= n_long) break;
    team_doc<kSIG>(ing, __ldcg(bp.long_list + x), smem, kq, bp.team_slots, blockDim.x, 1, threadIdx.x, tr);
  }
  uint8_t* wbase = smem + (size_t)warp * short_warp_bytes(kq, ing.narrow != 0);
  while (true) {
    int32_t d = 0;
    if (lane == 0) d = atomicAdd(bp.ctl + kCtlShortCur, 1);
    d = __shfl_sync(kFull, d, 0);
    if (d >= bp.max_docs) break;
    int64_t o0, len;
    doc_span(ing, d, o0, len);
    if (len > kShortMax || (team_all(n) && len > 0)) continue;  // a CTA took it
    warp_doc<kSIG>(ing, d, wbase, kq, lane, tr);
  }
  // the compare operands are read by TMA (the async proxy) after the next barrier
  asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Phase 3a: FP32 rescoring, one thread per candidate; kept pairs are appended (one atomic per
// warp) and counted per query (one atomic per query present in the warp).
__device__ void phase_rescore(const BatchParams& bp) {
  const int lane = threadIdx.x & 31;
  const int64_t nc0 = (int64_t)__ldcg(bp.n_cand);
  const int64_t nc = nc0 < bp.cand_cap ? nc0 : bp.cand_cap;
  if (nc0 > bp.cand_cap && blockIdx.x == 0 && threadIdx.x == 0) set_err(bp.err, kErrOverflow);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < nc; w0 += stride) {
    const int64_t c = w0 + lane;
    mrc_pair pr{0, 0, 0.f};
    bool keep = false;
    if (c < nc) {
      const int32_t* cw = reinterpret_cast<const int32_t*>(bp.cand + c);
      pr.i = __ldcg(cw);
      pr.j = __ldcg(cw + 1);
      pr.score = unit_dot<true>(bp.q_unit + (int64_t)pr.i * bp.k, bp.x_unit + (int64_t)pr.j * bp.k, bp.k);
      keep = pr.score >= bp.tau;
    }
    const unsigned m = __ballot_sync(kFull, keep);
    if (!m) continue;
    unsigned long long b = 0;
    if (lane == 0) b = atomicAdd(bp.n_pairs, (unsigned long long)__popc(m));
    b = __shfl_sync(kFull, b, 0) + (unsigned long long)__popc(m & ((1u << lane) - 1u));
    const bool stored = keep && b < (unsigned long long)bp.capacity;
    if (stored) bp.pairs[b] = pr;
    // the grouping counts the stored pairs
    const unsigned grp = __match_any_sync(kFull, stored ? pr.i : -1);
    if (stored && lane == __ffs(grp) - 1) atomicAdd(bp.qcnt + (int64_t)pr.i * bp.qstride, __popc(grp));
  }
}

__device__ __forceinline__ uint32_t block_key(uint64_t f, int shift, int width) {
  return (uint32_t)((f >> shift) & ((1ull << width) - 1ull));
}

// Exclusive scan by one CTA (phase 4, and the probe's chunk list): off[q] = sum of cnt[q' * stride]
// for q' < q (q < m), off[m] = the total. cnt is global memory written in this launch (read
// through L2) or, with GLOBAL_IN false, shared memory.
template <bool GLOBAL_IN = true>
__device__ void cta_exclusive_scan(const int32_t* cnt, int32_t stride, int64_t m, int64_t* off, int64_t* part) {
  const int T = blockDim.x;
  const int64_t per = (m + T - 1) / T;
  const int64_t a = min(m, (int64_t)threadIdx.x * per), b = min(m, a + per);
  int64_t s = 0;
  for (int64_t q = a; q < b; ++q) s += GLOBAL_IN ? __ldcg(cnt + q * stride) : cnt[q * stride];
  // inclusive scan of the threads' sums: by shuffles within each warp, then over the warp totals
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = T >> 5;
  int64_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) part[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int64_t v = lane < nw ? part[lane] : 0;
    int64_t w = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) part[lane] = w - v;  // exclusive warp offsets
    if (lane == nw - 1) off[m] = w;
  }
  __syncthreads();
  int64_t run = part[warp] + incl - s;
  for (int64_t q = a; q < b; ++q) {
    off[q] = run;
    run += GLOBAL_IN ? __ldcg(cnt + q * stride) : cnt[q * stride];
  }
  __syncthreads();
}

// Entries [a, b) of bucket (query qi, table t) against the query's fingerprint fq, 32 per warp
// step, the CTA's warps interleaved. A pair is emitted by the first table whose block agrees (so
// once), as in the probe kernel; stored pairs are counted per query.
__device__ void probe_range(const BatchParams& bp, int64_t qi, int t, uint64_t fq, int32_t a, int32_t b) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const SimhashLayout& L = bp.L;
  const uint64_t* tf = bp.hfp + (int64_t)t * bp.hn;
  const int32_t* ti = bp.hid + (int64_t)t * bp.hn;
  for (int32_t x0 = a + warp * 32; x0 < b; x0 += nwarps * 32) {
    const int32_t xx = x0 + lane;
    bool ok = false;
    int32_t j = 0, dist = 0;
    if (xx < b) {
      const uint64_t m = __ldg(reinterpret_cast<const unsigned long long*>(tf) + xx) ^ fq;
      dist = __popcll(m);
      ok = dist <= bp.hmax;
      if (ok) {
        j = __ldg(ti + xx);
        for (int u = 0; u < t && ok; ++u) ok = block_key(m, L.shift[u], L.width[u]) != 0u;
      }
    }
    const unsigned hit = __ballot_sync(kFull, ok);
    if (hit == 0u) continue;
    unsigned long long base = 0ull;
    if (lane == 0) base = atomicAdd(bp.n_hpairs, (unsigned long long)__popc(hit));
    base = __shfl_sync(kFull, base, 0);
    const unsigned long long at = base + __popc(hit & ((1u << lane) - 1u));
    const bool stored = ok && at < (unsigned long long)bp.hcapacity;
    if (stored) {
      mrc_pair pr;
      pr.i = (int32_t)qi;
      pr.j = j;
      pr.score = (float)dist;
      bp.hpairs[at] = pr;
    }
    const unsigned st = __ballot_sync(kFull, stored);
    if (st && lane == 0) atomicAdd(bp.hqcnt + qi * bp.qstride, __popc(st));
  }
}

// The bucket of item x = (query x / blocks, table x % blocks): its query's fingerprint and
// entry range.
__device__ __forceinline__ void probe_item(const BatchParams& bp, int64_t x, int64_t& qi, int& t, uint64_t& fq,
                                           int32_t& a, int32_t& b) {
  const SimhashLayout& L = bp.L;
  qi = x / L.blocks;
  t = (int)(x - qi * L.blocks);
  fq = __ldcg(reinterpret_cast<const unsigned long long*>(bp.qfp) + qi);
  const int32_t* o = bp.hoff + L.off_base[t];
  const uint32_t key = block_key(fq, L.shift[t], L.width[t]);
  a = __ldg(o + key);
  b = __ldg(o + key + 1);
}

constexpr int kProbeChunk = 2048;     // bucket entries per work unit of the chunked probe
constexpr int kProbeItemsMax = 4096;  // (query, table) items the chunked probe lists in shared memory

// Phase 3b: Hamming probe of the block-table index. Buckets differ in size by orders of
// magnitude (fingerprints of documents dominated by the same frequent terms share blocks), so
// work units are chunks of kProbeChunk entries of a bucket: every CTA lists the chunk counts of
// all items in shared memory (the same list in each CTA), and CTAs take chunks from one cursor.
// A batch with more items than kProbeItemsMax takes whole items instead.
__device__ void phase_probe(const BatchParams& bp, int64_t n, uint8_t* smem, int32_t* slot, int64_t* part) {
  if (bp.hmax < 0 || bp.hn <= 0) return;
  const int64_t items = n * bp.L.blocks;
  int64_t qi;
  int t;
  uint64_t fq;
  int32_t a, b;
  if (items > kProbeItemsMax) {
    while (true) {
      const int32_t x = cta_grab(bp.ctl + kCtlProbeCur, slot);
      if (x >= items) break;
      probe_item(bp, x, qi, t, fq, a, b);
      probe_range(bp, qi, t, fq, a, b);
    }
    return;
  }
  int32_t* cnt = reinterpret_cast<int32_t*>(smem);                        // [items] chunks per item
  int64_t* first = reinterpret_cast<int64_t*>(smem + 4 * kProbeItemsMax);  // [items + 1] first chunk
  for (int64_t x = threadIdx.x; x < items; x += blockDim.x) {
    probe_item(bp, x, qi, t, fq, a, b);
    cnt[x] = (b - a + kProbeChunk - 1) / kProbeChunk;
  }
  __syncthreads();
  cta_exclusive_scan<false>(cnt, 1, items, first, part);
  const int64_t chunks = first[items];
  __shared__ int64_t unit_s[2];
  while (true) {
    const int32_t c = cta_grab(bp.ctl + kCtlProbeCur, slot);
    if (c >= chunks) break;
    if (threadIdx.x == 0) {  // the item holding chunk c: the last x with first[x] <= c
      int64_t lo = 0, hi = items - 1;
      while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (first[mid] <= c) lo = mid;
        else hi = mid - 1;
      }
      unit_s[0] = lo;
      unit_s[1] = c - first[lo];
    }
    __syncthreads();
    const int64_t x = unit_s[0], k = unit_s[1];
    __syncthreads();
    probe_item(bp, x, qi, t, fq, a, b);
    const int32_t ca = a + (int32_t)k * kProbeChunk;
    probe_range(bp, qi, t, fq, ca, min(b, ca + kProbeChunk));
  }
}

// Phase 5: the first min(total, cap) pairs go to their query's slice of out, in the order the
// per-query cursors hand out.
__device__ void scatter_pairs(const mrc_pair* pairs, const unsigned long long* total, int64_t cap, const int64_t* off,
                              int32_t* fill, int32_t stride, mrc_pair* out) {
  const int lane = threadIdx.x & 31;
  const int64_t t = (int64_t)__ldcg(total);
  const int64_t m = t < cap ? t : cap;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < m; w0 += step) {
    const int64_t x = w0 + lane;
    mrc_pair pr{-1, 0, 0.f};
    if (x < m) {
      const int32_t* pw = reinterpret_cast<const int32_t*>(pairs + x);
      pr.i = __ldcg(pw);
      pr.j = __ldcg(pw + 1);
      pr.score = __int_as_float(__ldcg(pw + 2));
    }
    // one cursor atomic per query present in the warp
    const unsigned grp = __match_any_sync(kFull, pr.i);
    const int leader = __ffs(grp) - 1;
    int32_t base = 0;
    if (x < m && lane == leader) base = atomicAdd(fill + (int64_t)pr.i * stride, __popc(grp));
    base = __shfl_sync(grp, base, leader);
    if (x < m) out[__ldcg(off + pr.i) + base + __popc(grp & ((1u << lane) - 1u))] = pr;
  }
}

template <int FMT, int RB, int BN>
__global__ void __launch_bounds__(kResThreads, 1)
    k_batch(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB,
            const __grid_constant__ BatchParams bp) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ int32_t slot_s, ok_s;
  __shared__ int64_t part_s[kResThreads];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5;
  // the compare's 512 TMEM columns, held from the start (one CTA per SM)
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool tmem_held = true;
  auto free_tmem = [&]() {
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
      __syncwarp();
      tc_fence_after();
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
    tmem_held = false;
  };
  int64_t n = *bp.n_live;
  n = n < 0 ? 0 : (n > bp.max_docs ? bp.max_docs : n);
  unsigned target = 0;
  bool ok = true;
  int stamp = 0;
  auto mark = [&]() {
    if (blockIdx.x == 0 && threadIdx.x == 0) bp.stamps[stamp] = gtime();
    ++stamp;
  };
  mark();

  phase_list(bp, n);
  ok = grid_sync(bp, target, &ok_s);
  mark();
  if (ok) {
    phase_signature(bp, n, smem, &slot_s);
    ok = grid_sync(bp, target, &ok_s);
    mark();
  }
  if (ok) {
    // shared memory held tables (generic stores); TMA now writes it, and reads the operands
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
    const int64_t t_begin = bp.g.n_tiles * blockIdx.x / gridDim.x;
    const int64_t t_end = bp.g.n_tiles * (blockIdx.x + 1) / gridDim.x;
    resident_body<FMT, RB, BN>(&tA, &tA, &tB, &tB, bp.g, smem, tmem, t_begin, t_end);
    free_tmem();
    ok = grid_sync(bp, target, &ok_s);
    mark();
  }
  if (ok) {
    phase_rescore(bp);
    phase_probe(bp, n, smem, &slot_s, part_s);
    ok = grid_sync(bp, target, &ok_s);
    mark();
  }
  if (ok) {
    if (blockIdx.x == 0) {
      cta_exclusive_scan(bp.qcnt, bp.qstride, bp.max_docs, bp.qoff, part_s);
      if (bp.hmax >= 0) cta_exclusive_scan(bp.hqcnt, bp.qstride, bp.max_docs, bp.hqoff, part_s);
    }
    ok = grid_sync(bp, target, &ok_s);
    mark();
  }
  if (ok) {
    scatter_pairs(bp.pairs, bp.n_pairs, bp.capacity, bp.qoff, bp.qfill, bp.qstride, bp.grouped);
    if (bp.hmax >= 0) scatter_pairs(bp.hpairs, bp.n_hpairs, bp.hcapacity, bp.hqoff, bp.hqfill, bp.qstride, bp.hgrouped);
    mark();
  }
  if (tmem_held) free_tmem();
}

// Dynamic shared memory of the batch kernel: the compare's, which also holds the signature
// pass (ten warp tables, or one CTA-wide table of team_slots entries).
template <int FMT, int RB, int BN>
constexpr size_t batch_smem_bytes() {
  return resident_smem_bytes<FMT, RB, BN>();
}

template <int FMT, int RB, int BN>
cudaError_t run_batch(mrc_ctx* ctx, const BatchKernelArgs& a) {
  const mrc_index* x = a.index;
  const bool fp8 = FMT == OP_E4M3;
  CUtensorMap tA, tB;
  const int64_t kbytes = fp8 ? x->kp8 : 2ll * x->kp;
  if (!make_map(&tA, a.op, a.max_docs, kbytes, kBM, fp8, RB) ||
      !make_map(&tB, fp8 ? x->op_e4m3 : x->op_hi, x->n_docs, kbytes, BN, fp8, RB))
    return cudaErrorInvalidValue;
  BatchParams bp{};
  // signature pass (SIG mode, FP32 term table: the query operands come from FP32 weights)
  IngestParams& p = bp.ing;
  p.offsets = a.offsets;
  p.tokens = a.tokens;
  p.vocab = x->vocab;
  p.err = a.err;
  p.tinfo = x->tinfo;
  p.rinv = x->rinv;
  p.k = x->k;
  p.bf16w = 0;
  p.seed = x->params.seed;
  p.fhash = x->fhash;
  p.sig.sig_unit = a.unit;
  p.sig.simhash = a.simhash;
  if (fp8) {
    p.sig.op_e4m3 = a.op;
    p.sig.qnorm = a.qnorm;
    p.sig.kp8 = x->kp8;
  } else {
    p.sig.op_hi = a.op;
    p.sig.kp = x->kp;
  }
  p.n_live = a.n_live;
  p.n_tokens = a.max_tokens;
  p.narrow = narrow_slots(p.vocab) ? 1 : 0;
  const int kq = ingest_kq<kSIG>(p);
  constexpr size_t smem = batch_smem_bytes<FMT, RB, BN>();
  if ((size_t)(kResThreads / 32) * short_warp_bytes(kq, p.narrow != 0) > smem - 1024) return cudaErrorInvalidValue;
  int slots = kHugeSlots;
  while (slots > 1024 && long_huge_bytes(kq) - (size_t)(kHugeSlots - slots) * 10 > smem - 1024) slots >>= 1;
  if ((size_t)kq * 8 + 304 + (size_t)slots * 10 > smem - 1024) return cudaErrorInvalidValue;
  bp.team_slots = slots;
  // compare (resident kernel, query x index)
  GemmParams& g = bp.g;
  g.na = a.max_docs;
  g.nb = x->n_docs;
  g.kblocks = 1;
  g.triangle = 0;
  g.tiles_m = (g.na + kBM - 1) / kBM;
  g.tiles_n = (g.nb + BN - 1) / BN;
  g.super_rows = (g.na + BN - 1) / BN;
  g.n_tiles = g.tiles_m * g.tiles_n;
  if (g.n_tiles >= (1ll << 31)) return cudaErrorInvalidValue;
  g.thresh = a.thresh;
  g.out_scale = fp8 ? 1.0f / (kE4M3Scale * kE4M3Scale) : 1.0f;
  if (fp8) {
    g.a_norm = a.qnorm;
    g.b_norm = x->qnorm;
    g.b_norm_min = x->qnorm_min;
  }
  g.pairs = a.cand;
  g.count = a.counts + 1;
  g.capacity = a.cand_cap;
  g.err = a.err;
  g.timeout_ns = ctx->wait_limit_ns;
  g.exact = 0;
  g.stall = 0;
  g.ring = a.ring;
  g.pf = a.prefetch >= 0 ? a.prefetch : ((int64_t)g.nb * kbytes > kPrefetchMinBytes ? kPrefetchTiles : 0);
  g.na_live = a.n_live;
  g.row_rr = 0;
  // the rest of the pipeline
  bp.max_docs = a.max_docs;
  bp.n_live = a.n_live;
  bp.ctl = a.ctl;
  bp.long_list = a.long_list;
  bp.cand = a.cand;
  bp.n_cand = a.counts + 1;
  bp.cand_cap = a.cand_cap;
  bp.q_unit = a.unit;
  bp.x_unit = x->sig_unit;
  bp.k = x->k;
  bp.tau = a.tau;
  bp.pairs = a.pairs;
  bp.n_pairs = a.counts;
  bp.capacity = a.capacity;
  bp.qstride = a.qstride;
  bp.qcnt = a.qcnt;
  bp.qfill = a.qfill;
  bp.qoff = a.qoff;
  bp.grouped = a.grouped;
  bp.hmax = -1;
  if (a.shx) {
    const mrc_simhash_index* h = a.shx;
    bp.hmax = a.hmax;
    bp.L = h->layout;
    bp.hn = h->n;
    bp.hfp = h->fp;
    bp.hid = h->id;
    bp.hoff = h->off;
    bp.qfp = a.simhash;
    bp.hpairs = a.hpairs;
    bp.n_hpairs = a.hcount;
    bp.hcapacity = a.hcapacity;
    bp.hqcnt = a.hqcnt;
    bp.hqfill = a.hqfill;
    bp.hqoff = a.hqoff;
    bp.hgrouped = a.hgrouped;
  }
  bp.err = a.err;
  bp.timeout_ns = ctx->wait_limit_ns;
  bp.stamps = a.stamps;
  auto kern = k_batch<FMT, RB, BN>;
  if (resident_ctas(kern, kResThreads, smem) < 1) return cudaErrorInvalidConfiguration;
  // every CTA must be resident at once (grid barriers): one per SM, cooperative launch
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)ctx->num_sms);
  cfg.blockDim = dim3(kResThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, tA, tB, bp);
}

}  // namespace

// Compare rows of one K block: fp16 rows of 128 bytes (k <= 64), E4M3 rows of 64 or 128 bytes
// (k <= 128). Rows are padded to 64 entries, so fp16 rows of 64 bytes do not occur.
bool batch_kernel_supported(const mrc_index* x) {
  if (x->params.precision == MRC_PREC_BF16_FP8) return x->kp8 == 64 || x->kp8 == 128;
  return 2ll * x->kp == 128;
}

cudaError_t launch_batch_kernel(mrc_ctx* ctx, const BatchKernelArgs& a) {
  const mrc_index* x = a.index;
  if (!batch_kernel_supported(x) || a.max_docs < 1 || x->n_docs < 1) return cudaErrorInvalidValue;
  const bool fp8 = x->params.precision == MRC_PREC_BF16_FP8;
  const int64_t kbytes = fp8 ? x->kp8 : 2ll * x->kp;
  // 128-column tiles unless asked otherwise: a batch has few row blocks, and with four TMEM
  // accumulators in flight the index streams faster than with two 256-column ones
  const bool wide = a.tile_n == 256;
  if (fp8) {
    if (kbytes == 64) return wide ? run_batch<OP_E4M3, 64, 256>(ctx, a) : run_batch<OP_E4M3, 64, 128>(ctx, a);
    return wide ? run_batch<OP_E4M3, 128, 256>(ctx, a) : run_batch<OP_E4M3, 128, 128>(ctx, a);
  }
  return wide ? run_batch<OP_F16, 128, 256>(ctx, a) : run_batch<OP_F16, 128, 128>(ctx, a);
}

}  // namespace mrc
