// tc_dev.cuh -- device code of the tensor-core compare (tcgen05 MMA, TMEM accumulators, TMA
// operand loads, bounded mbarrier waits, the thresholding epilogue), shared by the compare
// kernels (compare_tc.cu) and the persistent batch kernel (batch_kernel.cu).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

constexpr int kBM = 128;
constexpr int kThreads = 192;
constexpr int kRowBytes = 128;  // K bytes per stage per row (one 128B swizzle atom)
// After a role gives up, the CTA still waits for its own TMA copies and MMAs in flight before it
// frees TMEM and exits. They complete in microseconds; the bound only keeps a broken invariant
// from spinning forever (it is then reported as a timeout too).
constexpr uint64_t kDrainNs = 2000000000ull;
constexpr int kPairBuf = 256;  // pairs buffered per epilogue warp (then its fill count)
constexpr int kFlushAt = 192;  // a warp flushes its buffer to the global list at this many pairs
constexpr size_t kWarpPairBytes = kPairBuf * sizeof(mrc_pair) + 16;  // one warp's buffer and count
constexpr float kNormLo = 0.93f;  // lower bound of |e4m3(x * 256)| / 256 for unit x (1 - 2^-4 = 0.9375)

template <int FMT>
struct Cfg;
template <>
struct Cfg<OP_SPLIT16> {
  static constexpr int BN = 128, NOPS = 2, STAGES = 3, ACCS = 2;
};
template <>
struct Cfg<OP_F16> {
  static constexpr int BN = 256, NOPS = 1, STAGES = 4, ACCS = 1;
};
template <>
struct Cfg<OP_E4M3> {
  static constexpr int BN = 256, NOPS = 1, STAGES = 4, ACCS = 1;
};

struct GemmParams {
  int64_t na, nb;
  int32_t kblocks;
  int32_t triangle;
  int64_t tiles_m, tiles_n, super_rows, n_tiles;
  float thresh, out_scale;
  const float* a_norm;
  const float* b_norm;
  const float* b_norm_min;  // [ceil(nb / 128)] smallest non-zero b_norm of each 128-column block
  mrc_pair* pairs;
  unsigned long long* count;
  int64_t capacity;
  float* store;
  __half* store16;
  int64_t ld;
  int32_t* err;
  int32_t row_rr;  // resident kernel, triangle: whole row blocks dealt round-robin (see TileSeq)
  const int32_t* kblocks_dev;  // streaming kernel: K blocks read from the device (see GemmArgs)
  uint64_t timeout_ns;         // bound of every pipeline wait (the context's wait limit)
  int32_t exact;               // E4M3: exact candidate test and quantized-cosine scores (see emit_chunk)
  int32_t stall;               // failure-detection test: the MMA issuer issues nothing, so the
                               // other roles' waits for its results run out (mrc_ctx_set_test_stall)
  int32_t pf;                  // resident kernel, contiguous order: B tiles prefetched into L2 this
                               // many tiles ahead of their loads (0: none)
  int32_t ring;                // resident kernel: B ring depth (0: as many stages as shared memory holds)
  const int64_t* na_live;      // non-null: rows from *na_live on emit nothing (the batch's padding)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count));
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false on abort (another role gave up) or timeout (records it).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort, int32_t* err,
                                          uint64_t timeout_ns) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtime();
  while (true) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (mbar_try(b, parity)) return true;
    if (*abort) return false;
    if (gtime() - t0 > timeout_ns) {
      *abort = 1;
      set_err(err, kErrTimeout);
      return false;
    }
  }
}
// Drain wait of the abort path: the copy or MMA behind the barrier was issued and completes on
// its own; the bound is a safeguard only.
__device__ __forceinline__ void mbar_drain(uint64_t* b, uint32_t parity, int32_t* err) {
  const uint64_t t0 = gtime();
  while (!mbar_try(b, parity)) {
    if (gtime() - t0 > kDrainNs) {
      set_err(err, kErrTimeout);
      return;
    }
  }
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B type code 0 (F16 for kind::f16,
// E4M3 for kind::f8f6f4), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

template <int FMT>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (FMT == OP_E4M3) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(
            d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  } else {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(id), "r"(acc));
  }
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%"
      "19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
// The same load, which also returns the largest of the 32 values each thread loads (the
// reduction of tcgen05.ld.red, sm_103a): a chunk's row maximum at no ALU cost.
__device__ __forceinline__ void tmem_ld32_max(uint32_t taddr, float (&v)[32], float& m) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x32.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
      "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, %32, [%33];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=f"(m)
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// L2 prefetch of one tensor-map tile (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* tm, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"((uint64_t)tm), "r"(x), "r"(y)
               : "memory");
}

// Three-input maximum (one instruction on sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// Maximum of 32 registers as a tree of three-input maxima: 15 instructions, 4 levels deep, so
// the chains of several chunks overlap instead of waiting on one 31-step dependency chain.
__device__ __forceinline__ float max32(const float (&v)[32]) {
  float a[11];
#pragma unroll
  for (int e = 0; e < 10; ++e) a[e] = fmax3(v[3 * e], v[3 * e + 1], v[3 * e + 2]);
  a[10] = fmaxf(v[30], v[31]);
  const float b0 = fmax3(a[0], a[1], a[2]), b1 = fmax3(a[3], a[4], a[5]), b2 = fmax3(a[6], a[7], a[8]);
  return fmax3(fmax3(a[9], a[10], b0), b1, b2);
}

// Writes a warp's buffered pairs (min(*fill, kPairBuf) slots of buf) to the global list with
// one atomic and empties the buffer. Slots with i < 0 are holes (a lane whose hits did not fit
// sent them out directly) and are skipped. Called by the whole warp.
__device__ __forceinline__ void flush_pairs(const GemmParams& p, mrc_pair* buf, int32_t* fill, int lane) {
  __syncwarp();
  const int n = min(*fill, kPairBuf);
  int valid = 0;
  for (int x = lane; x < n; x += 32) valid += buf[x].i >= 0 ? 1 : 0;
  valid = warp_sum(valid);
  if (valid) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(p.count, (unsigned long long)valid);
    base = __shfl_sync(kFull, base, 0);
    for (int b0 = 0; b0 < n; b0 += 32) {
      const int x = b0 + lane;
      const bool ok = x < n && buf[x].i >= 0;
      const unsigned bal = __ballot_sync(kFull, ok);
      const unsigned long long at = base + __popc(bal & ((1u << lane) - 1u));
      if (ok && at < (unsigned long long)p.capacity) p.pairs[at] = buf[x];
      base += __popc(bal);
    }
  }
  __syncwarp();
  if (lane == 0) *fill = 0;
  __syncwarp();
}

// Threshold one 32-column chunk held in registers (v[e] = score of column j0 + e for this
// lane's row i; m = this lane's maximum over the chunk) and append its pairs to the warp's
// buffer. The usual case, no lane at fast_thresh, costs one vote. Otherwise each lane builds
// the 32-bit mask of its hits straight from its registers and applies the bounds and the
// triangle's j > i with bit arithmetic; fp16: a hit is v[e] >= hit_lim (= fast_thresh),
// scored with v[e]. E4M3: a hit passes the row's block bound (fast_thresh, which uses the
// smallest column norm of the 128-column block); the caller rescores every hit in FP32, so
// the raw accumulator is its score. With p.exact (the candidates themselves are the result)
// each such hit is tested exactly, v[e] >= hit_lim * |q_j| with the column's norm (zero norms
// never hit), and scored with the cosine of the quantized vectors. A lane with hits stages its
// scores in its row of the warp's 32 x 33 area (so that the loops below index them at run time
// and stay compact: they run only for the rare chunks with hits), reserves its buffer slots
// with one shared-memory atomic and writes its hits; the warp flushes at kFlushAt pairs.
template <int FMT>
__device__ __forceinline__ void emit_chunk(const GemmParams& p, const float (&v)[32], float m, int64_t i, int64_t j0,
                                           int lane, float fast_thresh, float row_norm, float hit_lim, float* stage,
                                           mrc_pair* buf, int32_t* fill) {
  if (!__any_sync(kFull, m >= fast_thresh)) return;
  uint32_t mask = 0;
  if (FMT != OP_E4M3 || row_norm > 0.f) {
#pragma unroll
    for (int e = 0; e < 32; ++e) mask |= (v[e] >= fast_thresh ? 1u : 0u) << e;
  }
  const int64_t lim = p.nb - j0;  // columns j0 + e < nb
  if (lim < 32) mask &= lim <= 0 ? 0u : ((1u << lim) - 1u);
  if (p.triangle) {  // j0 + e > i
    const int64_t dlt = i - j0;
    if (dlt >= 31) mask = 0u;
    else if (dlt >= 0) mask &= ~((2u << dlt) - 1u);
  }
  if (i >= p.na || (p.na_live && i >= *p.na_live)) mask = 0u;
  if (mask) {
    float* sc = stage + lane * 33;
#pragma unroll
    for (int e = 0; e < 32; ++e) sc[e] = v[e];
    if (FMT == OP_E4M3 && p.exact) {
      for (uint32_t hh = mask; hh; hh &= hh - 1u) {
        const int e = __ffs(hh) - 1;
        const float nj = __ldg(p.b_norm + j0 + e);
        if (nj > 0.f && sc[e] >= hit_lim * nj)
          sc[e] = sc[e] * p.out_scale / (row_norm * nj);  // the cosine of the quantized vectors
        else
          mask &= ~(1u << e);
      }
    }
    const int cnt = __popc(mask);
    if (cnt) {
      int pos = atomicAdd(fill, cnt);
      const bool direct = pos + cnt > kPairBuf;
      unsigned long long g = 0;
      if (direct) {  // no room: holes in the slots reserved inside the buffer, the hits go out directly
        for (int x = pos; x < kPairBuf && x < pos + cnt; ++x) buf[x].i = -1;
        g = atomicAdd(p.count, (unsigned long long)cnt);
      }
      for (uint32_t hh = mask; hh; hh &= hh - 1u) {
        const int e = __ffs(hh) - 1;
        mrc_pair pr;
        pr.i = (int32_t)i;
        pr.j = (int32_t)(j0 + e);
        pr.score = sc[e];
        if (!direct) {
          buf[pos++] = pr;
        } else {
          if (g < (unsigned long long)p.capacity) p.pairs[g] = pr;
          ++g;
        }
      }
    }
  }
  __syncwarp();
  if (*fill >= kFlushAt) flush_pairs(p, buf, fill, lane);
}


// ---------------------------------------------------------------------------------------
// Small-K variant (one K block per row: 64- or 128-byte operand rows). Each CTA walks a
// contiguous, row-major range of tiles, so consecutive tiles share their A rows: A is
// loaded once per row block into one of two resident buffers and only B streams through
// a 4-stage ring. Eight epilogue warps (two per TMEM lane quarter) split the columns.
constexpr int kResEpiWarps = 8;  // epilogue warps: two per TMEM lane quarter, each half of the tile's columns
constexpr int kResThreads = 64 + 32 * kResEpiWarps;  // warp 0 TMA, warp 1 MMA + TMEM, then the epilogue
// Depth of the streamed-B ring: as many stages as shared memory holds next to the two A
// buffers and the epilogue's staging. The B tiles come from L2 with a latency of about
// a microsecond, so a CTA needs that many bytes in flight to stream at the rate its tensor core
// consumes them (E4M3 tiles are half the size of fp16 ones and go by twice as fast). 3 to 12.
constexpr size_t kResEpiBytes = kResEpiWarps * (kWarpPairBytes + 32 * 33 * sizeof(float));
__host__ __device__ constexpr int res_stages_b(int nops, int rb, int bn) {
  return (int)(((227u * 1024u - 1024u - kResEpiBytes - 512u) - 2u * nops * kBM * rb) / ((size_t)nops * bn * rb)) > 12
             ? 12
             : (int)(((227u * 1024u - 1024u - kResEpiBytes - 512u) - 2u * nops * kBM * rb) / ((size_t)nops * bn * rb));
}

// 64-byte-swizzle descriptor (8-row groups 512 bytes apart) or the 128-byte one.
template <int RB>
__device__ __forceinline__ uint64_t sdesc_rb(uint32_t saddr) {
  if (RB == 128) return sdesc(saddr);
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Row-major tile order: row block bi (units of 128), column block bj (units of BN).
// Triangle: row bi holds column blocks floor(bi / H) .. C - 1 (H = BN / 128).
template <int BN>
__device__ __forceinline__ bool decode_rowmajor(const GemmParams& p, int64_t t64, int64_t& bi, int64_t& bj) {
  const int32_t t = (int32_t)t64;
  if (!p.triangle) {
    const int32_t tn = (int32_t)p.tiles_n;
    bi = t / tn;
    bj = t - (int32_t)bi * tn;
    return true;
  }
  constexpr int H = BN / kBM;
  const int32_t C = (int32_t)p.super_rows;
  // super row I (H row blocks, C - I tiles each) starts at H * (I*C - I*(I-1)/2)
  const float b = 2.0f * (float)C + 1.0f;
  const float s = (float)t / (float)H;
  int32_t I = (int32_t)((b - sqrtf(fmaxf(b * b - 8.0f * s, 0.0f))) * 0.5f);
  I = I < 0 ? 0 : (I > C - 1 ? C - 1 : I);
  while (I > 0 && H * (I * C - I * (I - 1) / 2) > t) --I;
  while (I + 1 < C && H * ((I + 1) * C - (I + 1) * I / 2) <= t) ++I;
  const int32_t r = t - H * (I * C - I * (I - 1) / 2);
  const int32_t w = C - I;
  const int32_t h = r / w;
  bj = I + (r - h * w);
  bi = (int64_t)I * H + h;
  return bi * kBM < p.na;
}

// The tiles of one CTA of the resident kernel, in the order all its roles walk them.
// Contiguous mode: tiles [t_begin, t_end) of the row-major order (even shares; used when the
// streamed operand fits in L2). Round-robin mode (triangle with a streamed operand larger
// than L2 can hold): CTA c of G takes whole row blocks, kG + c in even rounds k and
// kG + G - 1 - c in odd rounds (two rounds give every CTA the same work), each swept from its
// diagonal column block up. The CTAs then sweep the column blocks together, a few dozen
// blocks apart, so a streamed tile is read from HBM once and served to the other CTAs by L2
// instead of every CTA streaming the whole operand at its own position.
template <int BN>
struct TileSeq {
  int64_t t, t_end, k, bi, bj;
  __device__ TileSeq(int64_t tb, int64_t te) : t(tb), t_end(te), k(-1), bi(0), bj(0) {}
  __device__ __forceinline__ bool next(const GemmParams& p, int64_t& obi, int64_t& obj) {
    constexpr int H = BN / kBM;
    if (!p.row_rr) {
      // the first tile is decoded, the following ones are stepped to in row-major order
      if (t >= t_end) return false;
      if (k < 0) {
        k = 0;
        decode_rowmajor<BN>(p, t, bi, bj);
      }
      if (bi * kBM >= p.na) return false;  // row blocks past the last row come last in the order
      obi = bi;
      obj = bj;
      ++t;
      if (++bj >= (p.triangle ? p.super_rows : p.tiles_n)) {
        ++bi;
        bj = p.triangle ? bi / H : 0;
      }
      return true;
    }
    while (k < 0 || bj >= p.super_rows) {
      ++k;
      const int64_t G = gridDim.x, c = blockIdx.x;
      bi = k * G + ((k & 1) ? G - 1 - c : c);
      if (bi >= p.tiles_m) return false;
      bj = bi / H;
    }
    obi = bi;
    obj = bj++;
    return true;
  }
};


// Dynamic shared memory of the resident kernel (at least 120 KB, so that one CTA, which owns
// all 512 TMEM columns, runs per SM).
template <int FMT, int RB, int BN>
__host__ __device__ constexpr size_t resident_smem_bytes() {
  using C = Cfg<FMT>;
  constexpr int NBUF = 512 / (C::ACCS * BN);
  constexpr int SB = res_stages_b(C::NOPS, RB, BN);
  constexpr size_t need = 1024 + 2 * (size_t)C::NOPS * kBM * RB + (size_t)SB * C::NOPS * BN * RB +
                         (size_t)(8 + 2 * SB + 2 * NBUF) * 8 + kResEpiBytes;
  return need > 120 * 1024 ? need : 120 * 1024;
}

// The roles of the resident kernel over tiles [t_begin, t_end) of its order, in shared memory
// `smem` (1024-byte aligned, resident_smem_bytes) with the CTA's 512 TMEM columns at `tmem`
// (allocated and freed by the caller). Called by all kResThreads threads of the CTA.
template <int FMT, int RB, int BN>
__device__ __forceinline__ void resident_body(const CUtensorMap* tA0, const CUtensorMap* tA1,
                                              const CUtensorMap* tB0, const CUtensorMap* tB1, const GemmParams& p,
                                              uint8_t* smem, uint32_t tmem, int64_t t_begin, int64_t t_end) {
  using C = Cfg<FMT>;
  // as many accumulator buffers as TMEM's 512 columns hold (2 at N = 256, 4 at N = 128): the MMA
  // runs that many tiles ahead of the epilogue's TMEM reads
  constexpr int NB = 512 / (C::ACCS * BN);
  static_assert(NB >= 2 && NB <= 4, "two to four accumulator buffers");
  constexpr uint32_t A_BYTES = kBM * RB, B_BYTES = BN * RB;
  constexpr uint32_t A_STAGE = C::NOPS * A_BYTES, B_STAGE = C::NOPS * B_BYTES;
  constexpr int kResStagesB = res_stages_b(C::NOPS, RB, BN);
  static_assert(kResStagesB >= 3, "at least three B stages");
  // B ring depth: p.ring stages if set (2 or more), else all that fit
  const int SB = (p.ring >= 2 && p.ring < kResStagesB) ? p.ring : kResStagesB;
  uint8_t* abuf = smem;                    // [2][A_STAGE]
  uint8_t* bbuf = smem + 2 * A_STAGE;      // [kResStagesB][B_STAGE]
  uint64_t* bar = reinterpret_cast<uint64_t*>(bbuf + kResStagesB * B_STAGE);
  uint64_t* a_full = bar;
  uint64_t* a_empty = bar + 2;
  uint64_t* b_full = bar + 4;
  uint64_t* b_empty = b_full + kResStagesB;
  uint64_t* acc_full = b_empty + kResStagesB;
  uint64_t* acc_empty = acc_full + NB;
  uint64_t* drain = acc_empty + NB;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(drain + 1);
  float* stage_all = reinterpret_cast<float*>(drain + 4);  // [epilogue warps][32 x 33] scores
  uint8_t* pbuf_all = reinterpret_cast<uint8_t*>(stage_all + kResEpiWarps * 32 * 33);  // [epilogue warps] pairs, fill

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* stage = stage_all + (warp >= 2 ? warp - 2 : 0) * 32 * 33;
  mrc_pair* pbuf = reinterpret_cast<mrc_pair*>(pbuf_all + (warp >= 2 ? warp - 2 : 0) * kWarpPairBytes);
  int32_t* pfill = reinterpret_cast<int32_t*>(pbuf + kPairBuf);
  if (warp >= 2 && (threadIdx.x & 31) == 0) *pfill = 0;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&a_full[b], 1);
      mbar_init(&a_empty[b], 1);
    }
    for (int b = 0; b < NB; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kResEpiWarps);
    }
    for (int s = 0; s < kResStagesB; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (warp == 0) {
    if (lane == 0) {
      // ------------------------------------------------------------ TMA producer
      int32_t a_armed[2] = {-1, -1};
      int32_t b_armed[kResStagesB];
      for (int s = 0; s < kResStagesB; ++s) b_armed[s] = -1;
      uint32_t stage = 0, phase = 0, a_use = 0;
      int64_t last_bi = -1;
      TileSeq<BN> seq(t_begin, t_end);
      int64_t bi, bj;
      // contiguous order: the B tile p.pf tiles ahead is prefetched into L2 as each tile is
      // loaded, so a load waits for L2 rather than for DRAM and the ring's shared memory does
      // not bound the DRAM bytes in flight
      const bool pf = p.pf > 0 && !p.row_rr;
      TileSeq<BN> ahead(t_begin, t_end);
      int64_t pbi, pbj;
      if (pf)
        for (int u = 0; u < p.pf && ahead.next(p, pbi, pbj); ++u) {
          tma_prefetch_2d(tB0, 0, (int)(pbj * BN));
          if (C::NOPS == 2) tma_prefetch_2d(tB1, 0, (int)(pbj * BN));
        }
      while (seq.next(p, bi, bj)) {
        if (bi != last_bi) {
          const uint32_t ab = a_use & 1u;
          if (!mbar_wait(&a_empty[ab], ((a_use >> 1) & 1u) ^ 1u, abort_flag, p.err, p.timeout_ns)) break;
          mbar_expect_tx(&a_full[ab], A_STAGE);
          a_armed[ab] = (int32_t)((a_use >> 1) & 1u);
          uint8_t* dst = abuf + ab * A_STAGE;
          tma_load_2d(dst, tA0, 0, (int)(bi * kBM), &a_full[ab]);
          if (C::NOPS == 2) tma_load_2d(dst + A_BYTES, tA1, 0, (int)(bi * kBM), &a_full[ab]);
          last_bi = bi;
          ++a_use;
        }
        if (!mbar_wait(&b_empty[stage], phase ^ 1u, abort_flag, p.err, p.timeout_ns)) break;
        mbar_expect_tx(&b_full[stage], B_STAGE);
        b_armed[stage] = (int32_t)phase;
        uint8_t* dst = bbuf + stage * B_STAGE;
        tma_load_2d(dst, tB0, 0, (int)(bj * BN), &b_full[stage]);
        if (C::NOPS == 2) tma_load_2d(dst + B_BYTES, tB1, 0, (int)(bj * BN), &b_full[stage]);
        if (pf && ahead.next(p, pbi, pbj)) {
          tma_prefetch_2d(tB0, 0, (int)(pbj * BN));
          if (C::NOPS == 2) tma_prefetch_2d(tB1, 0, (int)(pbj * BN));
        }
        if (++stage == SB) {
          stage = 0;
          phase ^= 1u;
        }
      }
      // drain: every armed copy lands before the CTA may exit
      for (int b = 0; b < 2; ++b) {
        if (a_armed[b] < 0) continue;
        mbar_drain(&a_full[b], (uint32_t)a_armed[b], p.err);
      }
      for (int s = 0; s < kResStagesB; ++s) {
        if (b_armed[s] < 0) continue;
        mbar_drain(&b_full[s], (uint32_t)b_armed[s], p.err);
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && !p.stall) {
      // ------------------------------------------------------------ MMA issuer
      const uint32_t id = idesc(BN);
      uint32_t stage = 0, phase = 0, a_use = 0, ab_a = 0;
      int64_t last_bi = -1, it = 0;
      TileSeq<BN> seq(t_begin, t_end);
      int64_t bi, bj;
      while (seq.next(p, bi, bj)) {
        if (bi != last_bi) {
          if (last_bi >= 0) umma_commit(&a_empty[ab_a]);  // previous row's MMAs release its A buffer
          ab_a = a_use & 1u;
          if (!mbar_wait(&a_full[ab_a], (a_use >> 1) & 1u, abort_flag, p.err, p.timeout_ns)) break;
          last_bi = bi;
          ++a_use;
        }
        const uint32_t ab = (uint32_t)(it % NB);
        if (!mbar_wait(&acc_empty[ab], (uint32_t)((it / NB) & 1) ^ 1u, abort_flag, p.err, p.timeout_ns)) break;
        if (!mbar_wait(&b_full[stage], phase, abort_flag, p.err, p.timeout_ns)) break;
        tc_fence_after();
        const uint32_t d0 = tmem + ab * (uint32_t)(C::ACCS * BN), d1 = d0 + (uint32_t)BN;
        const uint32_t sa = smem_u32(abuf + ab_a * A_STAGE), sb = smem_u32(bbuf + stage * B_STAGE);
        // descriptors built once per tile; a 32-byte K step adds 2 to the start-address field
        const uint64_t ad0 = sdesc_rb<RB>(sa), bd0 = sdesc_rb<RB>(sb);
        const uint64_t al0 = sdesc_rb<RB>(sa + A_BYTES), bl0 = sdesc_rb<RB>(sb + B_BYTES);
#pragma unroll
        for (int kk = 0; kk < RB / 32; ++kk) {
          const uint32_t first = kk == 0 ? 0u : 1u;
          umma<FMT>(d0, ad0 + 2 * kk, bd0 + 2 * kk, id, first);
          if (C::NOPS == 2) {
            umma<FMT>(d1, ad0 + 2 * kk, bl0 + 2 * kk, id, first);
            umma<FMT>(d1, al0 + 2 * kk, bd0 + 2 * kk, id, 1u);
          }
        }
        umma_commit(&b_empty[stage]);
        umma_commit(&acc_full[ab]);
        if (++stage == SB) {
          stage = 0;
          phase ^= 1u;
        }
        ++it;
      }
      // every MMA issued completes before the CTA frees TMEM (a CTA without tiles issued none)
      if (it > 0) {
        umma_commit(drain);
        mbar_drain(drain, 0, p.err);
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    // kResEpiWarps / 4 warps per TMEM lane quarter, each a contiguous share of the columns
    constexpr int PARTS = kResEpiWarps / 4;
    constexpr int CH = BN / 32 / PARTS;  // 32-column chunks per warp
    static_assert(CH >= 1 && CH * 32 * PARTS == BN, "columns split evenly over the epilogue warps");
    const int q = warp & 3;
    const int half = (warp - 2) >> 2;  // which share of the tile's columns
    int64_t it = 0;
    TileSeq<BN> ahead(t_begin, t_end);
    int64_t bi, bj, nbi = -1, nbj = -1;
    bool have_next = ahead.next(p, nbi, nbj);
    // E4M3: the score is the cosine of the quantized vectors, acc * out_scale / (|q_i| |q_j|);
    // raw accumulators below thresh * |q_i| * min_j |q_j| / out_scale (minimum over the warp's
    // 128-column block) cannot reach the threshold (fast path). The row's values change only
    // with the row block; the block minimum of the next tile is loaded one tile ahead.
    int64_t row_of = -1;
    float row_norm = 1.f, hit_lim = p.thresh, row_bound = p.thresh;
    const int64_t nbk = (p.nb + 127) >> 7;
    auto block_min = [&](int64_t cj) {
      const int64_t b = ((cj * BN) >> 7) + ((half * CH * 32) >> 7);
      return b < nbk ? __ldg(p.b_norm_min + b) : 1.f;
    };
    float nmin_next = (FMT == OP_E4M3 && have_next) ? block_min(nbj) : 1.f;
    while (have_next) {
      bi = nbi;
      bj = nbj;
      const float nmin = nmin_next;
      have_next = ahead.next(p, nbi, nbj);
      if (FMT == OP_E4M3 && have_next) nmin_next = block_min(nbj);
      const uint32_t ab = (uint32_t)(it % NB);
      const int64_t i = bi * kBM + q * 32 + lane;
      if (FMT == OP_E4M3 && bi != row_of) {
        row_of = bi;
        row_norm = i < p.na ? __ldcg(p.a_norm + i) : 0.f;  // L2: may be written earlier in the same kernel
        hit_lim = p.thresh * row_norm / p.out_scale;
        row_bound = p.thresh > 0.f ? (row_norm > 0.f ? hit_lim : __int_as_float(0x7f800000))
                                   : -__int_as_float(0x7f800000);
      }
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&acc_full[ab], (uint32_t)((it / NB) & 1), abort_flag, p.err, p.timeout_ns) ? 1 : 0;
      ok = __shfl_sync(kFull, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + ab * (uint32_t)(C::ACCS * BN);
      // all of this warp's TMEM loads are issued before one wait, so they overlap; with one
      // accumulator the load also reduces each chunk to its row maximum
      float v[CH][32];
      float mc[CH];
      if (C::ACCS == 2) {
#pragma unroll
        for (int c = 0; c < CH; ++c) tmem_ld32(trow + (half * CH + c) * 32, v[c]);
        float x[CH][32];
#pragma unroll
        for (int c = 0; c < CH; ++c) tmem_ld32(trow + BN + (half * CH + c) * 32, x[c]);
        tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < CH; ++c) {
#pragma unroll
          for (int e = 0; e < 32; ++e) v[c][e] = fmaf(x[c][e], 1.0f / kSplitLoScale, v[c][e]);
          mc[c] = max32(v[c]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < CH; ++c) tmem_ld32_max(trow + (half * CH + c) * 32, v[c], mc[c]);
        tmem_wait_ld();
      }
      // the accumulators are in registers: hand the TMEM buffer back before thresholding
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
      // a warp's columns lie in one 128-column block, so one fast threshold covers all its
      // chunks; the usual case, no lane near it in any chunk, costs one vote on the maxima
      const float fast_thresh = (FMT == OP_E4M3 && p.thresh > 0.f) ? row_bound * nmin : row_bound;
      float mall = mc[0];
#pragma unroll
      for (int c = 1; c < CH; ++c) mall = fmaxf(mall, mc[c]);
      if (__any_sync(kFull, mall >= fast_thresh)) {
#pragma unroll
        for (int c = 0; c < CH; ++c) {
          const int64_t j0 = bj * BN + (half * CH + c) * 32;
          emit_chunk<FMT>(p, v[c], mc[c], i, j0, lane, fast_thresh, row_norm, hit_lim, stage, pbuf, pfill);
        }
      }
      ++it;
    }
    flush_pairs(p, pbuf, pfill, lane);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

// 2D K-major operand map: rows x row_bytes, box = box_bytes (64 or 128) x box_rows,
// swizzle of the same width, zero fill out of bounds.
bool make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t row_bytes, int box_rows, bool fp8,
              int box_bytes = kRowBytes) {
  auto fn = encode_fn();
  if (!fn || rows <= 0) return false;
  const int eb = fp8 ? 1 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)(row_bytes / eb), (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {(cuuint32_t)(box_bytes / eb), (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  const CUtensorMapSwizzle sw = box_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  const CUresult r = fn(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                        const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace
}  // namespace mrc
