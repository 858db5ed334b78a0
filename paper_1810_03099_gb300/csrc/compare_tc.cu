// compare_tc.cu -- tensor-core comparison of unit vectors with a fused epilogue (rows a5 and a8).
//
// Computes scores S = A B^T (A, B row-major with a padded K; rows are unit
// signatures for the signature comparison of Eq. 2, or unit TF-IDF vectors
// restricted to frequent terms for the exact cosine of Eq. 1), one 128 x BN
// output tile at a time, and either keeps the pairs with score >= threshold
// (warp-ballot compaction into a global list with an atomic cursor) or
// stores the tile as FP32 (the exact-cosine head, completed by tail.cu).
//
// Blackwell (sm_103a) structure, one persistent CTA per SM, warp-specialised:
//   warp 0     : TMA producer (cp.async.bulk.tensor, 128-byte swizzle) into a
//                ring of shared-memory stages guarded by mbarriers;
//   warp 1     : allocates the 512 TMEM columns; one lane issues tcgen05.mma
//                (cta_group::1, M = 128) into double-buffered TMEM accumulators
//                and tcgen05.commit's the stage / accumulator barriers;
//   warps 2..5 : epilogue, tcgen05.ld 32 columns at a time from their 32-lane
//                TMEM quarter, threshold / store, then hand the buffer back.
// Operand formats:
//   SPLIT16: x = hi + lo * 2^-12 with hi, lo fp16; S = Ahi Bhi + 2^-12 (Ahi Blo + Alo Bhi)
//            in two FP32 accumulators (error ~2^-22 relative: FP32-accurate scores);
//   F16    : one fp16 operand pair, one accumulator;
//   E4M3   : fp8 operands (unit vectors scaled by 256), kind::f8f6f4, score = acc / 65536.
// Every wait is bounded (4 s): on expiry the kernel records kErrTimeout,
// drains its own copies and MMAs (bounded), frees TMEM and returns.
#include "tc_dev.cuh"

namespace mrc {
namespace {

// Tile t -> (row block bi in units of 128, column block bj in units of BN). 32-bit integer
// and FP32 arithmetic only (the host guarantees n_tiles < 2^31 and super_rows^2 < 2^31).
template <int BN>
__device__ __forceinline__ bool decode_tile(const GemmParams& p, int64_t t64, int64_t& bi, int64_t& bj) {
  const int32_t t = (int32_t)t64;
  if (!p.triangle) {
    const int32_t tm = (int32_t)p.tiles_m;
    bi = t % tm;
    bj = t / tm;
    return true;
  }
  constexpr int H = BN / kBM;  // 1 or 2 row blocks per super tile
  const int32_t s = t / H;
  const int32_t h = t - s * H;
  const int32_t R = (int32_t)p.super_rows;
  // row-major upper triangle of R x R super tiles: row I starts at I*R - I*(I-1)/2
  const float b = 2.0f * (float)R + 1.0f;
  int32_t I = (int32_t)((b - sqrtf(fmaxf(b * b - 8.0f * (float)s, 0.0f))) * 0.5f);
  I = I < 0 ? 0 : (I > R - 1 ? R - 1 : I);
  while (I > 0 && I * R - I * (I - 1) / 2 > s) --I;
  while (I + 1 < R && (I + 1) * R - (I + 1) * I / 2 <= s) ++I;
  const int32_t J = I + (s - (I * R - I * (I - 1) / 2));
  bi = (int64_t)I * H + h;
  bj = J;
  return bi * kBM < p.na;
}


// Streaming kernel (any K): every CTA loads its own A and B tiles into a STAGES-deep ring.
template <int FMT>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_compare(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
                   const __grid_constant__ CUtensorMap tB0, const __grid_constant__ CUtensorMap tB1, GemmParams p) {
  using C = Cfg<FMT>;
  constexpr int BN = C::BN;
  constexpr uint32_t A_BYTES = kBM * kRowBytes;
  constexpr uint32_t B_BYTES = BN * kRowBytes;
  constexpr uint32_t STAGE_BYTES = C::NOPS * (A_BYTES + B_BYTES);
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * STAGE_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* drain = acc_empty + 2;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(drain + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 2);
  float* stage_all = reinterpret_cast<float*>(drain + 4);  // [4 epilogue warps][32 x 33] scores
  uint8_t* pbuf_all = reinterpret_cast<uint8_t*>(stage_all + 4 * 32 * 33);  // [4 epilogue warps] pairs, fill

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* stage = stage_all + (warp >= 2 ? warp - 2 : 0) * 32 * 33;
  mrc_pair* pbuf = reinterpret_cast<mrc_pair*>(pbuf_all + (warp >= 2 ? warp - 2 : 0) * kWarpPairBytes);
  int32_t* pfill = reinterpret_cast<int32_t*>(pbuf + kPairBuf);
  if (warp >= 2 && (threadIdx.x & 31) == 0) *pfill = 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int32_t kblocks = p.kblocks_dev ? *p.kblocks_dev : p.kblocks;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t stage = 0, phase = 0;
      int32_t armed[C::STAGES];
      for (int s = 0; s < C::STAGES; ++s) armed[s] = -1;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < p.n_tiles && ok; t += gridDim.x) {
        int64_t bi, bj;
        if (!decode_tile<BN>(p, t, bi, bj)) continue;
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, p.err, p.timeout_ns)) {
            ok = false;
            break;
          }
          uint8_t* sbase = smem + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], STAGE_BYTES);
          armed[stage] = (int32_t)phase;
          const int x = kb * (FMT == OP_E4M3 ? kRowBytes : kRowBytes / 2);
          tma_load_2d(sbase, &tA0, x, (int)(bi * kBM), &full[stage]);
          tma_load_2d(sbase + A_BYTES, &tB0, x, (int)(bj * BN), &full[stage]);
          if (C::NOPS == 2) {
            tma_load_2d(sbase + A_BYTES + B_BYTES, &tA1, x, (int)(bi * kBM), &full[stage]);
            tma_load_2d(sbase + 2 * A_BYTES + B_BYTES, &tB1, x, (int)(bj * BN), &full[stage]);
          }
          if (++stage == C::STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      // drain: the last copy armed on each stage lands before the CTA may exit
      for (int s = 0; s < C::STAGES; ++s) {
        if (armed[s] < 0) continue;
        mbar_drain(&full[s], (uint32_t)armed[s], p.err);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0 && !p.stall) {
      uint32_t stage = 0, phase = 0;
      int64_t it = 0;
      bool ok = true;
      const uint32_t id = idesc(BN);
      for (int64_t t = blockIdx.x; t < p.n_tiles && ok; t += gridDim.x) {
        int64_t bi, bj;
        if (!decode_tile<BN>(p, t, bi, bj)) continue;
        const uint32_t ab = (uint32_t)(it & 1);
        if (!mbar_wait(&acc_empty[ab], (uint32_t)((it >> 1) & 1) ^ 1u, abort_flag, p.err, p.timeout_ns)) break;
        tc_fence_after();
        const uint32_t d0 = tmem + ab * 256u;
        const uint32_t d1 = d0 + 128u;
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag, p.err, p.timeout_ns)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
          const uint32_t sb = sa + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < kRowBytes / 32; ++kk) {
            const uint32_t first = (kb == 0 && kk == 0) ? 0u : 1u;
            const uint64_t ad = sdesc(sa + kk * 32), bd = sdesc(sb + kk * 32);
            umma<FMT>(d0, ad, bd, id, first);
            if (C::NOPS == 2) {
              const uint32_t sa1 = sa + A_BYTES + B_BYTES, sb1 = sa + 2 * A_BYTES + B_BYTES;
              umma<FMT>(d1, ad, sdesc(sb1 + kk * 32), id, first);
              umma<FMT>(d1, sdesc(sa1 + kk * 32), bd, id, 1u);
            }
          }
          umma_commit(&empty[stage]);
          if (++stage == C::STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        umma_commit(&acc_full[ab]);
        ++it;
      }
      // wait for every MMA issued so far before TMEM can be released
      umma_commit(drain);
      mbar_drain(drain, 0, p.err);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    int64_t it = 0;
    for (int64_t t = blockIdx.x; t < p.n_tiles; t += gridDim.x) {
      int64_t bi, bj;
      if (!decode_tile<BN>(p, t, bi, bj)) continue;
      const uint32_t ab = (uint32_t)(it & 1);
      int ok = 1;
      if (lane == 0) ok = mbar_wait(&acc_full[ab], (uint32_t)((it >> 1) & 1), abort_flag, p.err, p.timeout_ns) ? 1 : 0;
      ok = __shfl_sync(kFull, ok, 0);
      if (!ok) break;
      tc_fence_after();
      const int64_t i = bi * kBM + q * 32 + lane;
      const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + ab * 256u;
      // E4M3: the score is the cosine of the quantized vectors, acc * out_scale / (|q_i| |q_j|).
      // Every non-zero quantized unit row has norm >= 1 - 2^-4 > kNormLo, so raw accumulators
      // below thresh * |q_i| * kNormLo / out_scale cannot reach the threshold (fast path).
      float row_norm = 1.f, fast_thresh = p.thresh, hit_lim = p.thresh;
      if (FMT == OP_E4M3) {
        row_norm = i < p.na ? p.a_norm[i] : 0.f;
        hit_lim = p.thresh * row_norm / p.out_scale;
        if (p.thresh > 0.f)
          fast_thresh = row_norm > 0.f ? p.thresh * row_norm * kNormLo / p.out_scale : __int_as_float(0x7f800000);
        else
          fast_thresh = -__int_as_float(0x7f800000);
      }
#pragma unroll 1
      for (int c = 0; c < BN / 32; ++c) {
        float v[32];
        float m;  // the chunk's row maximum (thresholding)
        if (C::ACCS == 2) {
          tmem_ld32(trow + c * 32, v);
          float x[32];
          tmem_ld32(trow + 128 + c * 32, x);
          tmem_wait_ld();
#pragma unroll
          for (int e = 0; e < 32; ++e) v[e] = fmaf(x[e], 1.0f / kSplitLoScale, v[e]);
          m = max32(v);
        } else {
          tmem_ld32_max(trow + c * 32, v, m);
          tmem_wait_ld();
        }
        const int64_t j0 = bj * BN + c * 32;
        if (p.store16) {
          if (i < p.na) {
            __half* dst = p.store16 + i * p.ld + j0;
            if (j0 + 32 <= p.nb && (p.ld & 7) == 0) {
#pragma unroll
              for (int e = 0; e < 32; e += 8) {
                uint4 w;
                __half2 h0 = __floats2half2_rn(v[e], v[e + 1]), h1 = __floats2half2_rn(v[e + 2], v[e + 3]);
                __half2 h2 = __floats2half2_rn(v[e + 4], v[e + 5]), h3 = __floats2half2_rn(v[e + 6], v[e + 7]);
                w.x = *reinterpret_cast<uint32_t*>(&h0);
                w.y = *reinterpret_cast<uint32_t*>(&h1);
                w.z = *reinterpret_cast<uint32_t*>(&h2);
                w.w = *reinterpret_cast<uint32_t*>(&h3);
                *reinterpret_cast<uint4*>(dst + e) = w;
              }
            } else {
#pragma unroll
              for (int e = 0; e < 32; ++e)
                if (j0 + e < p.nb) dst[e] = __float2half_rn(v[e]);
            }
          }
        } else if (p.store) {
          if (i < p.na) {
            float* dst = p.store + i * p.ld + j0;
            if (j0 + 32 <= p.nb && (p.ld & 3) == 0) {
#pragma unroll
              for (int e = 0; e < 32; e += 4)
                *reinterpret_cast<float4*>(dst + e) = make_float4(v[e], v[e + 1], v[e + 2], v[e + 3]);
            } else {
#pragma unroll
              for (int e = 0; e < 32; ++e)
                if (j0 + e < p.nb) dst[e] = v[e];
            }
          }
        } else {
          emit_chunk<FMT>(p, v, m, i, j0, lane, fast_thresh, row_norm, hit_lim, stage, pbuf, pfill);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[ab]);
      ++it;
    }
    flush_pairs(p, pbuf, pfill, lane);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// Resident kernel: the CTA's tiles are an even share of the order (contiguous mode) or whole
// row blocks dealt round-robin (see TileSeq).
template <int FMT, int RB, int BN>
__global__ void __launch_bounds__(kResThreads, 1)
    k_gemm_resident(const __grid_constant__ CUtensorMap tA0, const __grid_constant__ CUtensorMap tA1,
                    const __grid_constant__ CUtensorMap tB0, const __grid_constant__ CUtensorMap tB1, GemmParams p) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ uint32_t tmem_slot;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int warp = threadIdx.x >> 5;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int64_t t_begin = p.n_tiles * blockIdx.x / gridDim.x;
  const int64_t t_end = p.n_tiles * (blockIdx.x + 1) / gridDim.x;
  resident_body<FMT, RB, BN>(&tA0, &tA1, &tB0, &tB1, p, smem, tmem, t_begin, t_end);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

template <int FMT, int RB, int BN>
cudaError_t run_gemm_resident(mrc_ctx* ctx, const GemmArgs& g) {
  using C = Cfg<FMT>;
  const bool fp8 = FMT == OP_E4M3;
  CUtensorMap tA0, tA1, tB0, tB1;
  if (!make_map(&tA0, g.a_hi, g.na, g.kbytes, kBM, fp8, RB) || !make_map(&tB0, g.b_hi, g.nb, g.kbytes, BN, fp8, RB))
    return cudaErrorInvalidValue;
  if (C::NOPS == 2) {
    if (!make_map(&tA1, g.a_lo, g.na, g.kbytes, kBM, fp8, RB) || !make_map(&tB1, g.b_lo, g.nb, g.kbytes, BN, fp8, RB))
      return cudaErrorInvalidValue;
  } else {
    tA1 = tA0;
    tB1 = tB0;
  }
  GemmParams p{};
  p.na = g.na;
  p.nb = g.nb;
  p.kblocks = 1;
  p.triangle = g.triangle;
  p.tiles_m = (g.na + kBM - 1) / kBM;
  p.tiles_n = (g.nb + BN - 1) / BN;
  p.super_rows = (g.na + BN - 1) / BN;
  p.n_tiles = g.triangle ? p.super_rows * (p.super_rows + 1) / 2 * (BN / kBM) : p.tiles_m * p.tiles_n;
  if (p.n_tiles >= (1ll << 31) || p.super_rows * p.super_rows >= (1ll << 31)) return cudaErrorInvalidValue;
  p.thresh = g.thresh;
  p.out_scale = g.out_scale;
  p.a_norm = g.a_norm;
  p.b_norm = g.b_norm;
  p.b_norm_min = g.b_norm_min;
  if (FMT == OP_E4M3 && (!g.a_norm || !g.b_norm || !g.b_norm_min)) return cudaErrorInvalidValue;
  p.pairs = g.pairs;
  p.count = g.count;
  p.capacity = g.capacity;
  p.err = g.err;
  p.timeout_ns = ctx->wait_limit_ns;
  p.exact = g.exact_scores;
  p.stall = ctx->test_stall ? 1 : 0;
  p.ring = g.ring;
  p.pf = g.prefetch >= 0 ? g.prefetch
                         : (!g.triangle && (int64_t)C::NOPS * g.nb * g.kbytes > kPrefetchMinBytes ? kPrefetchTiles : 0);
  // round-robin rows whenever there are at least two rounds of row blocks to balance: the CTAs
  // then share each streamed tile through L2 even when the operand would fit there (300,000
  // documents, 19 MB of E4M3 rows: 15.2 -> 11.5 ms)
  p.row_rr = g.triangle && p.tiles_m >= 2 * (int64_t)ctx->num_sms;
  constexpr size_t smem = resident_smem_bytes<FMT, RB, BN>();
  if (resident_ctas(k_gemm_resident<FMT, RB, BN>, kResThreads, smem) <= 0) return cudaErrorInvalidConfiguration;
  int64_t grid = ctx->num_sms;
  if (p.n_tiles < grid) grid = p.n_tiles;
  if (grid <= 0) return cudaSuccess;
  const double k_elems = (double)g.kbytes / (fp8 ? 1.0 : 2.0);
  const double pairs = g.triangle ? (double)g.na * (double)(g.na - 1) / 2.0 : (double)g.na * (double)g.nb;
  const double flops = 2.0 * k_elems * pairs * (C::NOPS == 2 ? 3.0 : 1.0);
  const char* name = FMT == OP_SPLIT16 ? "gemm_split16_thresh" : (FMT == OP_F16 ? "gemm_f16_thresh" : "gemm_e4m3_thresh");
  const double bytes = (double)C::NOPS * (double)(g.na + (g.triangle ? 0 : g.nb)) * g.kbytes;
  cudaEvent_t ev = nullptr;
  timing_begin(ctx, g.name ? g.name : name, bytes, flops, &ev);
  k_gemm_resident<FMT, RB, BN><<<(unsigned)grid, kResThreads, smem, ctx->stream>>>(tA0, tA1, tB0, tB1, p);
  timing_end(ctx, ev);
  return cudaGetLastError();
}

template <int FMT>
cudaError_t run_gemm(mrc_ctx* ctx, const GemmArgs& g) {
  using C = Cfg<FMT>;
  constexpr int BN = C::BN;
  const bool fp8 = FMT == OP_E4M3;
  CUtensorMap tA0, tA1, tB0, tB1;
  if (!make_map(&tA0, g.a_hi, g.na, g.kbytes, kBM, fp8) ||
      !make_map(&tB0, g.b_hi, g.nb, g.kbytes, BN, fp8))
    return cudaErrorInvalidValue;
  if (C::NOPS == 2) {
    if (!make_map(&tA1, g.a_lo, g.na, g.kbytes, kBM, fp8) || !make_map(&tB1, g.b_lo, g.nb, g.kbytes, BN, fp8))
      return cudaErrorInvalidValue;
  } else {
    tA1 = tA0;
    tB1 = tB0;
  }
  GemmParams p{};
  p.na = g.na;
  p.nb = g.nb;
  p.kblocks = g.kbytes / kRowBytes;
  p.triangle = g.triangle;
  p.tiles_m = (g.na + kBM - 1) / kBM;
  p.tiles_n = (g.nb + BN - 1) / BN;
  p.super_rows = (g.na + BN - 1) / BN;
  p.n_tiles = g.triangle ? p.super_rows * (p.super_rows + 1) / 2 * (BN / kBM) : p.tiles_m * p.tiles_n;
  if (p.n_tiles >= (1ll << 31) || p.super_rows * p.super_rows >= (1ll << 31)) return cudaErrorInvalidValue;
  p.thresh = g.thresh;
  p.out_scale = g.out_scale;
  p.a_norm = g.a_norm;
  p.b_norm = g.b_norm;
  if (FMT == OP_E4M3 && (!g.a_norm || !g.b_norm) && !g.store && !g.store16) return cudaErrorInvalidValue;
  p.pairs = g.pairs;
  p.count = g.count;
  p.capacity = g.capacity;
  p.store = g.store;
  p.store16 = reinterpret_cast<__half*>(g.store16);
  p.ld = g.ld;
  p.err = g.err;
  p.kblocks_dev = g.kblocks_dev;
  p.timeout_ns = ctx->wait_limit_ns;
  p.exact = g.exact_scores;
  p.stall = ctx->test_stall ? 1 : 0;
  const size_t smem =
      1024 + (size_t)C::STAGES * C::NOPS * (kBM + BN) * kRowBytes + 256 + 4 * (32 * 33 * 4 + kWarpPairBytes);
  if (resident_ctas(k_gemm_compare<FMT>, kThreads, smem) <= 0) return cudaErrorInvalidConfiguration;
  int64_t grid = ctx->num_sms;
  if (p.n_tiles < grid) grid = p.n_tiles;
  if (grid <= 0) return cudaSuccess;
  // algorithmic work: 2 K flops per evaluated pair (the triangle counts i < j only)
  const double k_elems = (double)g.kbytes / (fp8 ? 1.0 : 2.0);
  const double pairs = g.triangle ? (double)g.na * (double)(g.na - 1) / 2.0 : (double)g.na * (double)g.nb;
  const double flops = 2.0 * k_elems * pairs * (C::NOPS == 2 ? 3.0 : 1.0);
  const bool st = g.store || g.store16;
  const char* name = FMT == OP_SPLIT16 ? (st ? "gemm_split16_store" : "gemm_split16_thresh")
                                        : (FMT == OP_F16 ? (st ? "gemm_f16_store" : "gemm_f16_thresh")
                                                         : "gemm_e4m3_thresh");
  const double bytes = (double)C::NOPS * (double)(g.na + (g.triangle ? 0 : g.nb)) * g.kbytes;
  cudaEvent_t ev = nullptr;
  timing_begin(ctx, g.name ? g.name : name, bytes, flops, &ev);
  k_gemm_compare<FMT><<<(unsigned)grid, kThreads, smem, ctx->stream>>>(tA0, tA1, tB0, tB1, p);
  timing_end(ctx, ev);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_compare(mrc_ctx* ctx, const GemmArgs& g) {
  if (g.na <= 0 || g.nb <= 0) return cudaErrorInvalidValue;
  if (g.na >= (1ll << 31) || g.nb >= (1ll << 31)) return cudaErrorInvalidValue;
  if (!g.store && !g.store16 && (g.kbytes == 64 || g.kbytes == 128)) {
    // one K block: resident-A kernel
    // tile width: by default 256 columns for single-accumulator formats, except for a query x
    // index compare of at most two row blocks (four TMEM accumulators in flight stream the index
    // faster); 128 or 256 on request
    const bool few_rows = !g.triangle && g.na <= 2 * kBM;
    const int wide = (g.fmt != OP_SPLIT16 && (g.tile_n == 256 || (g.tile_n == 0 && !few_rows))) ? 1 : 0;
    switch ((g.fmt * 2 + (g.kbytes == 128 ? 1 : 0)) * 2 + wide) {
      case (OP_SPLIT16 * 2) * 2: return run_gemm_resident<OP_SPLIT16, 64, 128>(ctx, g);
      case (OP_SPLIT16 * 2 + 1) * 2: return run_gemm_resident<OP_SPLIT16, 128, 128>(ctx, g);
      case (OP_F16 * 2) * 2: return run_gemm_resident<OP_F16, 64, 128>(ctx, g);
      case (OP_F16 * 2) * 2 + 1: return run_gemm_resident<OP_F16, 64, 256>(ctx, g);
      case (OP_F16 * 2 + 1) * 2: return run_gemm_resident<OP_F16, 128, 128>(ctx, g);
      case (OP_F16 * 2 + 1) * 2 + 1: return run_gemm_resident<OP_F16, 128, 256>(ctx, g);
      case (OP_E4M3 * 2) * 2: return run_gemm_resident<OP_E4M3, 64, 128>(ctx, g);
      case (OP_E4M3 * 2) * 2 + 1: return run_gemm_resident<OP_E4M3, 64, 256>(ctx, g);
      case (OP_E4M3 * 2 + 1) * 2: return run_gemm_resident<OP_E4M3, 128, 128>(ctx, g);
      case (OP_E4M3 * 2 + 1) * 2 + 1: return run_gemm_resident<OP_E4M3, 128, 256>(ctx, g);
      default: return cudaErrorInvalidValue;
    }
  }
  if (g.kbytes <= 0 || g.kbytes % kRowBytes != 0) return cudaErrorInvalidValue;
  switch (g.fmt) {
    case OP_SPLIT16:
      return run_gemm<OP_SPLIT16>(ctx, g);
    case OP_F16:
      return run_gemm<OP_F16>(ctx, g);
    case OP_E4M3:
      return run_gemm<OP_E4M3>(ctx, g);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace mrc
