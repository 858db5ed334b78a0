// simhash_index.cu -- block-table Hamming search over 64-bit Simhash fingerprints.
//
// Section I cites the use of Simhash at web scale, where new pages are compared with a large
// database of fingerprints. Comparing a query with every fingerprint (simhash_match.cu) costs
// n POPCs per query; this index finds the same pairs from a few buckets.
//
// The 64 bits are cut into b >= h + 1 blocks (h = the largest Hamming distance searched). Two
// fingerprints within distance h differ in at most h bits, so at least one block is equal in
// both (pigeonhole). Table t holds every fingerprint grouped by the value of block t (a
// counting sort: bucket offsets over the 2^width values, then the entries); a query reads, in
// each table, the bucket of its own block value and tests the popcount of the XOR. A pair is
// emitted only by the table of the first block on which the two fingerprints agree, so each
// pair comes out once. With b = 4 blocks of 16 bits and random fingerprints a bucket holds
// n / 65,536 entries: a query reads 4 n / 65,536 candidates instead of n.
#include "device.cuh"
#include "internal.h"

namespace mrc {
namespace {

__device__ __forceinline__ uint32_t block_key(uint64_t f, int shift, int width) {
  return (uint32_t)((f >> shift) & ((1ull << width) - 1ull));
}

__global__ void k_sh_hist(const uint64_t* __restrict__ fps, int64_t n, SimhashLayout L, int32_t* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t f = fps[i];
  for (int t = 0; t < L.blocks; ++t) atomicAdd(cnt + L.off_base[t] + block_key(f, L.shift[t], L.width[t]), 1);
}

// One CTA per table: off[v] = entries of table t with block value < v (exclusive scan of the
// 2^width counts); off[2^width] = n. cursor gets a copy of the starts.
__global__ void __launch_bounds__(1024) k_sh_scan(const int32_t* __restrict__ cnt, SimhashLayout L, int32_t* off,
                                                  int32_t* cursor) {
  __shared__ int32_t warp_sum[32];
  const int t = blockIdx.x;
  const int32_t bins = 1 << L.width[t];
  const int32_t per = (bins + 1023) / 1024;
  const int32_t b0 = min((int32_t)threadIdx.x * per, bins), b1 = min(b0 + per, bins);
  const int32_t* c = cnt + L.off_base[t];
  int32_t s = 0;
  for (int32_t v = b0; v < b1; ++v) s += c[v];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  int32_t run = incl - s;
  for (int w = 0; w < warp; ++w) run += warp_sum[w];
  int32_t* o = off + L.off_base[t];
  int32_t* cu = cursor + L.off_base[t];
  for (int32_t v = b0; v < b1; ++v) {
    o[v] = run;
    cu[v] = run;
    run += c[v];
  }
  if (threadIdx.x == 1023) o[bins] = run;
}

__global__ void k_sh_scatter(const uint64_t* __restrict__ fps, int64_t n, SimhashLayout L, int32_t* cursor,
                             uint64_t* __restrict__ fp_out, int32_t* __restrict__ id_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t f = fps[i];
  for (int t = 0; t < L.blocks; ++t) {
    const int32_t at = atomicAdd(cursor + L.off_base[t] + block_key(f, L.shift[t], L.width[t]), 1);
    fp_out[(int64_t)t * n + at] = f;
    id_out[(int64_t)t * n + at] = (int32_t)i;
  }
}

// One warp per (query, table): the query's bucket in table t, 32 candidates per step.
// all_pairs: the queries are the index's own fingerprints and only ids > q are emitted.
__global__ void __launch_bounds__(256) k_sh_probe(const uint64_t* __restrict__ q, int64_t nq, int all_pairs,
                                                  int32_t hmax, SimhashLayout L, int64_t n,
                                                  const uint64_t* __restrict__ fp, const int32_t* __restrict__ id,
                                                  const int32_t* __restrict__ off, mrc_pair* pairs,
                                                  unsigned long long* count, int64_t capacity) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t qi = gw / L.blocks;
  const int t = (int)(gw - qi * L.blocks);
  if (qi >= nq) return;  // warp-uniform
  const uint64_t fq = __ldg(q + qi);
  const int32_t* o = off + L.off_base[t];
  const uint32_t key = block_key(fq, L.shift[t], L.width[t]);
  const int32_t s = __ldg(o + key), e = __ldg(o + key + 1);
  const uint64_t* tf = fp + (int64_t)t * n;
  const int32_t* ti = id + (int64_t)t * n;
  // two candidate loads in flight per lane: the second step's load is issued with the first
  uint64_t nxt = s + lane < e ? __ldg(tf + s + lane) : 0ull;
  for (int32_t x0 = s; x0 < e; x0 += 32) {
    const int32_t x = x0 + lane;
    const uint64_t cur = nxt;
    if (x0 + 32 < e) nxt = x + 32 < e ? __ldg(tf + x + 32) : 0ull;  // warp-uniform branch
    bool ok = false;
    int32_t j = 0, d = 0;
    if (x < e) {
      const uint64_t m = cur ^ fq;
      d = __popcll(m);
      ok = d <= hmax;
      if (ok) {
        j = __ldg(ti + x);
        if (all_pairs) ok = j > qi;
        for (int u = 0; u < t && ok; ++u) ok = block_key(m, L.shift[u], L.width[u]) != 0u;  // first equal block
      }
    }
    const unsigned hit = __ballot_sync(kFull, ok);
    if (hit == 0u) continue;
    unsigned long long base = 0ull;
    if (lane == __ffs(hit) - 1) base = atomicAdd(count, (unsigned long long)__popc(hit));
    base = __shfl_sync(kFull, base, __ffs(hit) - 1);
    if (ok) {
      const unsigned long long at = base + __popc(hit & ((1u << lane) - 1u));
      if (at < (unsigned long long)capacity) {
        mrc_pair pr;
        pr.i = (int32_t)qi;
        pr.j = j;
        pr.score = (float)d;
        pairs[at] = pr;
      }
    }
  }
}

}  // namespace

SimhashLayout simhash_layout(int32_t hamming_max) {
  SimhashLayout L{};
  L.blocks = std::max(hamming_max + 1, 4);
  int64_t shift = 0, base = 0;
  for (int t = 0; t < L.blocks; ++t) {
    L.width[t] = 64 / L.blocks + (t < 64 % L.blocks ? 1 : 0);
    L.shift[t] = (int32_t)shift;
    L.off_base[t] = base;
    shift += L.width[t];
    base += (1ll << L.width[t]) + 1;
  }
  L.off_words = base;
  return L;
}

cudaError_t launch_simhash_index_build(mrc_ctx* ctx, const uint64_t* fps, int64_t n, const SimhashLayout& L,
                                       int32_t* cnt, int32_t* cursor, int32_t* off, uint64_t* fp_out,
                                       int32_t* id_out) {
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)L.off_words, ctx->stream);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (n > 0) {
    KernelTimer kt(ctx, "simhash_index_hist", 8.0 * (double)n);
    k_sh_hist<<<grid, 256, 0, ctx->stream>>>(fps, n, L, cnt);
  }
  {
    KernelTimer kt(ctx, "simhash_index_scan", 12.0 * (double)L.off_words);
    k_sh_scan<<<L.blocks, 1024, 0, ctx->stream>>>(cnt, L, off, cursor);
  }
  if (n > 0) {
    KernelTimer kt(ctx, "simhash_index_scatter", 8.0 * (double)n + 12.0 * (double)n * L.blocks);
    k_sh_scatter<<<grid, 256, 0, ctx->stream>>>(fps, n, L, cursor, fp_out, id_out);
  }
  return cudaGetLastError();
}

cudaError_t launch_simhash_index_probe(mrc_ctx* ctx, const uint64_t* q, int64_t nq, bool all_pairs, int32_t hmax,
                                       const SimhashLayout& L, int64_t n, const uint64_t* fp, const int32_t* id,
                                       const int32_t* off, mrc_pair* pairs, unsigned long long* count,
                                       int64_t capacity) {
  if (nq <= 0 || n <= 0) return cudaSuccess;
  const int64_t warps = nq * L.blocks;
  KernelTimer kt(ctx, "simhash_index_probe", 8.0 * (double)nq);
  k_sh_probe<<<(unsigned)((warps + 7) / 8), 256, 0, ctx->stream>>>(q, nq, all_pairs ? 1 : 0, hmax, L, n, fp, id,
                                                                    off, pairs, count, capacity);
  return cudaGetLastError();
}

}  // namespace mrc
