// batch.cu -- graph-captured query batches against a resident signature index.
//
// A batch pipeline compares new documents with every document of an index, the way
// the method is meant to be served (each new page is signatured and compared with
// the signature database, Section I / Section IV):
//   signature pass (bag of terms, TF-IDF, cosine to each reference partition; unit
//   signature and compare operands written directly) -> tensor-core compare of the
//   batch against the whole index at a lowered threshold -> FP32 rescoring -> pairs grouped
//   by query; with a fingerprint index attached, the batch's Simhashes then probe it
//   (Hamming pairs, grouped by query as well).
// For compare rows of 64 or 128 bytes (k <= 64) the whole pipeline is one persistent
// cooperative kernel (batch_kernel.cu), captured with the memset of its control block into a
// CUDA graph on the batch's own stream; the kernel reads the number of documents of each
// launch from the device, so documents past it cost nothing but an empty signature row.
// Wider rows take the same steps as separate kernels in the graph, the batch then padded with
// empty documents (zero signatures, which match nothing). Each batch is one graph launch,
// after the copies of its offsets, tokens and document count.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"

using namespace mrc;

struct mrc_batch {
  mrc_ctx* ctx = nullptr;  // private context: its own stream and workspace
  const mrc_index* index = nullptr;
  int64_t max_docs = 0, max_tokens = 0, capacity = 0, cand_cap = 0;
  float tau = 0.f;
  int32_t tile_n = 0;
  int64_t* d_offsets = nullptr;
  int32_t* d_tokens = nullptr;
  float* d_unit = nullptr;
  void* d_op = nullptr;
  float* d_qnorm = nullptr;
  mrc_pair* d_cand = nullptr;
  mrc_pair* d_pairs = nullptr;
  mrc_pair* d_grouped = nullptr;           // pairs grouped by query
  int64_t* d_qoff = nullptr;               // [max_docs + 1] start of each query's pairs
  int32_t* d_qcnt = nullptr;               // [max_docs] pairs per query
  int32_t* d_qfill = nullptr;              // [max_docs] scatter cursors
  // control block (one allocation, zeroed before each launch): pair and candidate counts,
  // the Hamming pair count, the error word and the batch kernel's control words; then the
  // launch's document count (not zeroed)
  void* d_block = nullptr;
  unsigned long long* d_counts = nullptr;  // [0] pairs, [1] candidates
  unsigned long long* d_hcount = nullptr;
  int32_t* d_err = nullptr;
  int32_t* d_ctl = nullptr;
  int64_t* d_nlive = nullptr;
  int32_t* d_long = nullptr;               // [max_docs] the batch kernel's long-document list
  unsigned long long* d_stamps = nullptr;  // [kBatchStamps] phase timestamps of the batch kernel
  bool fused = false;                      // one persistent kernel (else separate kernels)
  int32_t qstride = 1;                     // per-query counter stride (words)
  int32_t ring = 0, prefetch = -1;         // compare tuning (B ring depth, L2 prefetch distance)
  unsigned long long* h_counts = nullptr;  // pinned: [0] pairs [1] candidates [2] error word [3] Hamming pairs
                                           // [4] the launch's document count (staging)
  uint64_t* d_simhash = nullptr;           // [max_docs] the batch's Simhash fingerprints
  // Hamming leg (mrc_batch_attach_simhash): the batch's fingerprints probe a block-table index
  const mrc_simhash_index* shx = nullptr;
  int32_t hmax = 0;
  int64_t h_capacity = 0;
  mrc_pair* d_hpairs = nullptr;
  mrc_pair* d_hgrouped = nullptr;
  int64_t* d_hqoff = nullptr;
  int32_t* d_hqcnt = nullptr;
  int32_t* d_hqfill = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t kernel_nodes = 0;  // kernel nodes of the captured graph
  cudaEvent_t done = nullptr;
  bool pending = false;
  bool has_result = false;  // the last launch finished; its results can be copied out (again)
  int64_t last_n = 0;  // documents of the last launch
};

namespace {

constexpr float kF16Bound = 2e-3f;  // > max |fp16 cosine - cosine| of unit vectors
constexpr size_t kBlockZeroBytes = 64;  // counts (16), Hamming count (8), error word (8), control words (32)
static_assert(kBlockZeroBytes == 32 + 8 * sizeof(int32_t) && kBatchCtlWords == 8, "control block layout");

// Groups the batch's pairs by query: per-query counts, exclusive scan (one CTA), scatter.
__global__ void k_group_count(const mrc_pair* pairs, const unsigned long long* n_pairs, int64_t cap, int32_t* cnt) {
  const int64_t n = min((int64_t)*n_pairs, cap);
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[pairs[x].i], 1);
}

__global__ void k_group_scan(const int32_t* cnt, int64_t n_q, int64_t* qoff, int32_t* fill) {
  __shared__ int64_t part[1024];
  const int64_t per = (n_q + blockDim.x - 1) / blockDim.x;
  const int64_t a = threadIdx.x * per, b = min(n_q, a + per);
  int64_t s = 0;
  for (int64_t q = a; q < b; ++q) s += cnt[q];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (unsigned t = 0; t < blockDim.x; ++t) {
      const int64_t v = part[t];
      part[t] = run;
      run += v;
    }
    qoff[n_q] = run;
  }
  __syncthreads();
  int64_t run = part[threadIdx.x];
  for (int64_t q = a; q < b; ++q) {
    qoff[q] = run;
    fill[q] = 0;
    run += cnt[q];
  }
}

__global__ void k_group_scatter(const mrc_pair* pairs, const unsigned long long* n_pairs, int64_t cap,
                                const int64_t* qoff, int32_t* fill, mrc_pair* out) {
  const int64_t n = min((int64_t)*n_pairs, cap);
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (int64_t)gridDim.x * blockDim.x) {
    const mrc_pair pr = pairs[x];
    out[qoff[pr.i] + atomicAdd(&fill[pr.i], 1)] = pr;
  }
}

__global__ void k_pad_offsets(int64_t* off, int64_t n, int64_t max_docs) {
  const int64_t i = n + 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= max_docs) off[i] = off[n];
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The persistent kernel's launch (captured into the graph).
cudaError_t record_fused(mrc_batch* b) {
  mrc_ctx* ctx = b->ctx;
  const mrc_index* x = b->index;
  const int32_t prec = x->params.precision;
  cudaError_t e = cudaMemsetAsync(b->d_block, 0, kBlockZeroBytes, ctx->stream);
  if (e != cudaSuccess) return e;
  BatchKernelArgs a{};
  a.index = x;
  a.max_docs = b->max_docs;
  a.max_tokens = b->max_tokens;
  a.offsets = b->d_offsets;
  a.tokens = b->d_tokens;
  a.n_live = b->d_nlive;
  a.unit = b->d_unit;
  a.op = b->d_op;
  a.qnorm = b->d_qnorm;
  a.simhash = b->d_simhash;
  a.tau = b->tau;
  a.thresh = b->tau - (prec == MRC_PREC_BF16_FP8 ? x->params.margin : kF16Bound);
  a.tile_n = b->tile_n;
  a.ring = b->ring;
  a.prefetch = b->prefetch;
  a.cand = b->d_cand;
  a.cand_cap = b->cand_cap;
  a.pairs = b->d_pairs;
  a.capacity = b->capacity;
  a.counts = b->d_counts;
  a.err = b->d_err;
  a.ctl = b->d_ctl;
  a.long_list = b->d_long;
  a.qstride = b->qstride;
  a.qcnt = b->d_qcnt;
  a.qfill = b->d_qfill;
  a.qoff = b->d_qoff;
  a.grouped = b->d_grouped;
  a.stamps = b->d_stamps;
  if (b->shx) {
    a.shx = b->shx;
    a.hmax = b->hmax;
    a.hpairs = b->d_hpairs;
    a.hcount = b->d_hcount;
    a.hcapacity = b->h_capacity;
    a.hqcnt = b->d_hqcnt;
    a.hqfill = b->d_hqfill;
    a.hqoff = b->d_hqoff;
    a.hgrouped = b->d_hgrouped;
  }
  return launch_batch_kernel(ctx, a);
}

// The stream-ordered work of one batch as separate kernels (captured into the graph).
cudaError_t record(mrc_batch* b) {
  if (b->fused) return record_fused(b);
  mrc_ctx* ctx = b->ctx;
  const mrc_index* x = b->index;
  const int32_t prec = x->params.precision;
  cudaError_t e = cudaMemsetAsync(b->d_counts, 0, 2 * sizeof(unsigned long long), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int32_t), ctx->stream);
  if (e != cudaSuccess) return e;
  DocsDev d{};
  d.n_docs = b->max_docs;
  d.offsets = b->d_offsets;
  d.tokens = b->d_tokens;
  d.n_tokens = b->max_tokens;
  d.err = b->d_err;
  SigOut o{};
  o.sig_unit = b->d_unit;
  o.simhash = b->d_simhash;
  if (prec == MRC_PREC_BF16_FP8) {
    o.op_e4m3 = b->d_op;
    o.qnorm = b->d_qnorm;
    o.kp8 = x->kp8;
  } else {
    o.op_hi = b->d_op;
    o.kp = x->kp;
  }
  // query operands from FP32 weights, as mrc_match packs the signatures of mrc_signature
  e = launch_signature(ctx, d, x->vocab, x->tinfo, x->rinv, nullptr, x->k, x->params.seed, x->fhash, o);
  if (e != cudaSuccess) return e;
  GemmArgs g{};
  g.na = b->max_docs;
  g.nb = x->n_docs;
  g.triangle = 0;
  g.err = b->d_err;
  g.out_scale = 1.0f;
  g.tile_n = b->tile_n;
  g.fmt = prec == MRC_PREC_BF16_FP8 ? OP_E4M3 : OP_F16;
  g.a_hi = b->d_op;
  g.b_hi = prec == MRC_PREC_BF16_FP8 ? x->op_e4m3 : x->op_hi;
  g.kbytes = prec == MRC_PREC_BF16_FP8 ? x->kp8 : x->kp * 2;
  if (prec == MRC_PREC_BF16_FP8) {
    g.out_scale = 1.0f / (kE4M3Scale * kE4M3Scale);
    g.a_norm = b->d_qnorm;
    g.b_norm = x->qnorm;
    g.b_norm_min = x->qnorm_min;
  }
  g.thresh = b->tau - (prec == MRC_PREC_BF16_FP8 ? x->params.margin : kF16Bound);
  g.pairs = b->d_cand;
  g.count = b->d_counts + 1;
  g.capacity = b->cand_cap;
  g.ring = b->ring;
  g.prefetch = b->prefetch;
  e = launch_gemm_compare(ctx, g);
  if (e != cudaSuccess) return e;
  e = launch_rescore(ctx, b->d_cand, b->d_counts + 1, b->cand_cap, b->d_unit, x->sig_unit, x->k, b->tau,
                     b->d_pairs, b->d_counts, b->capacity, b->d_err);
  if (e != cudaSuccess) return e;
  // group the pairs by query, so each query's pairs come back as one slice
  e = cudaMemsetAsync(b->d_qcnt, 0, sizeof(int32_t) * (size_t)b->max_docs, ctx->stream);
  if (e != cudaSuccess) return e;
  const int grid = ctx->num_sms * 4;
  k_group_count<<<grid, 256, 0, ctx->stream>>>(b->d_pairs, b->d_counts, b->capacity, b->d_qcnt);
  k_group_scan<<<1, 1024, 0, ctx->stream>>>(b->d_qcnt, b->max_docs, b->d_qoff, b->d_qfill);
  k_group_scatter<<<grid, 256, 0, ctx->stream>>>(b->d_pairs, b->d_counts, b->capacity, b->d_qoff, b->d_qfill,
                                                 b->d_grouped);
  if (b->shx) {
    // Hamming leg: the batch's fingerprints (padding documents included: they are empty, and
    // their pairs fall after the real queries' once grouped) against the block-table index
    const mrc_simhash_index* h = b->shx;
    e = cudaMemsetAsync(b->d_hcount, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_hqcnt, 0, sizeof(int32_t) * (size_t)b->max_docs, ctx->stream);
    if (e != cudaSuccess) return e;
    e = launch_simhash_index_probe(ctx, b->d_simhash, b->max_docs, false, b->hmax, h->layout, h->n, h->fp, h->id,
                                   h->off, b->d_hpairs, b->d_hcount, b->h_capacity);
    if (e != cudaSuccess) return e;
    k_group_count<<<grid, 256, 0, ctx->stream>>>(b->d_hpairs, b->d_hcount, b->h_capacity, b->d_hqcnt);
    k_group_scan<<<1, 1024, 0, ctx->stream>>>(b->d_hqcnt, b->max_docs, b->d_hqoff, b->d_hqfill);
    k_group_scatter<<<grid, 256, 0, ctx->stream>>>(b->d_hpairs, b->d_hcount, b->h_capacity, b->d_hqoff,
                                                   b->d_hqfill, b->d_hgrouped);
  }
  return cudaGetLastError();
}

// Runs the pipeline once uncaptured (sizing every workspace buffer), then captures it into
// the batch's graph (replacing an earlier one).
cudaError_t capture(mrc_batch* b) {
  cudaStream_t s = b->ctx->stream;
  cudaError_t e = record(b);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaGraph_t graph = nullptr;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    const cudaError_t er = record(b);
    e = cudaStreamEndCapture(s, &graph);
    if (er != cudaSuccess) e = er;
  }
  cudaGraphExec_t exec = nullptr;
  int32_t kernels = 0;
  if (e == cudaSuccess) {
    size_t nn = 0;
    e = cudaGraphGetNodes(graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(graph, nodes.data(), &nn);
    for (size_t i = 0; e == cudaSuccess && i < nn; ++i) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[i], &t);
      if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) return e;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = exec;
  b->kernel_nodes = kernels;
  return cudaSuccess;
}

void release(mrc_batch* b) {
  if (!b) return;
  if (b->ctx) cudaStreamSynchronize(b->ctx->stream);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->done) cudaEventDestroy(b->done);
  void* ptrs[] = {b->d_offsets, b->d_tokens,    b->d_unit,  b->d_op,    b->d_qnorm,  b->d_cand,
                  b->d_pairs,   b->d_grouped,   b->d_qoff,  b->d_qcnt,  b->d_qfill,  b->d_block,
                  b->d_long,    b->d_simhash,   b->d_hpairs, b->d_hgrouped, b->d_hqoff, b->d_hqcnt,
                  b->d_hqfill,  b->d_stamps};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->h_counts) cudaFreeHost(b->h_counts);
  if (b->ctx) {
    cudaStream_t s = b->ctx->stream;
    mrc_ctx_destroy(b->ctx);
    cudaStreamDestroy(s);
  }
  delete b;
}

// Waits for the last launch (once) and checks its error word; the results stay available until
// the next launch.
mrc_status finish_launch(mrc_batch* b) {
  mrc_ctx* ctx = b->ctx;
  if (b->pending) {
    const cudaError_t e = cudaEventSynchronize(b->done);
    b->pending = false;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "mrc_batch_wait");
    b->has_result = true;
  }
  if (!b->has_result) return fail(ctx, MRC_ERR_INVALID, "mrc_batch_wait: nothing launched");
  int32_t err = 0;
  std::memcpy(&err, b->h_counts + 2, sizeof(int32_t));
  if (err & kErrTimeout) return fail(ctx, MRC_ERR_TIMEOUT, "a bounded device wait expired");
  if (err & kErrBadToken) return fail(ctx, MRC_ERR_INVALID, "a token id is outside [0, vocab)");
  if (err & kErrBadOffsets) return fail(ctx, MRC_ERR_INVALID, "offsets must start at 0 and be non-decreasing");
  if (err & kErrTooLong) return fail(ctx, MRC_ERR_UNSUPPORTED, "a document is longer than MRC_MAX_DOC_TOKENS tokens");
  return MRC_OK;
}

// Copies a finished launch's grouped pairs (min(total, own capacity, capacity) of them) and
// its query offsets out, on the batch's stream.
mrc_status copy_out(mrc_batch* b, const mrc_pair* d_pairs, int64_t total, int64_t own_cap, const int64_t* d_off,
                    mrc_pair* pairs, int64_t capacity, int64_t* query_offsets, const char* what) {
  mrc_ctx* ctx = b->ctx;
  const int64_t m = std::min<int64_t>(std::min<int64_t>(total, own_cap), capacity);
  cudaError_t e = cudaSuccess;
  if (m > 0 && pairs)
    e = cudaMemcpyAsync(pairs, d_pairs, sizeof(mrc_pair) * (size_t)m, cudaMemcpyDefault, ctx->stream);
  if (e == cudaSuccess && query_offsets)
    e = cudaMemcpyAsync(query_offsets, d_off, sizeof(int64_t) * (size_t)(b->last_n + 1), cudaMemcpyDefault,
                        ctx->stream);
  if (e == cudaSuccess && ((m > 0 && pairs) || query_offsets)) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, what);
  if (pairs && total > std::min(capacity, own_cap))
    return fail(ctx, MRC_ERR_CAPACITY, "more pairs than capacity; *n_pairs holds the total");
  if (!pairs && total > own_cap) return fail(ctx, MRC_ERR_CAPACITY, "more pairs than the batch's capacity");
  return MRC_OK;
}

}  // namespace

extern "C" {

mrc_status mrc_batch_create(mrc_ctx* ctx, const mrc_index* index, int64_t max_docs, int64_t max_tokens, float tau,
                            int64_t capacity, int32_t tile_n, mrc_batch** out) {
  TraceRange trace(__func__);
  if (!ctx || !index || !out) return MRC_ERR_INVALID;
  *out = nullptr;
  if (max_docs < 1 || max_docs > (1 << 24) || max_tokens < 1 || capacity < 1)
    return fail(ctx, MRC_ERR_INVALID, "mrc_batch_create: max_docs in [1, 2^24], max_tokens and capacity >= 1");
  if (tile_n != 0 && tile_n != 128 && tile_n != 256)
    return fail(ctx, MRC_ERR_INVALID, "mrc_batch_create: tile_n must be 0, 128 or 256");
  cudaSetDevice(ctx->device);
  // the batch runs on a stream of its own: the index must be complete first
  wait_for_index(ctx, index);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "waiting for the index");
  mrc_batch* b = new mrc_batch();
  b->index = index;
  b->max_docs = max_docs;
  b->max_tokens = max_tokens;
  b->capacity = capacity;
  b->cand_cap = std::max<int64_t>(4 * capacity, 1 << 16);
  b->tau = tau;
  b->tile_n = tile_n;
  b->fused = batch_kernel_supported(index);
  // per-query counters in separate 128-byte lines (atomics on different L2 lines) while that
  // costs at most 8 MB
  b->qstride = b->fused && max_docs <= 65536 ? 32 : 1;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return cuda_fail(ctx, cudaGetLastError(), "creating the batch stream");
  }
  mrc_ctx* bc = nullptr;
  if (mrc_ctx_create(s, &bc) != MRC_OK) {
    cudaStreamDestroy(s);
    delete b;
    return fail(ctx, MRC_ERR_CUDA, "creating the batch context");
  }
  b->ctx = bc;
  const int32_t prec = index->params.precision;
  const size_t op_bytes = prec == MRC_PREC_BF16_FP8 ? (size_t)max_docs * index->kp8 : 2 * (size_t)max_docs * index->kp;
  cudaError_t e = cudaMalloc(&b->d_offsets, sizeof(int64_t) * (size_t)(max_docs + 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tokens, sizeof(int32_t) * (size_t)max_tokens);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_unit, sizeof(float) * (size_t)max_docs * index->k);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_op, op_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_qnorm, sizeof(float) * (size_t)max_docs);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_cand, sizeof(mrc_pair) * (size_t)b->cand_cap);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_pairs, sizeof(mrc_pair) * (size_t)capacity);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_grouped, sizeof(mrc_pair) * (size_t)capacity);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_qoff, sizeof(int64_t) * (size_t)(max_docs + 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_qcnt, sizeof(int32_t) * (size_t)max_docs * b->qstride);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_qfill, sizeof(int32_t) * (size_t)max_docs * b->qstride);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_block, kBlockZeroBytes + sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_long, sizeof(int32_t) * (size_t)max_docs);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_stamps, sizeof(unsigned long long) * kBatchStamps);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_stamps, 0, sizeof(unsigned long long) * kBatchStamps, s);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_simhash, sizeof(uint64_t) * (size_t)max_docs);
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_counts, 5 * sizeof(unsigned long long));
  if (e == cudaSuccess) {
    b->d_counts = reinterpret_cast<unsigned long long*>(b->d_block);
    b->d_hcount = b->d_counts + 2;
    b->d_err = reinterpret_cast<int32_t*>(b->d_counts + 3);
    b->d_ctl = b->d_err + 2;
    b->d_nlive = reinterpret_cast<int64_t*>(reinterpret_cast<uint8_t*>(b->d_block) + kBlockZeroBytes);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_offsets, 0, sizeof(int64_t) * (size_t)(max_docs + 1), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_block, 0, kBlockZeroBytes + sizeof(int64_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_op, 0, op_bytes, s);
  if (e != cudaSuccess) {
    mrc_status st = cuda_fail(ctx, e, "mrc_batch_create allocations");
    release(b);
    return st;
  }
  // one uncaptured run sizes every workspace buffer; then the same work is captured
  e = capture(b);
  if (e != cudaSuccess) {
    mrc_status st = cuda_fail(ctx, e, "capturing the batch pipeline");
    release(b);
    return st;
  }
  *out = b;
  return MRC_OK;
}

mrc_status mrc_batch_launch(mrc_batch* b, const mrc_docs* docs) {
  TraceRange trace(__func__);
  if (!b || !docs) return MRC_ERR_INVALID;
  mrc_ctx* ctx = b->ctx;
  cudaSetDevice(ctx->device);
  if (b->pending) return fail(ctx, MRC_ERR_INVALID, "mrc_batch_launch: the previous launch was not waited for");
  const int64_t n = docs->n_docs;
  if (n < 0 || n > b->max_docs || (n > 0 && !docs->offsets))
    return fail(ctx, MRC_ERR_INVALID, "mrc_batch_launch: n_docs outside [0, max_docs]");
  const bool dev = n > 0 && on_device(docs->offsets);
  int64_t T = 0;
  cudaError_t e = cudaSuccess;
  if (n > 0) {
    if (dev)
      e = cudaMemcpy(&T, docs->offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost);
    else
      T = docs->offsets[n];
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading offsets[n_docs]");
    if (T < 0 || T > b->max_tokens) return fail(ctx, MRC_ERR_INVALID, "mrc_batch_launch: more tokens than max_tokens");
    e = cudaMemcpyAsync(b->d_offsets, docs->offsets, sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyDefault,
                        ctx->stream);
    if (e == cudaSuccess && T > 0)
      e = cudaMemcpyAsync(b->d_tokens, docs->tokens, sizeof(int32_t) * (size_t)T, cudaMemcpyDefault, ctx->stream);
  } else {
    e = cudaMemsetAsync(b->d_offsets, 0, sizeof(int64_t), ctx->stream);
  }
  if (e == cudaSuccess && b->fused) {
    // the kernel reads the document count; offsets past it are not read
    b->h_counts[4] = (unsigned long long)n;
    e = cudaMemcpyAsync(b->d_nlive, b->h_counts + 4, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream);
  } else if (e == cudaSuccess && n < b->max_docs) {
    const int64_t m = b->max_docs - n;
    k_pad_offsets<<<(unsigned)((m + 255) / 256), 256, 0, ctx->stream>>>(b->d_offsets, n, b->max_docs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_counts, b->d_counts, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_counts + 2, b->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && b->shx)
    e = cudaMemcpyAsync(b->h_counts + 3, b->d_hqoff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->done, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mrc_batch_launch");
  b->pending = true;
  b->has_result = false;
  b->last_n = n;
  return MRC_OK;
}

int32_t mrc_batch_poll(mrc_batch* b) {
  if (!b || !b->pending) return 1;
  const cudaError_t e = cudaEventQuery(b->done);
  if (e == cudaErrorNotReady) {
    cudaGetLastError();
    return 0;
  }
  return 1;
}

mrc_status mrc_batch_wait(mrc_batch* b, mrc_pair* pairs, int64_t capacity, int64_t* n_pairs, int64_t* query_offsets) {
  TraceRange trace(__func__);
  if (!b) return MRC_ERR_INVALID;
  mrc_ctx* ctx = b->ctx;
  cudaSetDevice(ctx->device);
  if (n_pairs) *n_pairs = 0;
  const mrc_status st = finish_launch(b);
  if (st != MRC_OK) return st;
  const int64_t total = (int64_t)b->h_counts[0];
  const int64_t cand = (int64_t)b->h_counts[1];
  if (n_pairs) *n_pairs = total;
  if (cand > b->cand_cap)
    return fail(ctx, MRC_ERR_CAPACITY, "candidate list overflowed: create the batch with a larger capacity");
  return copy_out(b, b->d_grouped, total, b->capacity, b->d_qoff, pairs, capacity, query_offsets, "copying batch pairs");
}

mrc_status mrc_batch_attach_simhash(mrc_batch* b, const mrc_simhash_index* index, int32_t hamming_max,
                                    int64_t capacity) {
  TraceRange trace(__func__);
  if (!b) return MRC_ERR_INVALID;
  mrc_ctx* ctx = b->ctx;
  cudaSetDevice(ctx->device);
  if (b->pending) return fail(ctx, MRC_ERR_INVALID, "mrc_batch_attach_simhash: a launch is in flight");
  if (!index || capacity < 1 || hamming_max < 0 || hamming_max > index->hamming_max)
    return fail(ctx, MRC_ERR_INVALID, "mrc_batch_attach_simhash: NULL index, capacity < 1 or a distance above the "
                                      "index's");
  if (index->device != ctx->device) return fail(ctx, MRC_ERR_INVALID, "the fingerprint index is on another device");
  if (b->shx) return fail(ctx, MRC_ERR_INVALID, "mrc_batch_attach_simhash: a fingerprint index is attached already");
  cudaError_t e = cudaMalloc(&b->d_hpairs, sizeof(mrc_pair) * (size_t)capacity);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_hgrouped, sizeof(mrc_pair) * (size_t)capacity);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_hqoff, sizeof(int64_t) * (size_t)(b->max_docs + 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_hqcnt, sizeof(int32_t) * (size_t)b->max_docs * b->qstride);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_hqfill, sizeof(int32_t) * (size_t)b->max_docs * b->qstride);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "mrc_batch_attach_simhash allocations");
  b->shx = index;
  b->hmax = hamming_max;
  b->h_capacity = capacity;
  e = capture(b);
  if (e != cudaSuccess) {
    b->shx = nullptr;
    return cuda_fail(ctx, e, "capturing the batch pipeline with its Hamming leg");
  }
  return MRC_OK;
}

mrc_status mrc_batch_hamming(mrc_batch* b, mrc_pair* pairs, int64_t capacity, int64_t* n_pairs,
                             int64_t* query_offsets) {
  TraceRange trace(__func__);
  if (!b) return MRC_ERR_INVALID;
  mrc_ctx* ctx = b->ctx;
  if (n_pairs) *n_pairs = 0;
  if (!b->shx) return fail(ctx, MRC_ERR_INVALID, "mrc_batch_hamming: no fingerprint index attached");
  cudaSetDevice(ctx->device);
  const mrc_status st = finish_launch(b);
  if (st != MRC_OK) return st;
  int64_t total = 0;  // the real queries' pairs: grouped by query, they come first
  std::memcpy(&total, b->h_counts + 3, sizeof(int64_t));
  if (n_pairs) *n_pairs = total;
  return copy_out(b, b->d_hgrouped, total, b->h_capacity, b->d_hqoff, pairs, capacity, query_offsets,
                  "copying Hamming pairs");
}

mrc_status mrc_batch_tune(mrc_batch* b, int32_t tile_n, int32_t ring, int32_t prefetch) {
  TraceRange trace(__func__);
  if (!b) return MRC_ERR_INVALID;
  mrc_ctx* ctx = b->ctx;
  cudaSetDevice(ctx->device);
  if (b->pending) return fail(ctx, MRC_ERR_INVALID, "mrc_batch_tune: a launch is in flight");
  if ((tile_n != 0 && tile_n != 128 && tile_n != 256) || ring < 0 || ring == 1 || ring > 64 || prefetch < -1 ||
      prefetch > 64)
    return fail(ctx, MRC_ERR_INVALID, "mrc_batch_tune: tile_n in {0, 128, 256}, ring 0 or in [2, 64], prefetch in [-1, 64]");
  const int32_t old_tile = b->tile_n, old_ring = b->ring, old_pf = b->prefetch;
  b->tile_n = tile_n;
  b->ring = ring;
  b->prefetch = prefetch;
  const cudaError_t e = capture(b);
  if (e != cudaSuccess) {
    b->tile_n = old_tile;
    b->ring = old_ring;
    b->prefetch = old_pf;
    return cuda_fail(ctx, e, "re-capturing the batch pipeline");
  }
  return MRC_OK;
}

int32_t mrc_batch_kernels(const mrc_batch* b) { return b ? b->kernel_nodes : -1; }

mrc_status mrc_batch_phase_ns(mrc_batch* b, int64_t* phase_ns) {
  if (!b || !phase_ns) return MRC_ERR_INVALID;
  mrc_ctx* ctx = b->ctx;
  cudaSetDevice(ctx->device);
  if (!b->fused) return fail(ctx, MRC_ERR_UNSUPPORTED, "mrc_batch_phase_ns: the batch runs separate kernels");
  const mrc_status st = finish_launch(b);
  if (st != MRC_OK) return st;
  unsigned long long t[kBatchStamps];
  cudaError_t e = cudaMemcpyAsync(t, b->d_stamps, sizeof(t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the phase timestamps");
  for (int i = 0; i + 1 < kBatchStamps; ++i) phase_ns[i] = t[i + 1] >= t[i] ? (int64_t)(t[i + 1] - t[i]) : -1;
  return MRC_OK;
}

const char* mrc_batch_last_error(const mrc_batch* b) { return b ? b->ctx->last_error.c_str() : "no batch"; }

void mrc_batch_free(mrc_batch* b) { release(b); }

}  // extern "C"
