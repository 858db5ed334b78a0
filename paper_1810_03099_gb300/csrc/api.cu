// api.cu -- the C ABI declared in include/mrc.h: contexts, indexes and the five entry points.
//
// Host-side logic only; every per-document and per-pair step runs in the
// kernels of ingest.cu, compare_tc.cu, simhash_match.cu and tail.cu. The one
// host computation on the data path is the reference selection of Section IV
// (a sort of the vocabulary by document frequency, once per index build).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <tuple>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.h"

using mrc::Buffer;

namespace mrc {

mrc_status fail(mrc_ctx* ctx, mrc_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

mrc_status cuda_fail(mrc_ctx* ctx, cudaError_t e, const char* what) {
  cudaGetLastError();
  const mrc_status st = (e == cudaErrorMemoryAllocation) ? MRC_ERR_OOM : MRC_ERR_CUDA;
  return fail(ctx, st, std::string(what) + ": " + cudaGetErrorString(e));
}

void* ws_get(mrc_ctx* ctx, const char* slot, size_t bytes, mrc_status* st) {
  Buffer& b = ctx->ws[slot];
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return b.ptr;
  if (b.ptr) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
  }
  // grow geometrically so that slowly growing requests do not reallocate every call
  size_t want = std::max(bytes + bytes / 8, (size_t)256);
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    if (st) *st = MRC_ERR_OOM;
    ctx->last_error = std::string("device allocation of ") + std::to_string(want) + " bytes for " + slot + " failed";
    return nullptr;
  }
  b.ptr = p;
  b.bytes = want;
  return p;
}

static void record_index_event(mrc_ctx* ctx, cudaEvent_t* ev) {
  if (!*ev && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    *ev = nullptr;
    return;
  }
  cudaEventRecord(*ev, ctx->stream);
}

static void wait_index_event(mrc_ctx* ctx, const mrc_index* x, cudaEvent_t ev) {
  if (ctx->stream == x->stream) return;
  if (ev) cudaStreamWaitEvent(ctx->stream, ev, 0);
  else cudaStreamSynchronize(x->stream);
}

void mark_index_ready(mrc_ctx* ctx, mrc_index* x) { record_index_event(ctx, &x->ready); }
void wait_for_index(mrc_ctx* ctx, const mrc_index* x) { wait_index_event(ctx, x, x->ready); }
void mark_index_tables(mrc_ctx* ctx, mrc_index* x) { record_index_event(ctx, &x->tables); }
void wait_for_index_tables(mrc_ctx* ctx, const mrc_index* x) { wait_index_event(ctx, x, x->tables); }

int resident_ctas(const void* func, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> smem_set;  // (kernel, device) -> limit set
  static std::map<std::tuple<const void*, int, int, size_t>, int> occ;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_tuple(func, dev, threads, smem);
  const auto it = occ.find(key);
  if (it != occ.end()) return it->second;
  size_t& lim = smem_set[std::make_pair(func, dev)];
  if (smem > 48 * 1024 && smem > lim) {
    if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    lim = smem;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  occ[key] = per_sm;
  return per_sm;
}

void timing_begin(mrc_ctx* ctx, const char* name, double bytes, double flops, cudaEvent_t* ev_out) {
  *ev_out = nullptr;
  if (!ctx->timing) return;
  auto get = [&]() {
    cudaEvent_t e;
    if (!ctx->free_events.empty()) {
      e = ctx->free_events.back();
      ctx->free_events.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  };
  PendingTiming pt;
  pt.name = name;
  pt.start = get();
  pt.stop = get();
  pt.bytes = bytes;
  pt.flops = flops;
  cudaEventRecord(pt.start, ctx->stream);
  ctx->pending.push_back(pt);
  *ev_out = pt.start;
}

void timing_end(mrc_ctx* ctx, cudaEvent_t start) {
  if (!start) return;
  for (auto it = ctx->pending.rbegin(); it != ctx->pending.rend(); ++it)
    if (it->start == start) {
      cudaEventRecord(it->stop, ctx->stream);
      return;
    }
}

static void collect_timings(mrc_ctx* ctx) {
  for (auto& pt : ctx->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(pt.stop) == cudaSuccess) cudaEventElapsedTime(&ms, pt.start, pt.stop);
    cudaGetLastError();
    KernelStat* ks = nullptr;
    for (auto& s : ctx->stats)
      if (s.first == pt.name) ks = &s.second;
    if (!ks) {
      ctx->stats.emplace_back(pt.name, KernelStat{});
      ks = &ctx->stats.back().second;
    }
    ks->launches += 1;
    ks->ms += ms;
    ks->bytes += pt.bytes;
    ks->flops += pt.flops;
    ctx->free_events.push_back(pt.start);
    ctx->free_events.push_back(pt.stop);
  }
  ctx->pending.clear();
}

}  // namespace mrc

using namespace mrc;

namespace {

constexpr uint64_t kDefaultSeed = 0x1810030990ull;
constexpr float kF16CompareBound = 2e-3f;  // > max |fp16 cosine - cosine| of unit vectors (~1e-3)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device address of page-locked host memory (read by kernels over the CPU-GPU link), or
// NULL for any other pointer.
const void* pinned_device_ptr(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Device copy of a caller buffer (the buffer itself when it already lives on the device; with
// zero_copy, page-locked host memory is read in place by the kernels instead of being copied).
const void* stage_in(mrc_ctx* ctx, const char* slot, const void* p, size_t bytes, mrc_status* st,
                     bool zero_copy = false) {
  if (!p || is_device_ptr(p)) return p;
  if (zero_copy)
    if (const void* dp = pinned_device_ptr(p)) return dp;
  void* d = ws_get(ctx, slot, bytes, st);
  if (!d) return nullptr;
  if (bytes && cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
    *st = cuda_fail(ctx, cudaGetLastError(), "host-to-device copy");
    return nullptr;
  }
  return d;
}

struct Scope {
  Scope(mrc_ctx* c, const char* name) : trace(name), ctx(c) {
    int cur = -1;
    cudaGetDevice(&cur);
    prev = cur;
    if (cur != ctx->device) cudaSetDevice(ctx->device);
  }
  ~Scope() {
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
  }
  TraceRange trace;  // first constructed, last destroyed: the range covers the whole call
  mrc_ctx* ctx;
  int prev;
};

// Status of a call's device error word h (already on the host).
mrc_status err_status(mrc_ctx* ctx, int32_t h) {
  if (h & kErrTimeout) return fail(ctx, MRC_ERR_TIMEOUT, "a bounded device wait expired");
  if (h & kErrBadOffsets) return fail(ctx, MRC_ERR_INVALID, "offsets must start at 0 and be non-decreasing");
  if (h & kErrTooLong)
    return fail(ctx, MRC_ERR_UNSUPPORTED, "a document is longer than MRC_MAX_DOC_TOKENS tokens");
  if (h & kErrBadToken) return fail(ctx, MRC_ERR_INVALID, "a token id is outside [0, vocab)");
  if (h & kErrTable) return fail(ctx, MRC_ERR_CUDA, "internal: per-document term table overflow");
  if (h & kErrOverflow)
    return fail(ctx, MRC_ERR_CAPACITY, "a candidate buffer overflowed: pairs may be missing; repeat the call with "
                                       "its synchronous form");
  return MRC_OK;
}

mrc_status check_err_word(mrc_ctx* ctx, int32_t* d_err) {
  int32_t* h = (int32_t*)((char*)ctx->pinned + 256);
  cudaError_t e = cudaMemcpyAsync(h, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel execution");
  return err_status(ctx, *h);
}

int32_t* call_err(mrc_ctx* ctx, mrc_status* st) {
  int32_t* e = (int32_t*)ws_get(ctx, "call.err", sizeof(int32_t), st);
  if (e) cudaMemsetAsync(e, 0, sizeof(int32_t), ctx->stream);
  return e;
}

// Attaches a bag-of-terms workspace to d when it fits (8 bytes per token, at most 16 GB), so
// that a call's second pass over the same documents reads the bag instead of hashing again.
void attach_bag(mrc_ctx* ctx, DocsDev* d) {
  if (d->n_tokens <= 0 || 8.0 * (double)d->n_tokens > 16e9) return;
  mrc_status st = MRC_OK;
  int32_t* terms = (int32_t*)ws_get(ctx, "bag.terms", sizeof(int32_t) * (size_t)d->n_tokens, &st);
  int32_t* cnts = (int32_t*)ws_get(ctx, "bag.cnts", sizeof(int32_t) * (size_t)d->n_tokens, &st);
  int32_t* n = (int32_t*)ws_get(ctx, "bag.n", sizeof(int32_t) * (size_t)std::max<int64_t>(d->n_docs, 1), &st);
  if (st != MRC_OK) {  // not enough memory for the bag: the second pass hashes again
    ctx->last_error.clear();
    return;
  }
  d->bag_terms = terms;
  d->bag_cnts = cnts;
  d->bag_n = n;
}

// Docs on the device: host arrays are copied in; returns MRC_OK or an error.
mrc_status stage_docs(mrc_ctx* ctx, const mrc_docs* docs, const char* tag, DocsDev* out, int32_t* d_err) {
  if (!docs || docs->n_docs < 0 || (docs->n_docs > 0 && (!docs->offsets)))
    return fail(ctx, MRC_ERR_INVALID, "docs: NULL or negative n_docs");
  if (docs->n_docs >= (1ll << 31) - 1) return fail(ctx, MRC_ERR_UNSUPPORTED, "more than 2^31 - 2 documents");
  const int64_t n = docs->n_docs;
  mrc_status st = MRC_OK;
  int64_t T = 0;
  const bool off_dev = is_device_ptr(docs->offsets);
  if (off_dev) {
    if (cudaMemcpy(&T, docs->offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return cuda_fail(ctx, cudaGetLastError(), "reading offsets[n_docs]");
  } else {
    T = docs->offsets[n];
  }
  if (T < 0) return fail(ctx, MRC_ERR_INVALID, "offsets[n_docs] < 0");
  if (T > 0 && !docs->tokens) return fail(ctx, MRC_ERR_INVALID, "tokens is NULL");
  std::string s1 = std::string(tag) + ".offsets", s2 = std::string(tag) + ".tokens";
  out->n_docs = n;
  out->offsets = (const int64_t*)stage_in(ctx, s1.c_str(), docs->offsets, sizeof(int64_t) * (size_t)(n + 1), &st);
  if (st != MRC_OK) return st;
  // tokens are read once per pass: page-locked host tokens are read in place (no staging copy)
  out->tokens = (const int32_t*)stage_in(ctx, s2.c_str(), docs->tokens, sizeof(int32_t) * (size_t)T, &st, true);
  if (st != MRC_OK) return st;
  if (T == 0) {
    out->tokens = (const int32_t*)ws_get(ctx, "empty.tokens", 16, &st);
    if (st != MRC_OK) return st;
  }
  out->n_tokens = T;
  out->err = d_err;
  return MRC_OK;
}

bool valid_params(const mrc_params* p, std::string* why) {
  if (!p) return *why = "params is NULL", false;
  if (p->k < 1 || p->k > MRC_MAX_K) return *why = "k must be in [1, MRC_MAX_K]", false;
  if (p->select_mode < MRC_SELECT_ALL || p->select_mode > MRC_SELECT_DF1) return *why = "bad select_mode", false;
  if (p->weighting != MRC_WEIGHT_COUNT && p->weighting != MRC_WEIGHT_TFIDF) return *why = "bad weighting", false;
  if (p->precision < MRC_PREC_FP32 || p->precision > MRC_PREC_FP16) return *why = "bad precision", false;
  if (!(p->margin >= 0.f)) return *why = "margin must be >= 0", false;
  if (p->feature_hash < MRC_HASH_SPLITMIX64 || p->feature_hash > MRC_HASH_SHA1) return *why = "bad feature_hash", false;
  return true;
}

int32_t round_up(int32_t x, int32_t m) { return (x + m - 1) / m * m; }

// Padded operand rows: kp counts fp16 elements (rows of a multiple of 128 bytes, one 128B
// swizzle atom), kp8 counts E4M3 bytes (a multiple of 64: 64-byte rows use the 64B swizzle).
int32_t padded_kp(int32_t k) { return round_up(k, 64); }
int32_t padded_kp8(int32_t k) { return round_up(k, 64); }

// Round to the nearest bfloat16 (8 significant bits), ties to even.
float bf16_round(float f) {
  uint32_t u;
  std::memcpy(&u, &f, sizeof(u));
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  std::memcpy(&f, &u, sizeof(f));
  return f;
}

// The reference weight of term t: idf under TF-IDF, 1 under counts.
double reference_weight(const mrc_params& p, const float* idf, int32_t t) {
  if (p.weighting != MRC_WEIGHT_TFIDF) return 1.0;
  return idf[t];
}

// Index arrays come from the device's stream-ordered memory pool (kept, not returned to the
// driver, between builds), so building and freeing indexes does not synchronise the device.
void free_index_arrays(mrc_index* x) {
  if (x->block) cudaFreeAsync(x->block, x->stream);
  x->block = nullptr;
}

// Every device array of an index in one stream-ordered allocation (256-byte aligned slices):
// the term tables [vocab], the reference norms [k], the signatures and Simhashes [n_docs], and
// the compare operands of the index's precision form.
mrc_status alloc_index_arrays(mrc_ctx* ctx, mrc_index* x) {
  const size_t n = (size_t)std::max<int64_t>(x->n_docs, 1), V = (size_t)x->vocab, k = (size_t)x->k;
  const bool f16 = x->params.precision == MRC_PREC_FP32 || x->params.precision == MRC_PREC_FP16;
  const bool e4m3 = x->params.precision == MRC_PREC_BF16_FP8;
  const bool fh = x->params.feature_hash != MRC_HASH_SPLITMIX64;
  const size_t sizes[] = {4 * V, 4 * V, 8 * V, 4 * k, 4 * n * k, 4 * n * k, 8 * n,
                          f16 ? 2 * n * (size_t)x->kp : 0, e4m3 ? n * (size_t)x->kp8 : 0, e4m3 ? 4 * n : 0,
                          e4m3 ? 4 * ((n + 127) / 128) : 0, 8 * k, fh ? 8 * V : 0, e4m3 ? 4 * k : 0};
  size_t off[14], total = 0;
  for (int q = 0; q < 14; ++q) {
    off[q] = total;
    total += (sizes[q] + 255) / 256 * 256;
  }
  char* b = nullptr;
  if (cudaMallocAsync((void**)&b, total, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, MRC_ERR_OOM, "device allocation failed: index arrays");
  }
  x->block = b;
  x->df = (int32_t*)(b + off[0]);
  x->idf = (float*)(b + off[1]);
  x->tinfo = (TermInfo*)(b + off[2]);
  x->rinv = (float*)(b + off[3]);
  x->sig = (float*)(b + off[4]);
  x->sig_unit = (float*)(b + off[5]);
  x->simhash = (uint64_t*)(b + off[6]);
  x->op_hi = f16 ? (void*)(b + off[7]) : nullptr;
  x->op_lo = nullptr;
  x->op_e4m3 = e4m3 ? (void*)(b + off[8]) : nullptr;
  x->qnorm = e4m3 ? (float*)(b + off[9]) : nullptr;
  x->qnorm_min = e4m3 ? (float*)(b + off[10]) : nullptr;
  x->rnorm = (double*)(b + off[11]);
  x->fhash = fh ? (uint64_t*)(b + off[12]) : nullptr;
  x->rinv16 = e4m3 ? (float*)(b + off[13]) : nullptr;
  if (fh) {  // the Simhash feature of every vocabulary term, computed once per index
    const cudaError_t e = launch_feature_table(ctx, x->vocab, x->params.seed, x->params.feature_hash, x->fhash);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "feature hash table");
  }
  return MRC_OK;
}

// Reference tables of the signature pass: 1 / |R_p| from the squared norms in x->h_rnorm (which
// become the norms), the term table built on the device from the partition of every term
// (part_stage: pinned, [vocab]) and the device idf. The copies read pinned staging, so the
// context's host_ws_done event marks when the staging may be reused.
mrc_status upload_references(mrc_ctx* ctx, mrc_index* x, const int32_t* part_stage, float* rinv_stage,
                             const float* h_idf) {
  const int32_t V = x->vocab;
  for (int32_t q = 0; q < x->k; ++q) {
    x->h_rnorm[q] = std::sqrt(x->h_rnorm[q]);
    rinv_stage[q] = x->h_rnorm[q] > 0 ? (float)(1.0 / x->h_rnorm[q]) : 0.f;
  }
  if (x->rinv16) {  // 1 / |R_p| of the bfloat16-rounded reference weights, summed in term-id order
    std::vector<double> n16(x->k, 0.0);
    for (int32_t t = 0; t < V; ++t) {
      const int32_t q = part_stage[t];
      if (q < 0 || q >= x->k) continue;
      const double r = x->params.weighting == MRC_WEIGHT_TFIDF ? (double)bf16_round(h_idf[t]) : 1.0;
      n16[q] += r * r;
    }
    for (int32_t q = 0; q < x->k; ++q) rinv_stage[x->k + q] = n16[q] > 0 ? (float)(1.0 / std::sqrt(n16[q])) : 0.f;
  }
  mrc_status st = MRC_OK;
  int32_t* d_part = (int32_t*)ws_get(ctx, "build.part", sizeof(int32_t) * V, &st);
  if (st != MRC_OK) return st;
  cudaError_t e = cudaMemcpyAsync(d_part, part_stage, sizeof(int32_t) * V, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(x->rinv, rinv_stage, sizeof(float) * x->k, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && x->rinv16)
    e = cudaMemcpyAsync(x->rinv16, rinv_stage + x->k, sizeof(float) * x->k, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess)
    e = launch_term_info(ctx, x->idf, d_part, V, x->params.weighting == MRC_WEIGHT_TFIDF, 0, x->tinfo);
  if (e == cudaSuccess && !ctx->host_ws_done) e = cudaEventCreateWithFlags(&ctx->host_ws_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->host_ws_done, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "uploading references");
  return MRC_OK;
}

// Partition of every term, read back from the device term table.
mrc_status read_partition(mrc_ctx* ctx, const mrc_index* x, std::vector<int32_t>* part) {
  std::vector<TermInfo> ti(x->vocab);
  const cudaError_t e =
      cudaMemcpyAsync(ti.data(), x->tinfo, sizeof(TermInfo) * x->vocab, cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess || cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return cuda_fail(ctx, cudaGetLastError(), "reading the reference partition");
  part->resize(x->vocab);
  for (int32_t t = 0; t < x->vocab; ++t) (*part)[t] = ti[t].code;
  return MRC_OK;
}

// Grow-only pinned host scratch of the context.
void* host_ws(mrc_ctx* ctx, size_t bytes, mrc_status* st) {
  // copies still in flight may read the buffer: wait for the last of them
  if (ctx->host_ws_done) cudaEventSynchronize(ctx->host_ws_done);
  if (bytes <= ctx->host_ws_bytes) return ctx->host_ws;
  if (ctx->host_ws) cudaFreeHost(ctx->host_ws);
  ctx->host_ws = nullptr;
  ctx->host_ws_bytes = 0;
  if (cudaMallocHost(&ctx->host_ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    ctx->host_ws = nullptr;
    *st = fail(ctx, MRC_ERR_OOM, "pinned host allocation failed");
    return nullptr;
  }
  ctx->host_ws_bytes = bytes;
  return ctx->host_ws;
}

SigOut index_sig_out(mrc_index* x) {
  SigOut o{};
  o.sig = x->sig;
  o.sig_unit = x->sig_unit;
  o.simhash = x->simhash;
  o.op_hi = x->op_hi;
  o.op_lo = x->op_lo;
  o.op_e4m3 = x->op_e4m3;
  o.qnorm = x->qnorm;
  o.kp = x->op_hi ? x->kp : 0;
  o.kp8 = x->op_e4m3 ? x->kp8 : 0;
  return o;
}

// Copies device pairs to a host destination (when `pairs` is host memory).
// Ends a pair-producing call with one synchronisation: reads the pair count (and the call's
// error word, when given; an error takes precedence), then copies host-side results.
// With d_cand (an internal candidate count of capacity cand_cap), that count is read in the
// same synchronisation; when it overflowed, *overflow is set and nothing is copied (the caller
// takes its exhaustive path).
mrc_status finish_pairs(mrc_ctx* ctx, mrc_pair* user, mrc_pair* dev, unsigned long long* d_count, int64_t capacity,
                        int64_t* n_pairs, int32_t* d_err = nullptr, const unsigned long long* d_cand = nullptr,
                        int64_t cand_cap = 0, bool* overflow = nullptr) {
  unsigned long long* hc = (unsigned long long*)ctx->pinned;
  int32_t* he = (int32_t*)((char*)ctx->pinned + 256);
  cudaError_t e = cudaMemcpyAsync(hc, d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && d_cand)
    e = cudaMemcpyAsync(hc + 1, d_cand, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && d_err) e = cudaMemcpyAsync(he, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reading pair count");
  if (d_cand && hc[1] > (unsigned long long)cand_cap) {
    *overflow = true;
    return MRC_OK;
  }
  if (d_err) {
    const mrc_status st = err_status(ctx, *he);
    if (st != MRC_OK) return st;
  }
  const int64_t total = (int64_t)*hc;
  if (n_pairs) *n_pairs = total;
  const int64_t m = std::min<int64_t>(total, capacity);
  if (user != dev && m > 0) {
    e = cudaMemcpyAsync(user, dev, sizeof(mrc_pair) * (size_t)m, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copying pairs to host");
  }
  if (total > capacity)
    return fail(ctx, MRC_ERR_CAPACITY, "more pairs than capacity; *n_pairs holds the total");
  return MRC_OK;
}

mrc_pair* pair_dest(mrc_ctx* ctx, mrc_pair* user, int64_t capacity, mrc_status* st) {
  if (capacity <= 0) return (mrc_pair*)ws_get(ctx, "pairs.none", sizeof(mrc_pair), st);
  if (user && is_device_ptr(user)) return user;
  if (!user) {
    *st = fail(ctx, MRC_ERR_INVALID, "pairs is NULL with capacity > 0");
    return nullptr;
  }
  return (mrc_pair*)ws_get(ctx, "pairs.staging", sizeof(mrc_pair) * (size_t)capacity, st);
}

}  // namespace

extern "C" {

void mrc_params_default(mrc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->k = 8;
  p->L = -1;
  p->select_mode = MRC_SELECT_REGION;
  p->region_start = -1;
  p->weighting = MRC_WEIGHT_TFIDF;
  p->precision = MRC_PREC_FP32;
  p->tau = 0.9f;
  p->margin = 0.02f;
  p->hamming_max = 3;
  p->seed = kDefaultSeed;
}

mrc_status mrc_ctx_create(void* cuda_stream, mrc_ctx** out) {
  if (!out) return MRC_ERR_INVALID;
  *out = nullptr;
  mrc_ctx* c = new (std::nothrow) mrc_ctx();
  if (!c) return MRC_ERR_OOM;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MRC_ERR_CUDA;
  }
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, c->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, c->device);
  if (major != 10) {
    delete c;
    return MRC_ERR_UNSUPPORTED;  // built for sm_103a (Blackwell Ultra) only
  }
  c->stream = (cudaStream_t)cuda_stream;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, c->device) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // freed index memory stays in this process's pool for reuse
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  if (cudaMallocHost(&c->pinned, 4096) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return MRC_ERR_OOM;
  }
  if (cudaMalloc(&c->async_err, sizeof(int32_t)) != cudaSuccess ||
      cudaMemset(c->async_err, 0, sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    if (c->async_err) cudaFree(c->async_err);
    cudaFreeHost(c->pinned);
    delete c;
    return MRC_ERR_OOM;
  }
  *out = c;
  return MRC_OK;
}

void mrc_ctx_destroy(mrc_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->ws)
    if (kv.second.ptr) cudaFree(kv.second.ptr);
  for (auto& pt : ctx->pending) {
    cudaEventDestroy(pt.start);
    cudaEventDestroy(pt.stop);
  }
  for (auto e : ctx->free_events) cudaEventDestroy(e);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->async_err) cudaFree(ctx->async_err);
  if (ctx->host_ws) cudaFreeHost(ctx->host_ws);
  if (ctx->host_ws_done) cudaEventDestroy(ctx->host_ws_done);
  delete ctx;
}

const char* mrc_last_error(const mrc_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

// a2-a4 for an index: signatures, Simhash and packed compare operands of its documents.
mrc_status launch_index_signatures(mrc_ctx* ctx, mrc_index* x, const DocsDev& d) {
  if (x->op_hi) cudaMemsetAsync(x->op_hi, 0, sizeof(uint16_t) * (size_t)x->n_docs * x->kp, ctx->stream);
  if (x->op_lo) cudaMemsetAsync(x->op_lo, 0, sizeof(uint16_t) * (size_t)x->n_docs * x->kp, ctx->stream);
  if (x->op_e4m3) cudaMemsetAsync(x->op_e4m3, 0, (size_t)x->n_docs * x->kp8, ctx->stream);
  cudaError_t e = launch_signature(ctx, d, x->vocab, x->tinfo, x->rinv, x->rinv16, x->k, x->params.seed, x->fhash,
                                   index_sig_out(x));
  if (e == cudaSuccess && x->qnorm_min) e = launch_block_min(ctx, x->qnorm, x->n_docs, x->qnorm_min);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "signature pass");
  return MRC_OK;
}

mrc_status mrc_build_index(mrc_ctx* ctx, const mrc_docs* corpus, int32_t vocab, const mrc_params* params,
                           mrc_index** out) {
  if (!ctx || !out) return MRC_ERR_INVALID;
  *out = nullptr;
  Scope scope(ctx, __func__);
  std::string why;
  if (!valid_params(params, &why)) return fail(ctx, MRC_ERR_INVALID, why);
  if (vocab < 1) return fail(ctx, MRC_ERR_INVALID, "vocab must be >= 1");
  if (!corpus || corpus->n_docs < 1) return fail(ctx, MRC_ERR_INVALID, "the index corpus needs >= 1 document");
  mrc_status st = MRC_OK;
  int32_t* d_err = call_err(ctx, &st);
  if (!d_err) return st;
  DocsDev d;
  if ((st = stage_docs(ctx, corpus, "build", &d, d_err)) != MRC_OK) return st;

  mrc_index* x = new mrc_index();
  x->device = ctx->device;
  x->stream = ctx->stream;
  x->params = *params;
  x->n_docs = d.n_docs;
  x->vocab = vocab;
  x->k = params->k;
  x->kp = padded_kp(params->k);
  x->kp8 = padded_kp8(params->k);
  auto bail = [&](mrc_status s) {
    cudaStreamSynchronize(ctx->stream);
    free_index_arrays(x);
    delete x;
    return s;
  };
  if ((st = alloc_index_arrays(ctx, x)) != MRC_OK) return bail(st);
  cudaError_t e = cudaMemsetAsync(x->df, 0, sizeof(int32_t) * vocab, ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "memset"));

  // a1: document frequencies (storing each document's bag of terms), then idf
  attach_bag(ctx, &d);
  d.bag_write = 1;
  e = launch_df(ctx, d, x->df, vocab);
  d.bag_write = 0;
  d.bag_read = 1;
  d.lists_ready = 1;
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "df pass"));
  e = launch_idf(ctx, d.n_docs, x->df, vocab, params->weighting, x->idf, nullptr);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "idf"));
  // References (Section IV), on the device for every selection mode: the df histogram, the
  // band of df values the selection meets, and the band's terms ranked by (df descending, id
  // ascending); a band of more than 8,192 terms takes the general pass (a radix sort) after the
  // call's one synchronisation.
  {
    const size_t hb = sizeof(int32_t) * ((size_t)d.n_docs + 2);
    int32_t* hist = (int32_t*)ws_get(ctx, "sel.hist", hb, &st);
    int32_t* above = (int32_t*)ws_get(ctx, "sel.above", hb, &st);
    long long* sstate = (long long*)ws_get(ctx, "sel.state", sizeof(long long) * device_selection_words(), &st);
    unsigned long long* keys = (unsigned long long*)ws_get(ctx, "sel.keys", 8 * 8192, &st);
    int32_t* d_part = (int32_t*)ws_get(ctx, "build.part", sizeof(int32_t) * vocab, &st);
    if (st != MRC_OK) return bail(st);
    const bool tfidf = params->weighting == MRC_WEIGHT_TFIDF;
    const int64_t L = params->L < 0 ? 32ll * params->k : params->L;
    e = launch_select_region(ctx, x->df, vocab, d.n_docs, L, params->region_start, params->select_mode,
                             tfidf ? x->idf : nullptr, 0, x->k, hist, above, sstate, keys, d_part, x->rnorm, x->rinv,
                             x->rinv16);
    if (e == cudaSuccess) e = launch_term_info(ctx, x->idf, d_part, vocab, tfidf, 0, x->tinfo);
    if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "reference selection"));
    // one synchronisation, before the signature pass: the error word of the df pass, the
    // selection state and |R_p|; the call then returns while the signature pass runs (it meets
    // only documents the df pass validated)
    char* hs = (char*)ctx->pinned + 1024;
    auto read_selection = [&]() {
      cudaError_t r = cudaMemcpyAsync(hs, sstate, sizeof(long long) * device_selection_words(), cudaMemcpyDeviceToHost,
                                      ctx->stream);
      if (r == cudaSuccess)
        r = cudaMemcpyAsync(hs + 128, x->rnorm, sizeof(double) * x->k, cudaMemcpyDeviceToHost, ctx->stream);
      return r;
    };
    if ((e = read_selection()) != cudaSuccess) return bail(cuda_fail(ctx, e, "reading the selection"));
    if ((st = check_err_word(ctx, d_err)) != MRC_OK) return bail(st);  // synchronises the stream
    if (((const long long*)hs)[6] != 0) {  // a band larger than the small path holds
      void* gs = ws_get(ctx, "sel.general", select_general_bytes(vocab), &st);
      if (st != MRC_OK) return bail(st);
      e = launch_select_general(ctx, x->df, vocab, tfidf ? x->idf : nullptr, 0, x->k, sstate, gs, d_part, x->rnorm,
                                x->rinv, x->rinv16);
      if (e == cudaSuccess) e = launch_term_info(ctx, x->idf, d_part, vocab, tfidf, 0, x->tinfo);
      if (e == cudaSuccess) e = read_selection();
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "reference selection (general pass)"));
    }
    const long long* hss = (const long long*)hs;
    x->L_used = hss[1];
    x->h_rnorm.assign((const double*)(hs + 128), (const double*)(hs + 128) + x->k);
  }
  mark_index_tables(ctx, x);
  if ((st = launch_index_signatures(ctx, x, d)) != MRC_OK) return bail(st);
  // The df pass already validated these documents (offsets, lengths, token ids) and the
  // signature pass meets the same ones, so the call returns without waiting for it: the index
  // is ready in stream order, like any device result.
  mark_index_ready(ctx, x);
  *out = x;
  return MRC_OK;
}

mrc_status mrc_text_grams(mrc_ctx* ctx, int64_t n_docs, const int64_t* text_offsets, const uint8_t* text,
                          int64_t* gram_offsets, int32_t* grams, int64_t capacity, int64_t* n_grams) {
  if (!ctx) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  if (n_docs < 0 || !text_offsets || !gram_offsets || !n_grams || capacity < 0 || (capacity > 0 && !grams))
    return fail(ctx, MRC_ERR_INVALID, "mrc_text_grams: NULL pointer or negative size");
  if (n_docs >= (1ll << 40)) return fail(ctx, MRC_ERR_UNSUPPORTED, "too many documents");
  *n_grams = 0;
  mrc_status st = MRC_OK;
  int32_t* d_err = call_err(ctx, &st);
  if (!d_err) return st;
  int64_t B = 0;
  if (is_device_ptr(text_offsets)) {
    if (cudaMemcpy(&B, text_offsets + n_docs, sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return cuda_fail(ctx, cudaGetLastError(), "reading text_offsets[n_docs]");
  } else {
    B = text_offsets[n_docs];
  }
  if (B < 0) return fail(ctx, MRC_ERR_INVALID, "text_offsets[n_docs] < 0");
  if (B > 0 && !text) return fail(ctx, MRC_ERR_INVALID, "text is NULL");
  const int64_t* d_off =
      (const int64_t*)stage_in(ctx, "text.offsets", text_offsets, sizeof(int64_t) * (size_t)(n_docs + 1), &st);
  if (st != MRC_OK) return st;
  const uint8_t* d_text = B > 0 ? (const uint8_t*)stage_in(ctx, "text.bytes", text, (size_t)B, &st) : nullptr;
  if (st != MRC_OK) return st;
  const bool go_host = !is_device_ptr(gram_offsets), g_host = capacity > 0 && !is_device_ptr(grams);
  int64_t* d_go =
      go_host ? (int64_t*)ws_get(ctx, "text.gram_offsets", sizeof(int64_t) * (size_t)(n_docs + 1), &st) : gram_offsets;
  int32_t* d_g = g_host ? (int32_t*)ws_get(ctx, "text.grams", sizeof(int32_t) * (size_t)capacity, &st) : grams;
  const int64_t tiles = text_gram_tiles(B);
  int64_t* tile_doc = (int64_t*)ws_get(ctx, "text.tile_doc", sizeof(int64_t) * (size_t)std::max<int64_t>(tiles, 1), &st);
  int32_t* tile_cnt = (int32_t*)ws_get(ctx, "text.tile_cnt", sizeof(int32_t) * (size_t)std::max<int64_t>(tiles, 1), &st);
  int64_t* tile_base = (int64_t*)ws_get(ctx, "text.tile_base", sizeof(int64_t) * (size_t)(tiles + 1), &st);
  int64_t* group_sum =
      (int64_t*)ws_get(ctx, "text.group_sum", sizeof(int64_t) * (size_t)std::max<int64_t>((tiles + 1023) / 1024, 1), &st);
  if (st != MRC_OK) return st;
  cudaError_t e = launch_text_grams(ctx, n_docs, d_off, d_text, B, d_go, d_g, capacity, tile_doc, tile_cnt, group_sum,
                                    tile_base, d_err);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "text 3-grams");
  int64_t* h_total = (int64_t*)((char*)ctx->pinned + 512);
  e = cudaMemcpyAsync(h_total, tile_base + tiles, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "reading the 3-gram total");
  if ((st = check_err_word(ctx, d_err)) != MRC_OK) return st;  // synchronises the stream
  const int64_t total = *h_total;
  *n_grams = total;
  if (go_host)
    e = cudaMemcpyAsync(gram_offsets, d_go, sizeof(int64_t) * (size_t)(n_docs + 1), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && g_host && total > 0)
    e = cudaMemcpyAsync(grams, d_g, sizeof(int32_t) * (size_t)std::min(total, capacity), cudaMemcpyDeviceToHost,
                        ctx->stream);
  if (e == cudaSuccess && (go_host || g_host)) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copying the 3-grams out");
  if (total > capacity) return fail(ctx, MRC_ERR_CAPACITY, "more 3-grams than capacity");
  return MRC_OK;
}

mrc_status mrc_signature(mrc_ctx* ctx, const mrc_index* index, const mrc_docs* docs, float* sig, uint64_t* simhash) {
  if (!ctx || !index) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  wait_for_index(ctx, index);
  if (!docs) return fail(ctx, MRC_ERR_INVALID, "docs is NULL");
  if (docs->n_docs == 0) return MRC_OK;
  if (!sig && !simhash) return fail(ctx, MRC_ERR_INVALID, "no output requested");
  mrc_status st = MRC_OK;
  int32_t* d_err = call_err(ctx, &st);
  if (!d_err) return st;
  DocsDev d;
  if ((st = stage_docs(ctx, docs, "sig", &d, d_err)) != MRC_OK) return st;
  const int64_t n = d.n_docs;
  const bool sig_host = sig && !is_device_ptr(sig), sh_host = simhash && !is_device_ptr(simhash);
  SigOut o{};
  o.sig = sig_host ? (float*)ws_get(ctx, "sig.out", sizeof(float) * (size_t)n * index->k, &st) : sig;
  o.simhash = sh_host ? (uint64_t*)ws_get(ctx, "sig.simhash", sizeof(uint64_t) * (size_t)n, &st) : simhash;
  if (st != MRC_OK) return st;
  cudaError_t e = launch_signature(ctx, d, index->vocab, index->tinfo, index->rinv, nullptr, index->k,
                                   index->params.seed, index->fhash, o);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "signature pass");
  if ((st = check_err_word(ctx, d_err)) != MRC_OK) return st;
  if (sig_host) e = cudaMemcpyAsync(sig, o.sig, sizeof(float) * (size_t)n * index->k, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && sh_host)
    e = cudaMemcpyAsync(simhash, o.simhash, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess && (sig_host || sh_host)) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "copying signatures");
  return MRC_OK;
}

// mrc_match, or with d_total its stream-ordered form: the pair count goes to *d_total (device),
// errors to the context's stream-ordered error word, and nothing waits.
static mrc_status match_impl(mrc_ctx* ctx, const mrc_index* index, const float* query_sig, int64_t nq, float tau,
                      mrc_pair* pairs, int64_t capacity, int64_t* n_pairs, unsigned long long* d_total) {
  if (!ctx || !index) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  wait_for_index(ctx, index);
  if (capacity < 0) return fail(ctx, MRC_ERR_INVALID, "capacity < 0");
  if (query_sig && nq < 0) return fail(ctx, MRC_ERR_INVALID, "nq < 0");
  if (n_pairs) *n_pairs = 0;
  mrc_status st = MRC_OK;
  const bool async = d_total != nullptr;
  if (async && ((capacity > 0 && (!pairs || !is_device_ptr(pairs))) || !is_device_ptr(d_total)))
    return fail(ctx, MRC_ERR_INVALID, "stream-ordered calls take device pairs and a device pair count");
  int32_t* d_err = async ? ctx->async_err : call_err(ctx, &st);
  if (!d_err) return st;
  const int64_t N = index->n_docs;
  const int32_t prec = index->params.precision;
  unsigned long long* d_count = (unsigned long long*)ws_get(ctx, "match.count", 2 * sizeof(unsigned long long), &st);
  mrc_pair* dst = pair_dest(ctx, pairs, capacity, &st);
  if (st != MRC_OK) return st;
  cudaMemsetAsync(d_count, 0, 2 * sizeof(unsigned long long), ctx->stream);
  unsigned long long* pc = async ? d_total : d_count;  // the pair counter; d_count[1] counts candidates
  if (async) cudaMemsetAsync(pc, 0, sizeof(unsigned long long), ctx->stream);
  if ((query_sig && nq == 0) || (!query_sig && N < 2))
    return async ? MRC_OK : finish_pairs(ctx, pairs, dst, d_count, capacity, n_pairs);

  // query operands (packed unit signatures) or the index itself
  const void *a_hi = index->op_hi, *a8 = index->op_e4m3;
  const float* a_unit = index->sig_unit;
  const float* a_norm = index->qnorm;
  int64_t na = N;
  if (query_sig) {
    const float* q = (const float*)stage_in(ctx, "match.q", query_sig, sizeof(float) * (size_t)nq * index->k, &st);
    if (st != MRC_OK) return st;
    float* qu = (float*)ws_get(ctx, "match.qunit", sizeof(float) * (size_t)nq * index->k, &st);
    void* qh = prec != MRC_PREC_BF16_FP8 ? ws_get(ctx, "match.qhi", 2 * (size_t)nq * index->kp, &st) : nullptr;
    void* q8 = prec == MRC_PREC_BF16_FP8 ? ws_get(ctx, "match.q8", (size_t)nq * index->kp8, &st) : nullptr;
    float* qn = prec == MRC_PREC_BF16_FP8 ? (float*)ws_get(ctx, "match.qnorm", sizeof(float) * (size_t)nq, &st)
                                          : nullptr;
    if (st != MRC_OK) return st;
    cudaError_t e =
        launch_pack(ctx, q, nq, index->k, 1, qh, nullptr, q8, qn, qu, qh ? index->kp : 0, q8 ? index->kp8 : 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "packing queries");
    a_hi = qh;
    a8 = q8;
    a_unit = qu;
    a_norm = qn;
    na = nq;
  }

  // Candidates from the tensor cores at a lowered threshold, then FP32 rescoring of every
  // candidate. FP32 form: fp16 unit vectors; |fp16 cosine - cosine| <= 2^-10 sum|x_p y_p| +
  // subnormal and FP32-accumulation terms <= ~1e-3 (Cauchy-Schwarz), so tau - 2e-3 loses no
  // pair and the rescored scores are FP32-accurate; the FP16 form computes the same. E4M3
  // form: tau - margin.
  GemmArgs g{};
  g.na = na;
  g.nb = N;
  g.triangle = query_sig ? 0 : 1;
  g.prefetch = -1;
  g.err = d_err;
  g.out_scale = 1.0f;
  g.fmt = prec == MRC_PREC_BF16_FP8 ? OP_E4M3 : OP_F16;
  g.a_hi = prec == MRC_PREC_BF16_FP8 ? a8 : a_hi;
  g.b_hi = prec == MRC_PREC_BF16_FP8 ? index->op_e4m3 : index->op_hi;
  g.kbytes = prec == MRC_PREC_BF16_FP8 ? index->kp8 : index->kp * 2;
  if (prec == MRC_PREC_BF16_FP8) {
    g.out_scale = 1.0f / (kE4M3Scale * kE4M3Scale);
    g.a_norm = a_norm;
    g.b_norm = index->qnorm;
    g.b_norm_min = index->qnorm_min;
  }
  // fp16 operands (FP32 and FP16 forms): the proven bound; E4M3: the margin
  g.thresh = tau - (prec == MRC_PREC_BF16_FP8 ? index->params.margin : kF16CompareBound);
  if (!ctx->rescore) {  // diagnostics: the compare's candidates are the result
    g.exact_scores = 1;
    g.pairs = dst;
    g.count = pc;
    g.capacity = capacity;
    cudaError_t e = launch_gemm_compare(ctx, g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "signature compare");
    return async ? MRC_OK : finish_pairs(ctx, pairs, dst, d_count, capacity, n_pairs, d_err);
  }
  // candidates, then their rescoring (which reads the candidate count on the device), then one
  // synchronisation; only if the candidate buffer overflowed is the pass repeated, larger
  int64_t cand_cap = std::max<int64_t>(4 * capacity, 1 << 20);
  for (int attempt = 0; attempt < 2; ++attempt) {
    mrc_pair* cand = (mrc_pair*)ws_get(ctx, "match.cand", sizeof(mrc_pair) * (size_t)cand_cap, &st);
    if (st != MRC_OK) return st;
    cudaMemsetAsync(d_count, 0, 2 * sizeof(unsigned long long), ctx->stream);
    if (async) cudaMemsetAsync(pc, 0, sizeof(unsigned long long), ctx->stream);
    g.pairs = cand;
    g.count = d_count + 1;
    g.capacity = cand_cap;
    cudaError_t e = launch_gemm_compare(ctx, g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "signature compare");
    // the synchronous form retries an overflow below; the stream-ordered form reports it
    e = launch_rescore(ctx, cand, d_count + 1, cand_cap, a_unit, index->sig_unit, index->k, tau, dst, pc, capacity,
                       async ? d_err : nullptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rescoring");
    if (async) return MRC_OK;  // a candidate overflow is reported by mrc_ctx_sync
    unsigned long long* hc = (unsigned long long*)ctx->pinned;
    e = cudaMemcpyAsync(hc + 1, d_count + 1, sizeof(unsigned long long), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reading candidate count");
    if ((st = check_err_word(ctx, d_err)) != MRC_OK) return st;  // synchronises the stream
    const int64_t nc = (int64_t)hc[1];
    if (nc <= cand_cap) break;
    cand_cap = nc + nc / 8 + 1024;
  }
  return finish_pairs(ctx, pairs, dst, d_count, capacity, n_pairs);
}

// cosine_allpairs, or with d_total its stream-ordered form (see match_impl). The bound-pruned
// path reads the head/tail split's sizes on the device, so nothing waits (unless per-kernel
// timing is on or the head's upper bound is too wide); errors of the stream-ordered form go to
// the context's error word.
static mrc_status cosine_impl(mrc_ctx* ctx, const mrc_index* index, const mrc_docs* docs, float tau, mrc_pair* pairs,
                       int64_t capacity, int64_t* n_pairs, unsigned long long* d_total) {
  if (!ctx || !index) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  wait_for_index_tables(ctx, index);  // idf and the term table only
  if (capacity < 0) return fail(ctx, MRC_ERR_INVALID, "capacity < 0");
  if (n_pairs) *n_pairs = 0;
  mrc_status st = MRC_OK;
  const bool async = d_total != nullptr;
  if (async && ((capacity > 0 && (!pairs || !is_device_ptr(pairs))) || !is_device_ptr(d_total)))
    return fail(ctx, MRC_ERR_INVALID, "stream-ordered calls take device pairs and a device pair count");
  int32_t* d_err = async ? ctx->async_err : call_err(ctx, &st);
  if (!d_err) return st;
  DocsDev d;
  if ((st = stage_docs(ctx, docs, "cos", &d, d_err)) != MRC_OK) return st;
  const int64_t N = d.n_docs;
  const int32_t V = index->vocab;
  unsigned long long* d_count =
      async ? d_total : (unsigned long long*)ws_get(ctx, "cos.count", sizeof(unsigned long long), &st);
  mrc_pair* dst = pair_dest(ctx, pairs, capacity, &st);
  if (st != MRC_OK) return st;
  cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), ctx->stream);
  if (N < 2) return async ? MRC_OK : finish_pairs(ctx, pairs, dst, d_count, capacity, n_pairs);

  // Document frequencies within these documents decide the head/tail split: head = terms of
  // df >= cut (dense tensor-core columns), tail = the other terms with df >= 2 (a term in one
  // document joins no pair). The split is computed on the device; only its totals come back.
  const int64_t n_tblocks = ((int64_t)V + 1023) / 1024;
  int32_t* df = (int32_t*)ws_get(ctx, "cos.df", sizeof(int32_t) * V, &st);
  unsigned long long* d_norm = (unsigned long long*)ws_get(ctx, "cos.norm", sizeof(unsigned long long) * N, &st);
  int32_t* d_colmap = (int32_t*)ws_get(ctx, "cos.colmap", sizeof(int32_t) * V, &st);
  int64_t* d_tstart = (int64_t*)ws_get(ctx, "cos.tstart", sizeof(int64_t) * V, &st);
  int32_t* d_tfill = (int32_t*)ws_get(ctx, "cos.tfill", sizeof(int32_t) * V, &st);
  int64_t* d_cstart = (int64_t*)ws_get(ctx, "cos.cstart", sizeof(int64_t) * ((size_t)V + 1), &st);
  int32_t* d_rank_terms = (int32_t*)ws_get(ctx, "cos.rterms", sizeof(int32_t) * (size_t)V, &st);
  long long* d_tpart = (long long*)ws_get(ctx, "cos.tpart", sizeof(long long) * 8 * (size_t)n_tblocks, &st);
  long long* d_tsum = (long long*)ws_get(ctx, "cos.tsum", sizeof(long long) * 8, &st);
  int32_t* d_rcnt = (int32_t*)ws_get(ctx, "cos.rcnt", sizeof(int32_t) * (size_t)N, &st);
  float* d_rw = (float*)ws_get(ctx, "cos.rw", sizeof(float) * (size_t)std::max<int64_t>(d.n_tokens, 1), &st);
  if (st != MRC_OK) return st;
  cudaMemsetAsync(df, 0, sizeof(int32_t) * V, ctx->stream);
  const float* wid = index->params.weighting == MRC_WEIGHT_TFIDF ? index->idf : nullptr;
  attach_bag(ctx, &d);
  d.bag_write = 1;
  cudaError_t e = launch_df_norm(ctx, d, df, V, wid, d_norm);
  d.bag_write = 0;
  d.bag_read = 1;
  d.lists_ready = 1;
  if (e != cudaSuccess) return cuda_fail(ctx, e, "df pass");
  long long* h_tsum = (long long*)((char*)ctx->pinned + 1024);
  // runs the split for `cut` and reads its totals (one synchronisation, with the error word)
  auto split = [&](int32_t cut) -> mrc_status {
    cudaError_t se = cudaMemsetAsync(d_cstart, 0, sizeof(int64_t), ctx->stream);
    if (se == cudaSuccess)
      se = launch_cosine_terms(ctx, df, V, cut, d_tpart, d_tsum, d_colmap, d_tstart, d_cstart, d_rank_terms);
    if (se == cudaSuccess) se = cudaMemcpyAsync(h_tsum, d_tsum, sizeof(long long) * 6, cudaMemcpyDeviceToHost, ctx->stream);
    if (se != cudaSuccess) return cuda_fail(ctx, se, "head/tail split");
    return check_err_word(ctx, d_err);  // synchronises the stream
  };
  DenseOut o{};
  o.idf = wid;
  o.colmap = d_colmap;
  o.tail_start = d_tstart;
  o.tail_fill = d_tfill;
  o.row_cnt = d_rcnt;
  o.norm = d_norm;
  o.row_w = d_rw;
  GemmArgs g{};
  g.fmt = OP_F16;
  g.na = g.nb = N;
  g.triangle = 1;
  g.out_scale = 1.0f;
  g.err = async ? ctx->async_err : d_err;
  // The head GEMM's error against the exact sum of its columns is at most: fp16 rounding of
  // both operands, 2^-10 sum|a_c b_c| <= 2^-10 (each row's columns have norm <= 1: unit head
  // weights, and bucket norms whose squares add up to the tail's); FP32 accumulation over kd
  // terms, kd 2^-23; 2^-12 (the fp16 store of the tail-walk path); plus 1e-4 for subnormal
  // operands and the FP32 addition of the tail.
  auto delta_of = [](int32_t kd) {
    return (float)(std::ldexp(1.0, -10) + std::ldexp(1.0, -12) + (double)kd * std::ldexp(1.0, -23) + 1e-4);
  };

  // Bound-pruned path. Hash the tail terms into kTailBuckets buckets; by Cauchy-Schwarz in each
  // bucket a pair's tail dot product is at most sum_s |t_i^s| |t_j^s|, the dot product of the
  // two documents' bucket-norm vectors. Those norms ride in the head operand's last columns,
  // so the head GEMM computes head score + bound; a pair below tau - delta' there is below tau,
  // and the GEMM emits only the other pairs as candidates, each then scored exactly
  // (k_cosine_verify). delta' adds to delta the rounding of the tail sum (at most 2^-31 per
  // shared term, under 3.1e-5 for 65,536 terms). The bucket columns make a looser head cheap:
  // head = df >= max(32, N / 8).
  {
    const int32_t cut_b = (int32_t)std::min<int64_t>(std::max<int64_t>(32, N / 8), INT32_MAX);
    // The head has at most n_tokens / cut terms (each adds >= cut to sum df <= n_tokens). With
    // room for that many columns the split's totals never need to reach the host: the head
    // width is read on the device (row stride kd_max, K blocks from k_cosine_dims). Per-kernel
    // timing takes the synchronous split, so that the flop counts are exact.
    const int32_t kd_h_max =
        round_up((int32_t)std::min<int64_t>((int64_t)V, std::max<int64_t>(d.n_tokens, 0) / cut_b), 64);
    const bool dims_dev = !ctx->timing && 4.0 * (double)N * (double)(kd_h_max + kTailBuckets) <= 8e9;
    int32_t kd_h = 0, kd = 0;
    int32_t* d_dims = (int32_t*)ws_get(ctx, "cos.dims", sizeof(int32_t) * 2, &st);
    if (st != MRC_OK) return st;
    if (dims_dev) {
      e = cudaMemsetAsync(d_cstart, 0, sizeof(int64_t), ctx->stream);
      if (e == cudaSuccess)
        e = launch_cosine_terms(ctx, df, V, cut_b, d_tpart, d_tsum, d_colmap, d_tstart, d_cstart, d_rank_terms);
      if (e == cudaSuccess) e = launch_cosine_dims(ctx, d_tsum, kd_h_max, d_dims);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "head/tail split");
      kd_h = kd_h_max;  // an upper bound on the host
      kd = kd_h_max + kTailBuckets;
    } else {
      if ((st = split(cut_b)) != MRC_OK) return st;
      kd_h = round_up((int32_t)h_tsum[0], 64);  // may be 0
      kd = kd_h + kTailBuckets;
    }
    const int64_t cand_cap = std::max<int64_t>(4 * capacity, 1 << 22);
    void* d_hhi = ws_get(ctx, "cos.hhi", 2 * (size_t)N * kd, &st);
    void* d_hlo = ws_get(ctx, "cos.hlo", 2 * (size_t)N * kd, &st);
    int32_t* d_rterm = (int32_t*)ws_get(ctx, "cos.rterm", sizeof(int32_t) * (size_t)std::max<int64_t>(d.n_tokens, 1), &st);
    mrc_pair* d_cand = (mrc_pair*)ws_get(ctx, "cos.cand", sizeof(mrc_pair) * (size_t)cand_cap, &st);
    int32_t* d_clong = (int32_t*)ws_get(ctx, "cos.clong", sizeof(int32_t) * (size_t)cand_cap, &st);
    unsigned long long* d_nlong = (unsigned long long*)ws_get(ctx, "cos.nlong", sizeof(unsigned long long), &st);
    unsigned long long* d_ccount = (unsigned long long*)ws_get(ctx, "cos.ccount", sizeof(unsigned long long), &st);
    if (st != MRC_OK) return st;
    if (dims_dev) {
      e = launch_zero_head(ctx, d_hhi, d_hlo, N, kd, d_dims);
      // documents the ingest passes rejected (bad offsets or lengths) keep no tail terms
      if (e == cudaSuccess) e = cudaMemsetAsync(d_rcnt, 0, sizeof(int32_t) * (size_t)N, ctx->stream);
    } else {
      e = cudaMemsetAsync(d_hhi, 0, 2 * (size_t)N * kd, ctx->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(d_hlo, 0, 2 * (size_t)N * kd, ctx->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_ccount, 0, sizeof(unsigned long long), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cosine set-up");
    o.kd = kd;
    o.kd_h = kd_h;
    o.kd_h_dev = dims_dev ? d_dims : nullptr;
    o.head_hi = d_hhi;
    o.head_lo = d_hlo;
    o.postings = 0;
    o.row_term = d_rterm;
    e = launch_densify(ctx, d, V, index->tinfo, o);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "densify");
    g.a_hi = g.b_hi = d_hhi;
    g.kbytes = kd * 2;
    g.kblocks_dev = dims_dev ? d_dims + 1 : nullptr;
    g.thresh = tau - (delta_of(kd) + 4e-5f);  // kd: the actual width, or its upper bound
    g.pairs = d_cand;
    g.count = d_ccount;
    g.capacity = cand_cap;
    g.name = "gemm_f16_bound";
    e = launch_gemm_compare(ctx, g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "head GEMM");
    e = launch_cosine_verify(ctx, d_cand, d_ccount, cand_cap, d_hhi, d_hlo, kd, kd_h, dims_dev ? d_dims : nullptr,
                             d.offsets, d_rcnt, d_rterm, d_rw, tau, dst, d_count, capacity, d_clong, d_nlong,
                             async ? ctx->async_err : d_err);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "candidate verification");
    if (async) return MRC_OK;  // a candidate overflow is reported by mrc_ctx_sync
    bool overflow = false;
    st = finish_pairs(ctx, pairs, dst, d_count, capacity, n_pairs, d_err, d_ccount, cand_cap, &overflow);
    if (!overflow) return st;
    // too many candidates for the buffer: the exhaustive tail walk below
    e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int32_t), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cosine set-up");
  }

  // Tail-walk path: head = df >= max(32, N / 48), the break-even of a tensor-core column
  // against sparse products (capped so that tail lists stay <= 4096 postings); the head stored
  // as fp16 scores, the tail postings of each term ordered by document, each row's tail
  // products summed over the postings after it, candidates against tau - delta, exact head
  // for each candidate.
  if ((st = split((int32_t)std::min<int64_t>(std::max<int64_t>(32, N / 48), 4097))) != MRC_OK) return st;
  const int64_t n_head = h_tsum[0], n_post = h_tsum[2];
  const int32_t n_tail = (int32_t)h_tsum[1], n_small = (int32_t)h_tsum[3], max_m = (int32_t)h_tsum[4];
  const double tail_work = (double)h_tsum[5];
  const int32_t kd = std::max<int32_t>(64, round_up((int32_t)n_head, 64));
  const int64_t ldh = (N + 7) / 8 * 8;
  if (n_post >= (1ll << 31) - 64)
    return fail(ctx, MRC_ERR_UNSUPPORTED, "cosine_allpairs: more than 2^31 tail postings");
  if ((double)N * (double)ldh * 2.0 > 64e9)
    return fail(ctx, MRC_ERR_UNSUPPORTED, "cosine_allpairs: more documents than the 64 GB score buffer allows");
  void* d_hhi = ws_get(ctx, "cos.hhi", 2 * (size_t)N * kd, &st);
  void* d_hlo = ws_get(ctx, "cos.hlo", 2 * (size_t)N * kd, &st);
  int4* d_post = (int4*)ws_get(ctx, "cos.post", sizeof(int4) * (size_t)std::max<int64_t>(n_post, 1), &st);
  void* d_spost = ws_get(ctx, "cos.spost", 8 * (size_t)std::max<int64_t>(n_post, 1), &st);
  void* d_rwalk = ws_get(ctx, "cos.rwalk", 8 * (size_t)std::max<int64_t>(d.n_tokens, 1), &st);
  void* d_H = ws_get(ctx, "cos.H16", 2 * (size_t)N * ldh, &st);
  unsigned long long* d_next = (unsigned long long*)ws_get(ctx, "cos.next", sizeof(unsigned long long), &st);
  if (st != MRC_OK) return st;
  e = cudaMemsetAsync(d_tfill, 0, sizeof(int32_t) * V, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_hhi, 0, 2 * (size_t)N * kd, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_hlo, 0, 2 * (size_t)N * kd, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cosine set-up");
  o.kd = kd;
  o.kd_h = kd;
  o.kd_h_dev = nullptr;
  o.head_hi = d_hhi;
  o.head_lo = d_hlo;
  o.postings = 1;
  o.post = d_post;
  o.row_term = nullptr;
  e = launch_densify(ctx, d, V, index->tinfo, o);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "densify");
  e = launch_rank_postings(ctx, d_cstart, d_rank_terms, n_small, d_rank_terms + n_small, n_tail - n_small, max_m, d_post,
                           d.offsets, d_spost, d_rwalk);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "sorting postings");
  g.a_hi = g.b_hi = d_hhi;
  g.kbytes = kd * 2;
  g.kblocks_dev = nullptr;
  g.store16 = d_H;
  g.ld = ldh;
  g.thresh = 0.f;
  g.pairs = nullptr;
  g.count = nullptr;
  g.capacity = 0;
  g.name = nullptr;
  e = launch_gemm_compare(ctx, g);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "head GEMM");
  e = launch_cosine_tail(ctx, N, d_H, ldh, d.offsets, d_rcnt, d_rwalk, d_rw, d_spost, n_post, d_hhi, d_hlo, kd,
                         tau, delta_of(kd), dst, d_count, capacity, tail_work, d_next);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "tail pass");
  return finish_pairs(ctx, pairs, dst, d_count, capacity, n_pairs, d_err);
}

// simhash_match, or with d_total its stream-ordered form (see match_impl).
static mrc_status simhash_impl(mrc_ctx* ctx, const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb,
                        int32_t hamming_max, mrc_pair* pairs, int64_t capacity, int64_t* n_pairs,
                        unsigned long long* d_total) {
  if (!ctx) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  if (na < 0 || (b && nb < 0) || capacity < 0 || (na > 0 && !a))
    return fail(ctx, MRC_ERR_INVALID, "simhash_match: bad sizes or NULL input");
  if (na >= (1ll << 31) || nb >= (1ll << 31)) return fail(ctx, MRC_ERR_UNSUPPORTED, "more than 2^31 fingerprints");
  if (n_pairs) *n_pairs = 0;
  mrc_status st = MRC_OK;
  const bool async = d_total != nullptr;
  if (async && ((capacity > 0 && (!pairs || !is_device_ptr(pairs))) || !is_device_ptr(d_total)))
    return fail(ctx, MRC_ERR_INVALID, "stream-ordered calls take device pairs and a device pair count");
  unsigned long long* d_count =
      async ? d_total : (unsigned long long*)ws_get(ctx, "sh.count", sizeof(unsigned long long), &st);
  mrc_pair* dst = pair_dest(ctx, pairs, capacity, &st);
  if (st != MRC_OK) return st;
  cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), ctx->stream);
  const uint64_t* da = (const uint64_t*)stage_in(ctx, "sh.a", a, sizeof(uint64_t) * (size_t)na, &st);
  const uint64_t* db = b ? (const uint64_t*)stage_in(ctx, "sh.b", b, sizeof(uint64_t) * (size_t)nb, &st) : nullptr;
  if (st != MRC_OK) return st;
  if (na > 0 && (!b || nb > 0)) {
    cudaError_t e = launch_simhash_match(ctx, da, na, db, b ? nb : 0, hamming_max, dst, d_count, capacity);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "simhash match");
  }
  if (async) return MRC_OK;
  return finish_pairs(ctx, pairs, dst, d_count, capacity, n_pairs);
}

mrc_status mrc_match(mrc_ctx* ctx, const mrc_index* index, const float* query_sig, int64_t nq, float tau,
                     mrc_pair* pairs, int64_t capacity, int64_t* n_pairs) {
  return match_impl(ctx, index, query_sig, nq, tau, pairs, capacity, n_pairs, nullptr);
}

mrc_status mrc_match_async(mrc_ctx* ctx, const mrc_index* index, const float* query_sig, int64_t nq, float tau,
                           mrc_pair* pairs, int64_t capacity, int64_t* d_n_pairs) {
  if (!d_n_pairs) return ctx ? fail(ctx, MRC_ERR_INVALID, "d_n_pairs is NULL") : MRC_ERR_INVALID;
  return match_impl(ctx, index, query_sig, nq, tau, pairs, capacity, nullptr, (unsigned long long*)d_n_pairs);
}

mrc_status cosine_allpairs(mrc_ctx* ctx, const mrc_index* index, const mrc_docs* docs, float tau, mrc_pair* pairs,
                           int64_t capacity, int64_t* n_pairs) {
  return cosine_impl(ctx, index, docs, tau, pairs, capacity, n_pairs, nullptr);
}

mrc_status cosine_allpairs_async(mrc_ctx* ctx, const mrc_index* index, const mrc_docs* docs, float tau,
                                 mrc_pair* pairs, int64_t capacity, int64_t* d_n_pairs) {
  if (!d_n_pairs) return ctx ? fail(ctx, MRC_ERR_INVALID, "d_n_pairs is NULL") : MRC_ERR_INVALID;
  return cosine_impl(ctx, index, docs, tau, pairs, capacity, nullptr, (unsigned long long*)d_n_pairs);
}

mrc_status simhash_match(mrc_ctx* ctx, const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb,
                         int32_t hamming_max, mrc_pair* pairs, int64_t capacity, int64_t* n_pairs) {
  return simhash_impl(ctx, a, na, b, nb, hamming_max, pairs, capacity, n_pairs, nullptr);
}

mrc_status simhash_match_async(mrc_ctx* ctx, const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb,
                               int32_t hamming_max, mrc_pair* pairs, int64_t capacity, int64_t* d_n_pairs) {
  if (!d_n_pairs) return ctx ? fail(ctx, MRC_ERR_INVALID, "d_n_pairs is NULL") : MRC_ERR_INVALID;
  return simhash_impl(ctx, a, na, b, nb, hamming_max, pairs, capacity, nullptr, (unsigned long long*)d_n_pairs);
}

mrc_status mrc_simhash_index_build(mrc_ctx* ctx, const uint64_t* fps, int64_t n, int32_t hamming_max,
                                   mrc_simhash_index** out) {
  if (!ctx || !out) return MRC_ERR_INVALID;
  *out = nullptr;
  Scope scope(ctx, __func__);
  if (n < 0 || (n > 0 && !fps)) return fail(ctx, MRC_ERR_INVALID, "mrc_simhash_index_build: bad size or NULL input");
  if (n >= (1ll << 31) - 1) return fail(ctx, MRC_ERR_UNSUPPORTED, "more than 2^31 - 2 fingerprints");
  if (hamming_max < 0 || hamming_max > 15) return fail(ctx, MRC_ERR_INVALID, "hamming_max must be in [0, 15]");
  mrc_status st = MRC_OK;
  const SimhashLayout L = simhash_layout(hamming_max);
  const uint64_t* d_fps = (const uint64_t*)stage_in(ctx, "shx.in", fps, sizeof(uint64_t) * (size_t)n, &st);
  int32_t* cnt = (int32_t*)ws_get(ctx, "shx.cnt", sizeof(int32_t) * (size_t)L.off_words, &st);
  int32_t* cursor = (int32_t*)ws_get(ctx, "shx.cursor", sizeof(int32_t) * (size_t)L.off_words, &st);
  if (st != MRC_OK) return st;
  mrc_simhash_index* x = new mrc_simhash_index();
  x->device = ctx->device;
  x->stream = ctx->stream;
  x->n = n;
  x->hamming_max = hamming_max;
  x->layout = L;
  const size_t nn = (size_t)std::max<int64_t>(n, 1) * (size_t)L.blocks;
  const size_t b_fp = (8 * nn + 255) / 256 * 256, b_id = (4 * nn + 255) / 256 * 256;
  const size_t b_own = (8 * (size_t)std::max<int64_t>(n, 1) + 255) / 256 * 256;
  char* b = nullptr;
  if (cudaMallocAsync((void**)&b, b_fp + b_id + b_own + sizeof(int32_t) * (size_t)L.off_words, ctx->stream) !=
      cudaSuccess) {
    cudaGetLastError();
    delete x;
    return fail(ctx, MRC_ERR_OOM, "device allocation failed: fingerprint index");
  }
  x->block = b;
  x->fp = (uint64_t*)b;
  x->id = (int32_t*)(b + b_fp);
  x->own = (uint64_t*)(b + b_fp + b_id);
  x->off = (int32_t*)(b + b_fp + b_id + b_own);
  cudaError_t e = n > 0 ? cudaMemcpyAsync(x->own, d_fps, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToDevice,
                                          ctx->stream)
                        : cudaSuccess;
  if (e == cudaSuccess) e = launch_simhash_index_build(ctx, d_fps, n, L, cnt, cursor, x->off, x->fp, x->id);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // the staging slots may be reused after this
  if (e != cudaSuccess) {
    cudaFreeAsync(x->block, ctx->stream);
    delete x;
    return cuda_fail(ctx, e, "fingerprint index build");
  }
  *out = x;
  return MRC_OK;
}

mrc_status mrc_simhash_index_match(mrc_ctx* ctx, const mrc_simhash_index* index, const uint64_t* queries, int64_t nq,
                                   int32_t hamming_max, mrc_pair* pairs, int64_t capacity, int64_t* n_pairs) {
  if (!ctx) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  if (!index || (queries && nq < 0) || capacity < 0 || (!queries && nq != 0))
    return fail(ctx, MRC_ERR_INVALID, "mrc_simhash_index_match: bad sizes or NULL index");
  if (nq >= (1ll << 31)) return fail(ctx, MRC_ERR_UNSUPPORTED, "more than 2^31 queries");
  if (hamming_max < 0 || hamming_max > index->hamming_max)
    return fail(ctx, MRC_ERR_INVALID, "hamming_max above the distance the index was built for");
  if (n_pairs) *n_pairs = 0;
  mrc_status st = MRC_OK;
  unsigned long long* d_count = (unsigned long long*)ws_get(ctx, "shx.count", sizeof(unsigned long long), &st);
  mrc_pair* dst = pair_dest(ctx, pairs, capacity, &st);
  if (st != MRC_OK) return st;
  cudaError_t e = cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "clearing the pair count");
  const bool all = queries == nullptr;  // all pairs: the index's own fingerprints are the queries
  const uint64_t* dq = index->own;
  const int64_t m = all ? index->n : nq;
  if (!all) {
    dq = (const uint64_t*)stage_in(ctx, "shx.q", queries, sizeof(uint64_t) * (size_t)nq, &st);
    if (st != MRC_OK) return st;
  }
  e = launch_simhash_index_probe(ctx, dq, m, all, hamming_max, index->layout, index->n, index->fp,
                                             index->id, index->off, dst, d_count, capacity);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "fingerprint index probe");
  return finish_pairs(ctx, pairs, dst, d_count, capacity, n_pairs);
}

void mrc_simhash_index_free(mrc_simhash_index* x) {
  if (!x) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != x->device) cudaSetDevice(x->device);
  if (x->block) cudaFreeAsync(x->block, x->stream);
  if (cur >= 0 && cur != x->device) cudaSetDevice(cur);
  delete x;
}

mrc_status mrc_ctx_sync(mrc_ctx* ctx) {
  if (!ctx) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  int32_t* h = (int32_t*)((char*)ctx->pinned + 256);
  cudaError_t e = cudaMemcpyAsync(h, ctx->async_err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->async_err, 0, sizeof(int32_t), ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "synchronising the context's stream");
  return err_status(ctx, *h);
}

mrc_status mrc_index_get_info(const mrc_index* x, mrc_index_info* info) {
  if (!x || !info) return MRC_ERR_INVALID;
  std::memset(info, 0, sizeof(*info));
  info->n_docs = x->n_docs;
  info->vocab = x->vocab;
  info->k = x->k;
  info->L_used = x->L_used;
  info->precision = x->params.precision;
  info->weighting = x->params.weighting;
  info->kp = x->kp;
  return MRC_OK;
}

mrc_status mrc_index_export(mrc_ctx* ctx, const mrc_index* x, float* sig, uint64_t* simhash, int32_t* df, float* idf,
                            int32_t* part, double* rnorm) {
  if (!ctx || !x) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  wait_for_index(ctx, x);
  const size_t n = (size_t)x->n_docs;
  auto cp = [&](void* dst, const void* src, size_t bytes) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream);
  };
  cudaError_t e = cudaSuccess;
  if (sig) e = cp(sig, x->sig, sizeof(float) * n * x->k);
  if (e == cudaSuccess && simhash) e = cp(simhash, x->simhash, sizeof(uint64_t) * n);
  if (e == cudaSuccess && df) e = cp(df, x->df, sizeof(int32_t) * x->vocab);
  if (e == cudaSuccess && idf) e = cp(idf, x->idf, sizeof(float) * x->vocab);
  // device outputs are stream-ordered like every call's; host outputs are complete on return
  const bool host_out = (sig && !is_device_ptr(sig)) || (simhash && !is_device_ptr(simhash)) ||
                        (df && !is_device_ptr(df)) || (idf && !is_device_ptr(idf));
  if (e == cudaSuccess && host_out) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "index export");
  if (part) {
    std::vector<int32_t> hp;
    const mrc_status st = read_partition(ctx, x, &hp);
    if (st != MRC_OK) return st;
    std::memcpy(part, hp.data(), sizeof(int32_t) * x->vocab);
  }
  if (rnorm) std::memcpy(rnorm, x->h_rnorm.data(), sizeof(double) * x->k);
  return MRC_OK;
}

void mrc_index_free(mrc_index* x) {
  if (!x) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != x->device) cudaSetDevice(x->device);
  free_index_arrays(x);
  if (x->ready) cudaEventDestroy(x->ready);
  if (x->tables) cudaEventDestroy(x->tables);
  if (cur >= 0 && cur != x->device) cudaSetDevice(cur);
  delete x;
}

// ---- persistence -------------------------------------------------------------------------
static const char kMagic[8] = {'M', 'R', 'C', 'I', 'D', 'X', '0', '1'};

mrc_status mrc_index_save(mrc_ctx* ctx, const mrc_index* x, const char* path) {
  if (!ctx || !x || !path) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  // the copies below are plain ones: the index must be complete first
  wait_for_index(ctx, x);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "waiting for the index");
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, MRC_ERR_INVALID, std::string("cannot open ") + path);
  const size_t n = (size_t)x->n_docs;
  std::vector<float> sig(n * x->k), unit(n * x->k);
  std::vector<uint64_t> sh(n);
  cudaError_t e = cudaMemcpy(sig.data(), x->sig, sizeof(float) * sig.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(unit.data(), x->sig_unit, sizeof(float) * unit.size(), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(sh.data(), x->simhash, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    std::fclose(f);
    return cuda_fail(ctx, e, "index save");
  }
  std::vector<int32_t> hdf(x->vocab), hpart;
  std::vector<float> hidf(x->vocab);
  if (read_partition(ctx, x, &hpart) != MRC_OK) {
    std::fclose(f);
    return MRC_ERR_CUDA;
  }
  if (cudaMemcpy(hdf.data(), x->df, sizeof(int32_t) * x->vocab, cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hidf.data(), x->idf, sizeof(float) * x->vocab, cudaMemcpyDeviceToHost) != cudaSuccess) {
    std::fclose(f);
    return cuda_fail(ctx, cudaGetLastError(), "index save");
  }
  // version 2 appends the precision form's E4M3 operand rows and their norms (they come from
  // the bfloat16-weight signatures, which the file does not hold otherwise)
  std::vector<uint8_t> op8(x->op_e4m3 ? n * (size_t)x->kp8 : 0);
  std::vector<float> qn(x->op_e4m3 ? n : 0);
  if (x->op_e4m3 && (cudaMemcpy(op8.data(), x->op_e4m3, op8.size(), cudaMemcpyDeviceToHost) != cudaSuccess ||
                     cudaMemcpy(qn.data(), x->qnorm, sizeof(float) * n, cudaMemcpyDeviceToHost) != cudaSuccess)) {
    std::fclose(f);
    return cuda_fail(ctx, cudaGetLastError(), "index save");
  }
  const int32_t version = 2;
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8;
  ok = ok && std::fwrite(&version, sizeof(version), 1, f) == 1;
  ok = ok && std::fwrite(&x->params, sizeof(mrc_params), 1, f) == 1;
  ok = ok && std::fwrite(&x->n_docs, sizeof(int64_t), 1, f) == 1;
  ok = ok && std::fwrite(&x->vocab, sizeof(int32_t), 1, f) == 1;
  ok = ok && std::fwrite(&x->L_used, sizeof(int64_t), 1, f) == 1;
  ok = ok && std::fwrite(hdf.data(), sizeof(int32_t), x->vocab, f) == (size_t)x->vocab;
  ok = ok && std::fwrite(hidf.data(), sizeof(float), x->vocab, f) == (size_t)x->vocab;
  ok = ok && std::fwrite(hpart.data(), sizeof(int32_t), x->vocab, f) == (size_t)x->vocab;
  ok = ok && std::fwrite(sig.data(), sizeof(float), sig.size(), f) == sig.size();
  ok = ok && std::fwrite(unit.data(), sizeof(float), unit.size(), f) == unit.size();
  ok = ok && std::fwrite(sh.data(), sizeof(uint64_t), n, f) == n;
  ok = ok && std::fwrite(op8.data(), 1, op8.size(), f) == op8.size();
  ok = ok && std::fwrite(qn.data(), sizeof(float), qn.size(), f) == qn.size();
  std::fclose(f);
  if (!ok) return fail(ctx, MRC_ERR_INVALID, std::string("write failed: ") + path);
  return MRC_OK;
}

mrc_status mrc_index_load(mrc_ctx* ctx, const char* path, mrc_index** out) {
  if (!ctx || !path || !out) return MRC_ERR_INVALID;
  *out = nullptr;
  Scope scope(ctx, __func__);
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, MRC_ERR_INVALID, std::string("cannot open ") + path);
  char magic[8];
  int32_t version = 0;
  mrc_index* x = new mrc_index();
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0;
  ok = ok && std::fread(&version, sizeof(version), 1, f) == 1 && (version == 1 || version == 2);
  ok = ok && std::fread(&x->params, sizeof(mrc_params), 1, f) == 1;
  ok = ok && std::fread(&x->n_docs, sizeof(int64_t), 1, f) == 1;
  ok = ok && std::fread(&x->vocab, sizeof(int32_t), 1, f) == 1;
  ok = ok && std::fread(&x->L_used, sizeof(int64_t), 1, f) == 1;
  std::string why;
  ok = ok && valid_params(&x->params, &why) && x->vocab > 0 && x->n_docs > 0;
  std::vector<float> sig, unit, hidf;
  std::vector<int32_t> hdf, hpart;
  std::vector<uint64_t> sh;
  std::vector<uint8_t> op8;
  std::vector<float> qn;
  if (ok) {
    x->k = x->params.k;
    x->kp = padded_kp(x->k);
    x->kp8 = padded_kp8(x->k);
    x->device = ctx->device;
    x->stream = ctx->stream;
    const size_t n = (size_t)x->n_docs;
    hdf.resize(x->vocab);
    hidf.resize(x->vocab);
    hpart.resize(x->vocab);
    sig.resize(n * x->k);
    unit.resize(n * x->k);
    sh.resize(n);
    ok = std::fread(hdf.data(), sizeof(int32_t), x->vocab, f) == (size_t)x->vocab;
    ok = ok && std::fread(hidf.data(), sizeof(float), x->vocab, f) == (size_t)x->vocab;
    ok = ok && std::fread(hpart.data(), sizeof(int32_t), x->vocab, f) == (size_t)x->vocab;
    ok = ok && std::fread(sig.data(), sizeof(float), sig.size(), f) == sig.size();
    ok = ok && std::fread(unit.data(), sizeof(float), unit.size(), f) == unit.size();
    ok = ok && std::fread(sh.data(), sizeof(uint64_t), n, f) == n;
    if (ok && version >= 2 && x->params.precision == MRC_PREC_BF16_FP8) {
      op8.resize(n * (size_t)x->kp8);
      qn.resize(n);
      ok = std::fread(op8.data(), 1, op8.size(), f) == op8.size();
      ok = ok && std::fread(qn.data(), sizeof(float), n, f) == n;
    }
  }
  std::fclose(f);
  if (!ok) {
    delete x;
    return fail(ctx, MRC_ERR_INVALID, std::string("not a valid index file: ") + path);
  }
  mrc_status st;
  auto bail = [&](mrc_status s) {
    cudaStreamSynchronize(ctx->stream);
    free_index_arrays(x);
    delete x;
    return s;
  };
  if ((st = alloc_index_arrays(ctx, x)) != MRC_OK) return bail(st);
  const size_t n = (size_t)x->n_docs;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);  // stream-ordered allocations before plain copies
  if (e == cudaSuccess) e = cudaMemcpy(x->df, hdf.data(), sizeof(int32_t) * x->vocab, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(x->idf, hidf.data(), sizeof(float) * x->vocab, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(x->sig, sig.data(), sizeof(float) * sig.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(x->sig_unit, unit.data(), sizeof(float) * unit.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(x->simhash, sh.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "index load"));
  char* stage = (char*)host_ws(ctx, 4 * (size_t)x->vocab + 8 * (size_t)x->k + 64, &st);
  if (!stage) return bail(st);
  x->h_rnorm.assign(x->k, 0.0);
  for (int32_t t = 0; t < x->vocab; ++t) {
    const int32_t q = hpart[t];
    if (q >= x->k) return bail(fail(ctx, MRC_ERR_INVALID, std::string("not a valid index file: ") + path));
    if (q >= 0) {
      const double r = reference_weight(x->params, hidf.data(), t);
      x->h_rnorm[q] += r * r;
    }
  }
  std::memcpy(stage, hpart.data(), sizeof(int32_t) * x->vocab);
  if ((st = upload_references(ctx, x, (int32_t*)stage, (float*)(stage + 4 * (size_t)x->vocab), hidf.data())) != MRC_OK)
    return bail(st);
  // compare operands are re-packed from the unit signatures
  if (x->op_hi) cudaMemsetAsync(x->op_hi, 0, 2 * n * x->kp, ctx->stream);
  if (x->op_lo) cudaMemsetAsync(x->op_lo, 0, 2 * n * x->kp, ctx->stream);
  if (x->op_e4m3) cudaMemsetAsync(x->op_e4m3, 0, n * x->kp8, ctx->stream);
  if (!op8.empty()) {  // the stored E4M3 rows (version 2), else re-packed from the unit signatures
    e = cudaMemcpyAsync(x->op_e4m3, op8.data(), op8.size(), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(x->qnorm, qn.data(), sizeof(float) * n, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess && x->op_hi)
      e = launch_pack(ctx, x->sig_unit, x->n_docs, x->k, 0, x->op_hi, x->op_lo, nullptr, nullptr, nullptr, x->kp, 0);
  } else {
    e = launch_pack(ctx, x->sig_unit, x->n_docs, x->k, 0, x->op_hi, x->op_lo, x->op_e4m3, x->qnorm, nullptr,
                    x->op_hi ? x->kp : 0, x->op_e4m3 ? x->kp8 : 0);
  }
  if (e == cudaSuccess && x->qnorm_min) e = launch_block_min(ctx, x->qnorm, x->n_docs, x->qnorm_min);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return bail(cuda_fail(ctx, e, "index load packing"));
  mark_index_tables(ctx, x);
  mark_index_ready(ctx, x);
  *out = x;
  return MRC_OK;
}

mrc_status mrc_ctx_set_wait_limit(mrc_ctx* ctx, int64_t ns) {
  if (!ctx) return MRC_ERR_INVALID;
  if (ns < 1 || ns > 600000000000ll) return fail(ctx, MRC_ERR_INVALID, "wait limit outside [1 ns, 600 s]");
  ctx->wait_limit_ns = (uint64_t)ns;
  return MRC_OK;
}

mrc_status mrc_measure_popc_rate(mrc_ctx* ctx, double* popc_per_s) {
  if (!ctx || !popc_per_s) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  const cudaError_t e = measure_popc_rate(ctx, popc_per_s);
  return e == cudaSuccess ? MRC_OK : cuda_fail(ctx, e, "POPC rate probe");
}

mrc_status mrc_measure_smem_atomic_rate(mrc_ctx* ctx, double* atomics_per_s) {
  if (!ctx || !atomics_per_s) return MRC_ERR_INVALID;
  Scope scope(ctx, __func__);
  const cudaError_t e = measure_smem_atomic_rate(ctx, atomics_per_s);
  return e == cudaSuccess ? MRC_OK : cuda_fail(ctx, e, "shared-memory atomic rate probe");
}

mrc_status mrc_ctx_set_rescoring(mrc_ctx* ctx, int32_t on) {
  if (!ctx) return MRC_ERR_INVALID;
  ctx->rescore = on != 0;
  return MRC_OK;
}

mrc_status mrc_ctx_set_test_stall(mrc_ctx* ctx, int32_t on) {
  if (!ctx) return MRC_ERR_INVALID;
  ctx->test_stall = on != 0;
  return MRC_OK;
}

// ---- timing --------------------------------------------------------------------------------
mrc_status mrc_ctx_set_timing(mrc_ctx* ctx, int32_t on) {
  if (!ctx) return MRC_ERR_INVALID;
  ctx->timing = on != 0;
  return MRC_OK;
}

int32_t mrc_ctx_kernel_stat(mrc_ctx* ctx, int32_t slot, char* name, int64_t* launches, double* total_ms,
                            double* bytes, double* flops) {
  if (!ctx) return -1;
  collect_timings(ctx);
  const int32_t count = (int32_t)ctx->stats.size();
  if (slot < 0) return count;
  if (slot >= count) return -1;
  const auto& s = ctx->stats[slot];
  if (name) {
    std::strncpy(name, s.first.c_str(), 63);
    name[63] = 0;
  }
  if (launches) *launches = s.second.launches;
  if (total_ms) *total_ms = s.second.ms;
  if (bytes) *bytes = s.second.bytes;
  if (flops) *flops = s.second.flops;
  return count;
}

void mrc_ctx_reset_stats(mrc_ctx* ctx) {
  if (!ctx) return;
  collect_timings(ctx);
  ctx->stats.clear();
}

}  // extern "C"
