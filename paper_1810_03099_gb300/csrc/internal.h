// internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "mrc.h"

// A named NVTX range over one C-ABI call, so that a timeline profiler shows the library's calls
// around their kernels. Without a profiler attached the push and pop return at once.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

namespace mrc {

// Per-document term information looked up while streaming a document:
// x = idf(t) as float (1.0 under count weighting), y = partition of t or -1.
// For the exact-cosine densify pass y is the column code instead (see ingest.cu).
struct TermInfo {
  float idf;
  int32_t code;
};

// Operand formats of the tensor-core compare.
enum OperandFormat : int32_t { OP_SPLIT16 = 0, OP_F16 = 1, OP_E4M3 = 2 };

// Scale of the low half of the fp16 hi/lo split: lo = fp16((x - hi) * 2^12).
constexpr float kSplitLoScale = 4096.0f;
// Global scale of unit signatures stored as E4M3 (max element 1.0 -> 256 <= 448).
constexpr float kE4M3Scale = 256.0f;

struct KernelStat {
  int64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
  double flops = 0.0;
};

struct PendingTiming {
  std::string name;
  cudaEvent_t start, stop;
  double bytes, flops;
};

struct Buffer {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Blocks of the fingerprint index: block t covers bits [shift[t], shift[t] + width[t]); its
// bucket offsets start at off_base[t] in the offsets array (2^width[t] + 1 entries each).
struct SimhashLayout {
  int32_t blocks;
  int32_t shift[16];
  int32_t width[16];
  int64_t off_base[16];
  int64_t off_words;
};

}  // namespace mrc

struct mrc_simhash_index {
  int device = 0;
  cudaStream_t stream = nullptr;  // stream of the building context (the free is ordered on it)
  int64_t n = 0;
  int32_t hamming_max = 0;
  mrc::SimhashLayout layout{};
  uint64_t* fp = nullptr;  // [blocks * n] table t: fingerprints grouped by the value of block t
  int32_t* id = nullptr;   // [blocks * n] their positions in the input
  uint64_t* own = nullptr; // [n] the fingerprints in input order
  int32_t* off = nullptr;  // [layout.off_words] bucket offsets of every table
  void* block = nullptr;   // one stream-ordered allocation holding the arrays above
};

struct mrc_ctx {
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string last_error;
  std::map<std::string, mrc::Buffer> ws;  // grow-only scratch, by purpose
  bool timing = false;
  std::vector<mrc::PendingTiming> pending;
  std::vector<std::pair<std::string, mrc::KernelStat>> stats;
  std::vector<cudaEvent_t> free_events;
  void* pinned = nullptr;  // small pinned host scratch (counters)
  void* host_ws = nullptr;  // grow-only pinned host scratch (vocabulary-sized tables)
  size_t host_ws_bytes = 0;
  cudaEvent_t host_ws_done = nullptr;  // recorded after the last copy that reads host_ws
  int32_t* async_err = nullptr;  // device error word of the stream-ordered calls (until mrc_ctx_sync)
  uint64_t wait_limit_ns = 4000000000ull;  // bound of every device-side wait (mrc_ctx_set_wait_limit)
  bool test_stall = false;                 // compare kernels issue no MMA (mrc_ctx_set_test_stall)
  bool rescore = true;                     // mrc_match rescores its candidates (mrc_ctx_set_rescoring)
};

struct mrc_index {
  int device = 0;
  cudaStream_t stream = nullptr;  // stream of the building context (frees are ordered on it)
  mrc_params params{};
  int64_t n_docs = 0;
  int32_t vocab = 0;
  int32_t k = 0;
  int32_t kp = 0;       // padded row length (elements) of fp16 compare operands
  int32_t kp8 = 0;      // padded row length (bytes) of E4M3 compare operands
  int64_t L_used = 0;
  // reference norms |R_p| (host copy; the partition of each term lives in the device term table)
  std::vector<double> h_rnorm;
  // device arrays
  int32_t* df = nullptr;          // [vocab]
  float* idf = nullptr;           // [vocab]
  mrc::TermInfo* tinfo = nullptr; // [vocab]
  float* rinv = nullptr;          // [k] 1 / |R_p| (0 for empty partitions)
  float* rinv16 = nullptr;        // [k] the same of the bfloat16 weights (precision form only)
  float* sig = nullptr;           // [n * k] raw signatures
  float* sig_unit = nullptr;      // [n * k] unit signatures (FP32 rescoring)
  uint64_t* simhash = nullptr;    // [n]
  uint64_t* fhash = nullptr;      // [vocab] Simhash features (MD5 / SHA-1 modes; NULL under SplitMix64)
  void* op_hi = nullptr;          // [n * kp] fp16 (hi or the single fp16 operand)
  void* op_lo = nullptr;          // [n * kp] fp16 (lo of the split)
  void* op_e4m3 = nullptr;        // [n * kp8] e4m3
  float* qnorm = nullptr;         // [n] norms of the e4m3 rows
  float* qnorm_min = nullptr;     // [ceil(n / 128)] smallest non-zero qnorm of each 128-row block
  double* rnorm = nullptr;        // [k] |R_p| (written by the device reference selection)
  void* block = nullptr;          // one stream-ordered allocation holding every array above
  cudaEvent_t ready = nullptr;    // recorded on the building stream after the index's last pass
  cudaEvent_t tables = nullptr;   // recorded once the term tables (df, idf, tinfo) are complete
};

namespace mrc {

// ---- error / workspace helpers (api.cu) ----
mrc_status fail(mrc_ctx* ctx, mrc_status st, const std::string& msg);
// Index completion across streams: the build records x->ready after its last pass; a call on
// another stream makes that stream wait for it (no host wait).
void mark_index_ready(mrc_ctx* ctx, mrc_index* x);
void wait_for_index(mrc_ctx* ctx, const mrc_index* x);
// The same for the term tables alone (the exact cosine reads idf and the term table only, so it
// may run beside the index's signature pass).
void mark_index_tables(mrc_ctx* ctx, mrc_index* x);
void wait_for_index_tables(mrc_ctx* ctx, const mrc_index* x);
mrc_status cuda_fail(mrc_ctx* ctx, cudaError_t e, const char* what);
void* ws_get(mrc_ctx* ctx, const char* slot, size_t bytes, mrc_status* st);

// ---- launch set-up cache (api.cu) ----
// Resident CTAs per SM of `func` at `threads` threads and `smem` bytes of dynamic shared
// memory on the current device (at least 1). Raises the kernel's dynamic shared memory limit
// to `smem` first when needed. Results are cached per (kernel, device, threads, smem), so the
// runtime is queried once per configuration. Returns 0 if the limit cannot be raised.
int resident_ctas(const void* func, int threads, size_t smem);
template <typename K>
int resident_ctas(K* kernel, int threads, size_t smem) {
  return resident_ctas(reinterpret_cast<const void*>(kernel), threads, smem);
}

// ---- timing helpers (api.cu) ----
void timing_begin(mrc_ctx* ctx, const char* name, double bytes, double flops, cudaEvent_t* ev_out);
void timing_end(mrc_ctx* ctx, cudaEvent_t start);
// Times the launches made during its lifetime under `name` (when the context's timing is on).
struct KernelTimer {
  mrc_ctx* ctx;
  cudaEvent_t ev = nullptr;
  KernelTimer(mrc_ctx* c, const char* name, double bytes = 0.0, double flops = 0.0) : ctx(c) {
    timing_begin(c, name, bytes, flops, &ev);
  }
  ~KernelTimer() { timing_end(ctx, ev); }
  KernelTimer(const KernelTimer&) = delete;
  KernelTimer& operator=(const KernelTimer&) = delete;
};

// ---- launchers ----
struct DocsDev {
  int64_t n_docs;
  const int64_t* offsets;  // device
  const int32_t* tokens;   // device
  int64_t n_tokens;
  int32_t* err;            // the call's device error word (kErr* bits)
  // Optional bag of terms of these documents (device, [n_tokens] (term, count) pairs at the
  // documents' token offsets, [n_docs] pair counts): a pass with bag_write stores it, a later
  // pass with bag_read reads it instead of hashing the tokens again.
  int32_t* bag_terms = nullptr;
  int32_t* bag_cnts = nullptr;
  int32_t* bag_n = nullptr;
  int32_t bag_write = 0, bag_read = 0;
  // Set after a pass over these documents: its split into warp-path and CTA-path lists (in
  // the context's workspace) is still valid, so the next pass reuses it.
  int32_t lists_ready = 0;
};

// select.cu
// Reference selection on the device from df [V] (mode MRC_SELECT_*): partition of every term
// into part [V] (-1 unselected), |R_p| into rnorm [k] (double) and 1 / |R_p| into rinv [k];
// idf NULL under count weighting, bf16: weights rounded to bfloat16; rinv16 (may be NULL):
// 1 / |R_p| of the bfloat16-rounded weights (the precision form's compare operands). Scratch:
// hist and above [n_docs + 2] int32, state [device_selection_words()] int64, keys [8192]
// uint64. state[5] = band size, state[6] = 1 if the band exceeded 8192 terms (part, rnorm and
// rinv are then not written: run launch_select_general), state[1] = L.
int64_t device_selection_words();
cudaError_t launch_select_region(mrc_ctx* ctx, const int32_t* df, int32_t V, int64_t n_docs, int64_t L,
                                 int64_t region_start, int32_t mode, const float* idf, int32_t bf16, int32_t k,
                                 int32_t* hist, int32_t* above, long long* state, unsigned long long* keys,
                                 int32_t* part, double* rnorm, float* rinv, float* rinv16);
// The selection of a band of any size, after launch_select_region reported state[6] = 1 (a
// no-op otherwise): same outputs, from the same state. scratch: select_general_bytes(V) bytes
// of device memory.
size_t select_general_bytes(int32_t V);
cudaError_t launch_select_general(mrc_ctx* ctx, const int32_t* df, int32_t V, const float* idf, int32_t bf16,
                                  int32_t k, long long* state, void* scratch, int32_t* part, double* rnorm,
                                  float* rinv, float* rinv16);

// ingest.cu
cudaError_t launch_df(mrc_ctx* ctx, const DocsDev& d, int32_t* df, int32_t vocab);
// The df pass plus each document's squared weight norm |w|^2 (w = count * idf, or count when
// idf is NULL) as a 2^-22 fixed-point sum, written to norm[doc] for every document.
cudaError_t launch_df_norm(mrc_ctx* ctx, const DocsDev& d, int32_t* df, int32_t vocab, const float* idf,
                           unsigned long long* norm);
// Term table of the signature pass: tinfo[t] = {weight of t in a reference (idf under TF-IDF,
// bfloat16-rounded when bf16 != 0; 1 under counts), reference partition of t or -1}.
cudaError_t launch_term_info(mrc_ctx* ctx, const float* idf, const int32_t* part, int32_t vocab, int32_t tfidf,
                             int32_t bf16, TermInfo* tinfo);
cudaError_t launch_idf(mrc_ctx* ctx, int64_t n_docs, const int32_t* df, int32_t vocab, int32_t weighting,
                       float* idf, TermInfo* tinfo);
struct SigOut {
  float* sig;          // [n*k] raw (may be null)
  float* sig_unit;     // [n*k] unit (may be null)
  uint64_t* simhash;   // [n] (may be null)
  void* op_hi;         // [n*kp] fp16 (may be null)
  void* op_lo;         // [n*kp] fp16 (may be null)
  void* op_e4m3;       // [n*kp8] (may be null)
  float* qnorm;        // [n] norm of the quantized E4M3 unit signature (may be null)
  int32_t kp, kp8;
};
// Signature pass. The stored signatures (sig, sig_unit, fp16 operands) use the FP32 term table;
// with rinv16 (the precision form), the E4M3 operand and its norm come from signatures of the
// same documents whose weights and reference weights are rounded to bfloat16.
cudaError_t launch_signature(mrc_ctx* ctx, const DocsDev& d, int32_t vocab, const TermInfo* tinfo, const float* rinv,
                             const float* rinv16, int32_t k, uint64_t seed, const uint64_t* fhash,
                             const SigOut& out);
// Character 3-grams of a text CSR (text.cu): gram_offsets [n_docs + 1], grams [capacity] (ids past
// capacity dropped); tile_doc, tile_cnt [text_gram_tiles(n_bytes)], group_sum [ceil(tiles / 1024)],
// tile_base [tiles + 1] scratch, the total
// lands in tile_base[tiles]; invalid offsets set kErrBadOffsets in err.
int64_t text_gram_tiles(int64_t n_bytes);
cudaError_t launch_text_grams(mrc_ctx* ctx, int64_t n_docs, const int64_t* text_offsets, const uint8_t* text,
                              int64_t n_bytes, int64_t* gram_offsets, int32_t* grams, int64_t capacity,
                              int64_t* tile_doc, int32_t* tile_cnt, int64_t* group_sum, int64_t* tile_base,
                              int32_t* err);
// Block-table Hamming index (simhash_index.cu). cnt, cursor: [L.off_words] scratch.
SimhashLayout simhash_layout(int32_t hamming_max);
cudaError_t launch_simhash_index_build(mrc_ctx* ctx, const uint64_t* fps, int64_t n, const SimhashLayout& L,
                                       int32_t* cnt, int32_t* cursor, int32_t* off, uint64_t* fp_out,
                                       int32_t* id_out);
cudaError_t launch_simhash_index_probe(mrc_ctx* ctx, const uint64_t* q, int64_t nq, bool all_pairs, int32_t hmax,
                                       const SimhashLayout& L, int64_t n, const uint64_t* fp, const int32_t* id,
                                       const int32_t* off, mrc_pair* pairs, unsigned long long* count,
                                       int64_t capacity);
// batch_kernel.cu: a query batch's whole pipeline (signature pass, tensor-core compare with the
// index, FP32 rescoring, Hamming probe of a fingerprint index, grouping by query) as one
// persistent cooperative kernel. All pointers are device memory owned by the batch.
struct BatchKernelArgs {
  const mrc_index* index;
  int64_t max_docs, max_tokens;
  const int64_t* offsets;  // [max_docs + 1]; entries past n_live are not read
  const int32_t* tokens;   // [max_tokens]
  const int64_t* n_live;   // [1] documents of this launch (<= max_docs)
  float* unit;             // [max_docs * k] unit signatures
  void* op;                // [max_docs * kp] fp16 or [max_docs * kp8] E4M3 compare operands
  float* qnorm;            // [max_docs] E4M3 operand norms
  uint64_t* simhash;       // [max_docs]
  float tau, thresh;       // result threshold; compare threshold (tau less the form's bound or margin)
  int32_t tile_n, ring, prefetch;  // compare tile width (128 / 256), B ring depth, L2 prefetch distance
  mrc_pair* cand;
  int64_t cand_cap;
  mrc_pair* pairs;
  int64_t capacity;
  unsigned long long* counts;  // [0] pairs, [1] candidates
  int32_t* err;
  int32_t* ctl;            // [kBatchCtlWords], zero before each launch
  int32_t* long_list;      // [max_docs]
  int32_t qstride;         // per-query counter stride (words)
  int32_t* qcnt;           // [max_docs * qstride]
  int32_t* qfill;          // [max_docs * qstride]
  int64_t* qoff;           // [max_docs + 1]
  mrc_pair* grouped;       // [capacity]
  // Hamming leg (shx == NULL: none)
  const mrc_simhash_index* shx;
  int32_t hmax;
  mrc_pair* hpairs;
  unsigned long long* hcount;
  int64_t hcapacity;
  int32_t* hqcnt;
  int32_t* hqfill;
  int64_t* hqoff;
  mrc_pair* hgrouped;
  unsigned long long* stamps;  // [kBatchStamps] phase timestamps of the last launch (global timer, ns)
};
constexpr int kBatchCtlWords = 8;
constexpr int kBatchStamps = 7;  // start, then the end of phases 0..5
// True if the persistent batch kernel handles this index (compare rows of 64 or 128 bytes).
bool batch_kernel_supported(const mrc_index* index);
cudaError_t launch_batch_kernel(mrc_ctx* ctx, const BatchKernelArgs& a);
// out[t] = the MD5 (mode MRC_HASH_MD5) or SHA-1 (MRC_HASH_SHA1) Simhash feature of term t < vocab.
cudaError_t launch_feature_table(mrc_ctx* ctx, int32_t vocab, uint64_t seed, int32_t mode, uint64_t* out);
// Packs rows of `sig` (normalised to unit length first when `normalize`) into compare operands.
cudaError_t launch_pack(mrc_ctx* ctx, const float* sig, int64_t n, int32_t k, int32_t normalize, void* hi, void* lo,
                        void* e4m3, float* qnorm, float* unit, int32_t kp, int32_t kp8);
// out[b] = smallest non-zero norm[128 b .. 128 b + 127] (1 when the block has none)
cudaError_t launch_block_min(mrc_ctx* ctx, const float* norm, int64_t n, float* out);
struct DenseOut {
  const float* idf;       // [vocab] FP32 idf under TF-IDF weighting, NULL for counts
  const int32_t* colmap;  // [vocab] head column, -2 tail term, -1 skipped
  int32_t kd;             // padded head width (elements)
  void* head_hi;          // [n*kd] fp16
  void* head_lo;          // [n*kd] fp16
  const int64_t* tail_start;  // [vocab] start of the term's postings
  int32_t* tail_fill;         // [vocab] fill cursors (zeroed)
  int4* post;                 // [n_post] (document, weight bits, index of the posting's term in its
                              // document's tail list, 0): one 16-byte store per posting
  int32_t* row_cnt;           // [n] tail terms of each doc
  float* row_w;               // [n_tokens] at the doc's token offsets: unit weight of its r-th tail term
  const unsigned long long* norm;  // [n] squared norms, 2^-22 fixed point (from launch_df_norm)
  // postings == 1: tail postings (tail_start, tail_fill, post) for the tail walk. postings == 0
  // (bound-pruned exact cosine): instead each document's tail term ids (row_term, beside row_w)
  // and, in head columns kd_h .. kd_h + kTailBuckets - 1, the norms of its tail weights in each
  // of kTailBuckets hash buckets of the term ids (so the head GEMM also sums the bound).
  int32_t postings;
  int32_t* row_term;          // [n_tokens] at the doc's token offsets: id of its r-th tail term
  int32_t kd_h;               // head columns proper (a multiple of 64, may be 0; kd_h + kTailBuckets <= kd)
  const int32_t* kd_h_dev;    // non-null: kd_h read from the device (kd is then only the row stride)
};
constexpr int kTailBuckets = 256;
// Bucket of a tail term id (the top 8 bits of a multiplicative hash).
__host__ __device__ inline int32_t tail_bucket(int32_t t) { return (int32_t)(((uint32_t)t * 0x9E3779B1u) >> 24); }
cudaError_t launch_densify(mrc_ctx* ctx, const DocsDev& d, int32_t vocab, const TermInfo* tinfo, const DenseOut& out);

// compare_tc.cu
struct GemmArgs {
  int32_t fmt;          // OperandFormat
  const void* a_hi;     // [na * kpad] (rows of A)
  const void* a_lo;
  const void* b_hi;     // [nb * kpad] (rows of B); == A for the triangle
  const void* b_lo;
  int64_t na, nb;
  int32_t kbytes;       // bytes per row of one operand (padded)
  int32_t triangle;     // 1: A == B, only pairs i < j
  float thresh;         // epilogue threshold (score >= thresh)
  float out_scale;      // score = acc * out_scale (E4M3), 1 otherwise
  const float* a_norm;  // E4M3: norms of the quantized rows of A and B; the score is the
  const float* b_norm;  //   cosine of the quantized vectors, acc * out_scale / (|qa| |qb|)
  const float* b_norm_min;  // E4M3: smallest non-zero b_norm of each 128-row block of B
  // epilogue: pairs (thresh) or dense store
  mrc_pair* pairs;
  unsigned long long* count;
  int64_t capacity;
  float* store;         // non-null: write the score tile to store[i * ld + j] instead of thresholding
  void* store16;        // non-null: the same as fp16
  int64_t ld;
  int32_t tile_n;       // compare tile width for small K: 128, 256 or 0 (default)
  int32_t* err;         // device error word
  const char* name;     // timing name (NULL: by format and epilogue)
  const int32_t* kblocks_dev;  // non-null: the number of 64-element K blocks, read from the device
                               // (kbytes is then the row stride and the K extent of the maps)
  int32_t exact_scores;  // E4M3 thresholding: 1 = exact per-column test and quantized-cosine
                         // scores (the candidates are the result); 0 = the block bound alone,
                         // raw accumulators (every candidate is rescored afterwards)
  int32_t prefetch;      // resident kernel: L2 prefetch distance in B tiles (0: none, < 0: by size)
  int32_t ring;          // resident kernel: B ring depth (0: as deep as shared memory allows)
};
// L2 prefetch distance the resident compare uses when GemmArgs.prefetch < 0: B tiles streamed
// from DRAM (a query x index compare whose index rows exceed kPrefetchMinBytes) are prefetched
// this many tiles ahead.
constexpr int32_t kPrefetchTiles = 8;
constexpr int64_t kPrefetchMinBytes = 64ll << 20;
cudaError_t launch_gemm_compare(mrc_ctx* ctx, const GemmArgs& g);
// FP32 rescoring of the first min(*n_cand, cand_cap) candidates (unit_dot of rows i of qunit
// and j of xunit, k entries each); pairs scoring >= tau are appended to pairs / count (at most
// capacity written). A candidate count above cand_cap sets kErrOverflow in err (if given).
cudaError_t launch_rescore(mrc_ctx* ctx, const mrc_pair* cand, const unsigned long long* n_cand, int64_t cand_cap,
                           const float* qunit, const float* xunit, int32_t k, float tau, mrc_pair* pairs,
                           unsigned long long* count, int64_t capacity, int32_t* err);

// simhash_match.cu
// Measured issue rate of 32-bit POPC on this device (population counts per second).
cudaError_t measure_popc_rate(mrc_ctx* ctx, double* popc_per_s);
// ingest.cu: measured rate of 64-bit shared-memory atomic adds on this device (per second).
cudaError_t measure_smem_atomic_rate(mrc_ctx* ctx, double* atomics_per_s);
cudaError_t launch_simhash_match(mrc_ctx* ctx, const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb,
                                 int32_t hmax, mrc_pair* pairs, unsigned long long* count, int64_t capacity);

// Head/tail split of the vocabulary for the exact cosine: df >= cut -> head column (colmap =
// column, in term-id order), 2 <= df < cut -> tail term (colmap = -2, tstart = start of its
// postings; cstart[c], cstart[c + 1] bound the c-th tail list; rank_terms lists the tail
// terms of at most 32 postings first), else colmap = -1. part: [8 * ceil(V / 1024)] int64
// scratch. summary (int64): [0] head terms, [1] tail terms, [2] tail postings, [3] tail
// terms of <= 32 postings, [4] longest tail list, [5] sum over tail terms of df (df - 1) / 2.
cudaError_t launch_cosine_terms(mrc_ctx* ctx, const int32_t* df, int32_t V, int32_t cut, long long* part,
                                long long* summary, int32_t* colmap, int64_t* tstart, int64_t* cstart,
                                int32_t* rank_terms);

// tail.cu
// Orders every tail term's postings by document into spost ((document, weight bits) int32
// pairs) and records, for each
// (document, tail term) entry of the per-document lists, the range of the term's postings that
// follow that document. small_terms: tail terms (indices into cstart) with at most 32
// postings; big_terms: the others, each with at most max_m postings.
cudaError_t launch_rank_postings(mrc_ctx* ctx, const int64_t* cstart, const int32_t* small_terms, int32_t n_small,
                                 const int32_t* big_terms, int32_t n_big, int32_t max_m, const int4* post,
                                 const int64_t* doc_off, void* spost,
                                 void* row_walk);
// Exact cosine completion: approximate fp16 head scores H plus exact tail products, candidates
// >= tau - delta rescored exactly (head from the hi/lo split rows [n x kd], tail exact).
// Exact scores of the bound-pruned candidates (see k_cosine_verify); pairs with score >= tau
// go to pairs/count; a candidate count above cand_cap sets kErrOverflow in err.
// dims[0] = kd_h = head columns rounded up to 64 (from the split's totals, at most kd_h_max),
// dims[1] = (kd_h + kTailBuckets) / 64 K blocks of the bound-pruned head GEMM.
cudaError_t launch_cosine_dims(mrc_ctx* ctx, const long long* split_totals, int32_t kd_h_max, int32_t* dims);
// Zeroes columns [0, kd_h + kTailBuckets) of each hi row and [0, kd_h) of each lo row (stride ld).
cudaError_t launch_zero_head(mrc_ctx* ctx, void* head_hi, void* head_lo, int64_t n, int32_t ld, const int32_t* dims);
cudaError_t launch_cosine_verify(mrc_ctx* ctx, const mrc_pair* cand, const unsigned long long* n_cand,
                                 int64_t cand_cap, const void* head_hi, const void* head_lo, int32_t ld, int32_t kd,
                                 const int32_t* kd_dev,
                                 const int64_t* row_off, const int32_t* row_cnt, const int32_t* row_term,
                                 const float* row_w, float tau, mrc_pair* pairs, unsigned long long* count,
                                 int64_t capacity, int32_t* long_idx, unsigned long long* n_long, int32_t* err);
cudaError_t launch_cosine_tail(mrc_ctx* ctx, int64_t n, const void* H16, int64_t ldh, const int64_t* row_off,
                               const int32_t* row_cnt, const void* row_walk, const float* row_w, const void* spost,
                               int64_t n_postings, const void* head_hi, const void* head_lo,
                               int32_t kd, float tau, float delta, mrc_pair* pairs, unsigned long long* count,
                               int64_t capacity, double work_pairs, unsigned long long* next_item);

}  // namespace mrc
