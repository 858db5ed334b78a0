/*
 * mrc.h -- C ABI of the GB300 (sm_103a) Multi-reference Cosine library.
 *
 * Multi-reference Cosine (Mohammadi & Nikoukaran, arXiv 1810.03099) gives each
 * document a short signature: the cosine (Eq. 1) between the document's term
 * vector and each of k reference partitions (Section IV). Near-duplicate pairs
 * are then found by comparing signatures instead of whole documents. The
 * library also runs the two methods the paper measures against (Section V,
 * Table 1): exact cosine on the full term vectors, and 64-bit Simhash with
 * Hamming distance (Section III).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Documents are a token CSR: offsets[n_docs + 1] (int64, offsets[0] == 0,
 *   non-decreasing) and tokens[offsets[n_docs]] (int32 term ids in [0, vocab)).
 *   A term id stands for one character 3-gram of Section III.
 * - Every array argument may live in device memory or in host memory (pinned or
 *   pageable); the library inspects each pointer. Host inputs are copied to the
 *   device and host outputs are filled from the device inside the call.
 * - The caller owns every argument buffer. The library owns mrc_ctx, mrc_index
 *   and all device memory they hold.
 * - All work is issued on the stream given to mrc_ctx_create. Calls that return
 *   a pair count (mrc_match, cosine_allpairs, simhash_match) synchronise that
 *   stream before returning; their *_async forms and the other calls are
 *   stream-ordered and their device outputs are valid once the stream reaches
 *   them (mrc_ctx_sync waits for that and reports device-side errors).
 * - Pairs: all-pairs calls emit each unordered pair once with i < j; query
 *   calls emit (query index i, index/database position j). Self-pairs are never
 *   emitted. Pair order in the output is unspecified. *n_pairs always receives
 *   the total number found; when it exceeds `capacity`, `capacity` of them are
 *   written and the call returns MRC_ERR_CAPACITY (retry with more room).
 * - No exception crosses the ABI. A failing call returns a status and leaves a
 *   message for mrc_last_error(). One context per host thread.
 */
#ifndef MRC_H_
#define MRC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t mrc_status;
#define MRC_OK 0
#define MRC_ERR_INVALID 1     /* bad argument (sizes, ids out of range, NULL)      */
#define MRC_ERR_OOM 2         /* device allocation failed                           */
#define MRC_ERR_CAPACITY 3    /* more pairs than `capacity`; *n_pairs is the total  */
#define MRC_ERR_CUDA 4        /* a CUDA call failed; see mrc_last_error             */
#define MRC_ERR_TIMEOUT 5     /* a bounded device-side wait gave up                 */
#define MRC_ERR_UNSUPPORTED 6 /* valid request outside what this build implements   */

/* Reference selection modes (Section IV). */
#define MRC_SELECT_ALL 0    /* every term of non-zero document frequency              */
#define MRC_SELECT_REGION 1 /* L consecutive ranks of the df-sorted list from region_start */
#define MRC_SELECT_DF1 2    /* the first L terms (id order) that occur in one document */

/* Term weighting. The paper counts N-grams (Section III); TF-IDF is the
 * weighted vector space model its Section VI names as future work. */
#define MRC_WEIGHT_COUNT 0 /* w(d,t) = c(d,t)                                    */
#define MRC_WEIGHT_TFIDF 1 /* w(d,t) = c(d,t) * (ln((1+N)/(1+df(t))) + 1)       */

/* Arithmetic of the signature comparison. */
#define MRC_PREC_FP32 0     /* FP32-accurate: fp16 tensor-core candidates within a proven
                               bound of tau, every candidate rescored in FP32 */
#define MRC_PREC_BF16_FP8 1 /* compare operands from BF16 weights, FP8 E4M3 compare,
                               candidates within margin of tau rescored in FP32 from the
                               FP32-weight signatures (the stored signatures)           */
#define MRC_PREC_FP16 2     /* FP16 compare operands at the proven bound tau - 2e-3,
                               FP32 rescoring: the arithmetic of MRC_PREC_FP32 (the
                               serving configuration's name for it)                     */

/* The 64-bit Simhash feature hash of a term t (Section III hashes words with MD5 or SHA1). */
#define MRC_HASH_SPLITMIX64 0 /* one SplitMix64 step (Steele, Lea, Flood 2014) from t XOR seed */
#define MRC_HASH_MD5 1        /* MD5 (RFC 1321) of the 12 bytes t (int32, little-endian), seed
                                 (uint64, little-endian); the first 8 digest bytes, read as a
                                 little-endian word, are the feature                         */
#define MRC_HASH_SHA1 2       /* SHA-1 (FIPS 180-4) of the same message, same 8 bytes       */

#define MRC_MAX_K 256               /* longest signature                                */
#define MRC_MAX_DOC_TOKENS 65536    /* longest document (exact per-document sums)       */

typedef struct mrc_ctx mrc_ctx;
typedef struct mrc_index mrc_index;

typedef struct {
  int32_t i;   /* first document (query) index                          */
  int32_t j;   /* second document (index position) index                */
  float score; /* signature or exact cosine; Hamming distance for Simhash */
} mrc_pair;

/* A document batch (token CSR). offsets and tokens may be device or host memory. Host
 * offsets are copied in; page-locked host tokens (cudaHostAlloc / cudaHostRegister) are read in
 * place by the kernels over the CPU-GPU link, other host tokens are copied in. Either way the
 * caller keeps them unchanged until the call's stream has passed the call's kernels (a call
 * with host outputs has, on return). */
typedef struct {
  int64_t n_docs;
  const int64_t* offsets; /* [n_docs + 1] */
  const int32_t* tokens;  /* [offsets[n_docs]] */
} mrc_docs;

typedef struct {
  int32_t k;            /* signature length = number of reference partitions, 1..MRC_MAX_K */
  int32_t L;            /* reference terms selected; < 0 selects 32 * k                     */
  int32_t select_mode;  /* MRC_SELECT_*                                                     */
  int32_t region_start; /* REGION: first rank; < 0 = first rank with df <= n_docs / 100     */
  int32_t weighting;    /* MRC_WEIGHT_*                                                     */
  int32_t precision;    /* MRC_PREC_*                                                       */
  float tau;            /* similarity threshold (inclusive), e.g. 0.9                       */
  float margin;         /* precision form (E4M3): candidates >= tau - margin are rescored   */
  int32_t hamming_max;  /* Simhash: pairs with Hamming distance <= hamming_max              */
  int32_t feature_hash; /* MRC_HASH_*: Simhash feature hash (MD5 / SHA-1: a per-term table
                           of 8 * vocab bytes is computed with the index)                  */
  uint64_t seed;        /* seed of the 64-bit Simhash feature hash                          */
} mrc_params;

typedef struct {
  int64_t n_docs;
  int32_t vocab;
  int32_t k;
  int64_t L_used;     /* reference terms actually selected                      */
  int32_t precision;
  int32_t weighting;
  int32_t kp;         /* padded signature row length of the compare operands     */
  int32_t reserved;
} mrc_index_info;

/* Fill *p with the library defaults: k = 8, L = 32k, REGION from the default
 * start, TF-IDF, FP32, tau = 0.9, margin = 0.02, hamming_max = 3, SplitMix64
 * features, seed 0x1810030990. */
void mrc_params_default(mrc_params* p);

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
mrc_status mrc_ctx_create(void* cuda_stream, mrc_ctx** out);
void mrc_ctx_destroy(mrc_ctx* ctx);
/* Message of the last failing call on this context (never NULL). */
const char* mrc_last_error(const mrc_ctx* ctx);

/*
 * Character 3-grams of raw text (Section III: a document is the vector of its
 * 3-gram counts; a 3-gram is a sequence of three letters of the alphabet).
 * The alphabet is the 26 ASCII letters with case folded; every other byte
 * (digits, punctuation, white space, bytes >= 0x80) separates. A 3-gram is
 * any three consecutive letters of one document, numbered 676 x + 26 y + z
 * (letters 0..25), so ids lie in [0, MRC_GRAM_VOCAB).
 * Input: n_docs documents; text_offsets [n_docs + 1] int64 byte offsets
 * (text_offsets[0] = 0, non-decreasing), text [text_offsets[n_docs]] bytes.
 * Output, a token CSR for mrc_build_index / mrc_signature / cosine_allpairs
 * with vocab = MRC_GRAM_VOCAB: gram_offsets [n_docs + 1] int64 and grams
 * [capacity] int32, each document's 3-grams in text order. A document has at
 * most max(0, bytes - 2) 3-grams, so capacity >= text_offsets[n_docs]
 * always suffices. Every pointer may be device or host memory (host inputs
 * are copied in, host outputs copied back before the call returns; the call
 * synchronises the stream once). *n_grams (host) receives the total.
 * Errors: MRC_ERR_INVALID for NULL pointers or invalid offsets;
 * MRC_ERR_CAPACITY when the total exceeds capacity (gram_offsets complete,
 * the first `capacity` ids written).
 */
#define MRC_GRAM_VOCAB 17576 /* 26^3 */
mrc_status mrc_text_grams(mrc_ctx* ctx, int64_t n_docs, const int64_t* text_offsets, const uint8_t* text,
                          int64_t* gram_offsets, int32_t* grams, int64_t capacity, int64_t* n_grams);

/*
 * Build a device-resident signature index over `corpus` (Sections III-IV):
 * term counts per document, document frequencies, idf (frozen for later
 * queries), reference selection and partitioning (on the device in every
 * mode: the band of df values the selection meets is ranked by df, then id),
 * then every document's signature
 * s_p(d) = cos(v(d), v(R_p)) (Eq. 1 against partition p), its unit-length
 * packed form for comparison, and its 64-bit Simhash (Section III).
 * vocab: number of term ids. The returned index must be freed with
 * mrc_index_free. Errors: MRC_ERR_INVALID for bad sizes/params/term ids,
 * MRC_ERR_UNSUPPORTED for documents longer than MRC_MAX_DOC_TOKENS (the call
 * waits for the passes that validate the documents). The signature pass may
 * still be running when the call returns: the index is complete in order on
 * ctx's stream. Every call that takes the index on another context's stream
 * first makes that stream wait for the index (an event, no host wait).
 */
mrc_status mrc_build_index(mrc_ctx* ctx, const mrc_docs* corpus, int32_t vocab, const mrc_params* params,
                           mrc_index** out);

/*
 * Signatures (and Simhash) of new documents against a built index, with the
 * index's idf and references (Section IV; the paper compares each new page
 * with the signature database, Section I). sig: [n_docs * k] float32 raw
 * cosines (row-major); simhash: [n_docs] uint64 or NULL.
 */
mrc_status mrc_signature(mrc_ctx* ctx, const mrc_index* index, const mrc_docs* docs, float* sig,
                         uint64_t* simhash);

/*
 * mrc_signature for callers that cannot allocate device memory on the call
 * path: for example a serving process whose memory manager has already
 * reserved the GPU's free memory for its own pools and admission control, or
 * a request path that must not call cudaMalloc/cudaFree because they
 * synchronise the device and can fail under memory pressure. The paper has no
 * counterpart; this is a service of the library.
 *
 * Same results as mrc_signature (same kernels). Differences:
 * - it allocates nothing: its scratch is a fixed array of about 512 KB that
 *   the library keeps on every device that loads it, until the process exits;
 * - at most MRC_NOALLOC_MAX_DOCS documents per call (more: MRC_ERR_INVALID);
 * - offsets, tokens, sig and simhash must all be device memory (it copies
 *   nothing; host pointers: MRC_ERR_INVALID);
 * - every call looks up the array's device address on the current device
 *   (one runtime call; the first call on a device also loads the library's
 *   device code there), so a device reset between calls is harmless;
 * - it waits for its stream (list sizes, error word), so it cannot run while
 *   that stream is being captured into a graph (MRC_ERR_UNSUPPORTED);
 * - all calls on a device share the array: calls whose work overlaps on the
 *   GPU (other streams, other host threads) race and must be serialised.
 * The call synchronises the context's stream.
 */
#define MRC_NOALLOC_MAX_DOCS 65536
mrc_status mrc_signature_noalloc(mrc_ctx* ctx, const mrc_index* index, const mrc_docs* docs, float* sig,
                                 uint64_t* simhash);

/*
 * Signature comparison with a fused threshold: the cosine of two signatures
 * (the "multi reference cosine" of Eq. 2) >= tau. query_sig == NULL compares
 * all index pairs i < j; otherwise query_sig holds nq raw float32 signatures
 * ([nq * k], e.g. from mrc_signature) compared against every index document.
 * The index's precision decides the arithmetic (see MRC_PREC_*): the
 * tensor-core compare finds candidates at a lowered threshold (tau - 2e-3 in
 * the fp16 forms, a proven bound; tau - margin in the E4M3 form); each
 * candidate is then rescored as the FP32 dot product of the two unit
 * signatures and written iff that score >= tau (score = that FP32 cosine).
 * With rescoring turned off on the context (mrc_ctx_set_rescoring) the
 * candidates themselves are written, scored with the compare's own cosine.
 */
mrc_status mrc_match(mrc_ctx* ctx, const mrc_index* index, const float* query_sig, int64_t nq, float tau,
                     mrc_pair* pairs, int64_t capacity, int64_t* n_pairs);

/*
 * Exact cosine (Eq. 1) of the weighted term vectors of every pair i < j of
 * `docs` (the ground truth of Section V), emitting pairs with cosine >= tau.
 * Weights use the index's idf and weighting. FP32-accurate: the most frequent
 * terms form a dense fp16 head operand; every other term is hashed into one of
 * 256 buckets whose per-document norms ride as extra columns, so one
 * tensor-core GEMM gives head score + a Cauchy-Schwarz bound of the rest.
 * Pairs whose bound reaches tau minus the proven rounding slack are rescored
 * exactly (the head from its split rows, the rest by a hash join of the two
 * documents' term lists) and kept iff >= tau. If the candidates overflow their
 * buffer, the call falls back to an exhaustive sparse walk.
 */
mrc_status cosine_allpairs(mrc_ctx* ctx, const mrc_index* index, const mrc_docs* docs, float tau,
                           mrc_pair* pairs, int64_t capacity, int64_t* n_pairs);

/*
 * Simhash matching (Section III): Hamming distance popcount(a_i XOR b_j) <=
 * hamming_max. b == NULL compares all pairs i < j of a; otherwise every
 * (i in a, j in b). score = the Hamming distance.
 */
mrc_status simhash_match(mrc_ctx* ctx, const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb,
                         int32_t hamming_max, mrc_pair* pairs, int64_t capacity, int64_t* n_pairs);

/*
 * Stream-ordered forms of the three pair calls: the same work and the same
 * pairs, but nothing waits for the device. `pairs` (when capacity > 0) and
 * d_n_pairs must be device memory; d_n_pairs receives the total pair count
 * (int64) when the stream reaches the end of the call, and min(total,
 * capacity) pairs are written. A total above `capacity` is not an error here:
 * the caller reads *d_n_pairs and compares. Inputs may be host or device memory
 * as everywhere; a host input is copied before the call returns.
 * Device-side errors (a bounded wait that expired, a candidate buffer that
 * overflowed -- mrc_match collects its candidates in a buffer of
 * max(4 * capacity, 2^20) entries, which the synchronous form grows and
 * repeats on overflow; the exact cosine's buffer holds max(4 * capacity,
 * 2^22), and its synchronous form falls back to an exhaustive path) are
 * recorded in the context and returned by the next mrc_ctx_sync. cosine_allpairs_async waits for nothing unless per-kernel
 * timing is on (it then reads its head/tail split's sizes once).
 * Host-side argument errors return at once, as in the synchronous forms.
 *
 * mrc_ctx_sync waits for the context's stream and returns the first recorded
 * device-side error of the stream-ordered calls since the previous
 * mrc_ctx_sync (MRC_ERR_TIMEOUT, MRC_ERR_CAPACITY for a candidate overflow,
 * ...), clearing it; MRC_OK otherwise.
 */
mrc_status mrc_match_async(mrc_ctx* ctx, const mrc_index* index, const float* query_sig, int64_t nq, float tau,
                           mrc_pair* pairs, int64_t capacity, int64_t* d_n_pairs);
mrc_status cosine_allpairs_async(mrc_ctx* ctx, const mrc_index* index, const mrc_docs* docs, float tau,
                                 mrc_pair* pairs, int64_t capacity, int64_t* d_n_pairs);
mrc_status simhash_match_async(mrc_ctx* ctx, const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb,
                               int32_t hamming_max, mrc_pair* pairs, int64_t capacity, int64_t* d_n_pairs);
mrc_status mrc_ctx_sync(mrc_ctx* ctx);

/*
 * Batched queries, captured once as a CUDA graph (one graph launch per batch).
 * The paper signatures each new page and compares it with the signature
 * database (Section I, Section IV); a batch does that for up to max_docs new
 * documents at once against every document of `index`: signature pass,
 * tensor-core compare at a lowered threshold (tau - 2e-3 in the FP32 and FP16
 * forms, a proven bound; tau - margin in the E4M3 form), FP32 rescoring,
 * grouping of the pairs by query. Pairs are
 * (query position i in the batch, index document j).
 * With compare rows of one K block (k <= 64; k <= 128 in the E4M3 form) the graph holds one
 * persistent cooperative kernel (after a memset of its control words) that runs
 * every step, the Hamming leg included; wider rows run the steps as separate
 * kernels of the graph. mrc_batch_kernels returns the number of kernel nodes
 * in the captured graph (-1 for NULL).
 *   mrc_batch_create : allocates the pipeline's device buffers (inputs, outputs,
 *     workspace) and its own non-blocking stream, runs the pipeline once and
 *     captures it. max_tokens bounds the tokens of one batch; capacity bounds
 *     the pairs of one batch; tile_n is the compare tile width (0 = default:
 *     128 columns for the one-kernel batch; 128 or 256; see the autotuner). The
 *     batch keeps `index` (not owned).
 *   mrc_batch_launch : asynchronous. Copies the batch's offsets/tokens (host or
 *     device memory) and its document count into the pipeline (the separate-
 *     kernel form pads the batch to max_docs with empty documents) and launches
 *     the graph. At most one launch in flight per batch object; use several
 *     objects to overlap batches on the device.
 *   mrc_batch_tune   : the compare's tuning knobs (the autotuner's search space):
 *     tile_n (0, 128 or 256), ring = depth of the compare's streamed-operand ring
 *     (0 = as deep as shared memory allows, else 2..64, capped at what fits),
 *     prefetch = L2 prefetch distance in index tiles (-1 = by the index size:
 *     8 tiles when the index rows exceed 64 MB, else none; 0 = none; up to 64).
 *     Re-captures the graph; no launch may be in flight. Results do not depend
 *     on the knobs.
 *   mrc_batch_poll   : 1 when the last launch has finished (or none is pending), else 0.
 *   mrc_batch_wait   : waits for the last launch and copies min(total, capacity)
 *     pairs to `pairs` (host or device), grouped by query position i (order
 *     within a query unspecified); *n_pairs = total; query_offsets (may be NULL,
 *     [n_docs + 1] of the last launch) receives where each query's pairs start.
 *     pairs may be NULL (the total only). The results stay available until the
 *     next launch: calling it again copies them again. MRC_ERR_CAPACITY when the
 *     pairs (or the internal candidate list) overflowed.
 */
typedef struct mrc_batch mrc_batch;
typedef struct mrc_simhash_index mrc_simhash_index; /* block-table fingerprint index (below) */
mrc_status mrc_batch_create(mrc_ctx* ctx, const mrc_index* index, int64_t max_docs, int64_t max_tokens, float tau,
                            int64_t capacity, int32_t tile_n, mrc_batch** out);
mrc_status mrc_batch_launch(mrc_batch* batch, const mrc_docs* docs);
int32_t mrc_batch_poll(mrc_batch* batch);
mrc_status mrc_batch_wait(mrc_batch* batch, mrc_pair* pairs, int64_t capacity, int64_t* n_pairs,
                          int64_t* query_offsets);
mrc_status mrc_batch_tune(mrc_batch* batch, int32_t tile_n, int32_t ring, int32_t prefetch);
int32_t mrc_batch_kernels(const mrc_batch* batch);
/* Phase durations (ns, global timer of CTA 0) of the persistent kernel's last launch (waits for
 * it): [0] list documents, [1] signature pass, [2] compare, [3] rescoring and Hamming probe,
 * [4] offset scans, [5] scatter into query order (phase_ns: int64[6]). MRC_ERR_UNSUPPORTED
 * for a batch that runs separate kernels. */
mrc_status mrc_batch_phase_ns(mrc_batch* batch, int64_t* phase_ns);
const char* mrc_batch_last_error(const mrc_batch* batch);
void mrc_batch_free(mrc_batch* batch);

/*
 * Hamming leg of a batch pipeline (Section III: each new page's Simhash is
 * compared with the stored fingerprints; the serving form matches it against
 * the resident index's Simhashes). mrc_batch_attach_simhash adds, to the
 * captured graph, a probe of `index` (a block-table fingerprint index, see
 * mrc_simhash_index_build) with the batch's own Simhash fingerprints: every
 * (query position i, index position j) within hamming_max (<= the index's),
 * score = the Hamming distance, grouped by query like the signature pairs;
 * capacity bounds the Hamming pairs of one batch. Call it with no launch in
 * flight; the batch keeps `index` (not owned; it must outlive the batch).
 * mrc_batch_hamming (waits for the launch like mrc_batch_wait): copies
 * min(total, capacity) pairs of the last launch (host or device; pairs may be
 * NULL), *n_pairs = total, query_offsets (may be NULL, [n_docs + 1]) where each
 * query's pairs start. MRC_ERR_CAPACITY on overflow. The results equal mrc_simhash_index_match with the batch's
 * fingerprints as queries.
 */
mrc_status mrc_batch_attach_simhash(mrc_batch* batch, const mrc_simhash_index* index, int32_t hamming_max,
                                    int64_t capacity);
mrc_status mrc_batch_hamming(mrc_batch* batch, mrc_pair* pairs, int64_t capacity, int64_t* n_pairs,
                             int64_t* query_offsets);

/*
 * Block-table Hamming index over 64-bit Simhash fingerprints (Section I cites
 * Simhash for web-scale near-duplicate detection; Section III defines the
 * Hamming distance). The 64 bits are cut into b = max(hamming_max + 1, 4)
 * blocks; two fingerprints within distance hamming_max agree on at least one
 * block, so a search reads, in each of the b tables, only the bucket of the
 * query's block value. Results equal simhash_match's: same pairs, each once,
 * score = Hamming distance (pair order may differ).
 * Build: fps [n] uint64 (device or host; copied into the index), n < 2^31,
 * 0 <= hamming_max <= 15 (the largest distance later searches may ask for).
 * The index holds 12 * b * n bytes plus the bucket offsets; free it with
 * mrc_simhash_index_free (ordered on the building context's stream). Every
 * match call returns only after its probe has finished (it synchronises its
 * stream to read the pair count), so freeing the index after the match calls
 * that use it have returned is safe, whichever contexts they ran on.
 * Match: queries [nq] (device or host) x the index, pairs (q, x); queries ==
 * NULL: all pairs i < j of the index itself. hamming_max <= the build's.
 * Pairs, capacity and *n_pairs as simhash_match. Errors: MRC_ERR_INVALID for
 * bad sizes or a distance above the build's, MRC_ERR_CAPACITY on overflow.
 */
mrc_status mrc_simhash_index_build(mrc_ctx* ctx, const uint64_t* fps, int64_t n, int32_t hamming_max,
                                   mrc_simhash_index** out);
mrc_status mrc_simhash_index_match(mrc_ctx* ctx, const mrc_simhash_index* index, const uint64_t* queries, int64_t nq,
                                   int32_t hamming_max, mrc_pair* pairs, int64_t capacity, int64_t* n_pairs);
void mrc_simhash_index_free(mrc_simhash_index* index);

/* Index introspection and export (for checks and persistence). Each output
 * pointer may be NULL to skip it; sizes follow mrc_index_info. Host outputs
 * are complete on return; device outputs are written in order on the
 * context's stream, like every other call's device results. */
mrc_status mrc_index_get_info(const mrc_index* index, mrc_index_info* info);
mrc_status mrc_index_export(mrc_ctx* ctx, const mrc_index* index, float* sig /*[n*k]*/, uint64_t* simhash /*[n]*/,
                            int32_t* df /*[vocab]*/, float* idf /*[vocab]*/, int32_t* part /*[vocab]*/,
                            double* rnorm /*[k]*/);

/* Persist an index (params, idf, references, signatures, Simhashes and, in
 * the precision form, its E4M3 compare rows and their norms) to a versioned
 * binary file, and load it back onto ctx's device (version 1 files, which
 * lack the E4M3 rows, are re-packed from the unit signatures). */
mrc_status mrc_index_save(mrc_ctx* ctx, const mrc_index* index, const char* path);
mrc_status mrc_index_load(mrc_ctx* ctx, const char* path, mrc_index** out);
/* Release an index. Its memory is returned in order on the stream of the context that
 * built (or loaded) it, so that stream must still exist. */
void mrc_index_free(mrc_index* index);

/*
 * Bound of every device-side wait of the context's kernels (the pipeline
 * barriers of the tensor-core compares), in nanoseconds; default 4 s. Not in
 * the paper: failure detection of this library. A wait that runs out stops
 * its kernel early (after the kernel's own copies and tensor-core operations
 * in flight have landed and its tensor memory is freed); the call then returns
 * MRC_ERR_TIMEOUT (stream-ordered calls: at mrc_ctx_sync) and the context
 * stays usable. 1 <= ns <= 600e9, else MRC_ERR_INVALID. Applies to calls made
 * after it returns.
 */
mrc_status mrc_ctx_set_wait_limit(mrc_ctx* ctx, int64_t ns);

/*
 * Test of the bounded waits (failure detection; not in the paper). With
 * on != 0, the tensor-core compare kernels this context launches issue no
 * tensor-core operation, so the waits of their other roles for those results
 * are never met and run out after the wait limit: the call returns
 * MRC_ERR_TIMEOUT without hanging or faulting the GPU. Off by default; turn it
 * off again before normal use.
 */
mrc_status mrc_ctx_set_test_stall(mrc_ctx* ctx, int32_t on);

/*
 * Diagnostics of the reduced-precision forms (not in the paper). With on == 0,
 * mrc_match (and mrc_match_async) write the tensor-core compare's candidates
 * -- every pair whose compare cosine is >= tau - 2e-3 (fp16 forms) or
 * tau - margin (E4M3 form) -- scored with that cosine (fp16: the product
 * of the fp16 unit signatures; E4M3: the cosine of the quantized vectors),
 * without FP32 rescoring. Default on.
 */
mrc_status mrc_ctx_set_rescoring(mrc_ctx* ctx, int32_t on);

/*
 * Measurement helper (not in the paper): the rate at which ctx's device issues
 * 32-bit population counts, in POPC per second, from a probe kernel that keeps
 * eight independent XOR + POPC + add chains per thread in flight (best of three
 * timed runs after one warm-up). simhash_match evaluates one XOR and one POPC
 * per pair on the fingerprints' low halves, so this rate bounds its pairs/s.
 * Synchronises ctx's stream.
 */
mrc_status mrc_measure_popc_rate(mrc_ctx* ctx, double* popc_per_s);

/*
 * Measurement helper (not in the paper): the rate at which ctx's device completes 64-bit
 * shared-memory atomic adds, per second, from a probe kernel in which every thread keeps eight
 * adds to distinct slots of a 4,096-slot shared table in flight (best of three timed runs after
 * one warm-up). Building a document's bag of terms takes at least one such atomic per token (a
 * claim or an increment of the term's slot), so this rate bounds the signature pass's tokens/s.
 * Synchronises ctx's stream.
 */
mrc_status mrc_measure_smem_atomic_rate(mrc_ctx* ctx, double* atomics_per_s);

/*
 * Per-kernel timing. With timing on, every kernel the context launches is
 * bracketed by CUDA events on the context's stream; mrc_ctx_kernel_stat
 * returns, for kernel slot `slot` (0..count-1), its name, launches, summed
 * device time and the algorithmic bytes and flops its launches account for.
 * Returns the number of kernel slots, or -1 when `slot` is out of range.
 */
mrc_status mrc_ctx_set_timing(mrc_ctx* ctx, int32_t on);
int32_t mrc_ctx_kernel_stat(mrc_ctx* ctx, int32_t slot, char* name /*[64]*/, int64_t* launches,
                            double* total_ms, double* bytes, double* flops);
void mrc_ctx_reset_stats(mrc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* MRC_H_ */
