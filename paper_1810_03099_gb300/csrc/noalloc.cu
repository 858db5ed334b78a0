// noalloc.cu -- mrc_signature_noalloc: document signatures without any device allocation.
//
// Some callers cannot allocate device memory at the time they need
// signatures: a serving process whose memory manager has already reserved
// the GPU's free memory for its own pools and admission control, or any
// request path that must not call cudaMalloc/cudaFree because those calls
// synchronise the device and may fail under memory pressure. mrc_signature
// takes its scratch from the context's grow-on-demand workspace, which can
// call cudaMalloc. This entry point runs the same kernels but takes its
// scratch from the fixed device array below, which the CUDA runtime creates
// when it loads this library's module on a device and which stays resident on
// that device until the process exits (about 512 KB per device).
//
// The array holds the per-call document lists (warp path and CTA path) and
// the call's counters and error word: at most MRC_NOALLOC_MAX_DOCS documents
// per call. Every call on a device shares it and finds the previous call's
// contents there: the counters and error word are cleared at the start of
// each call, and the lists are rewritten before they are read. Two calls
// whose work overlaps on the same device (different streams or host
// threads) race on the array and must be serialised by the caller.
#include <string>

#include "device.cuh"
#include "internal.h"

namespace mrc {
cudaError_t launch_signature_scratch(mrc_ctx* ctx, const DocsDev& d, int32_t vocab, const TermInfo* tinfo,
                                     const float* rinv, int32_t k, uint64_t seed,
                                     const uint64_t* fhash, const SigOut& out, int32_t* lists, int64_t cap, int32_t* counts, int32_t* err,
                                     int32_t* host_err);
}  // namespace mrc

namespace {

constexpr int64_t kMaxDocs = MRC_NOALLOC_MAX_DOCS;
// [0, kMaxDocs): warp-path list; [kMaxDocs, 2 kMaxDocs): CTA-path list;
// then 32 counter words and the error word.
constexpr int64_t kWords = 2 * kMaxDocs + 64;

static __device__ __align__(256) int32_t g_signature_scratch[kWords];

// Device address of the array on the current device. The host-side name of a __device__ array
// is not a device address; the runtime resolves it for the current device's context. It is
// looked up on every call (a host-side table lookup once the module is loaded, which the
// first call on a device does), so no address outlives a device reset or a module reload.
mrc_status scratch_on(mrc_ctx* ctx, int32_t** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_signature_scratch);
  if (e != cudaSuccess || !p) return mrc::cuda_fail(ctx, e, "cudaGetSymbolAddress of the signature scratch");
  *out = static_cast<int32_t*>(p);
  return MRC_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" mrc_status mrc_signature_noalloc(mrc_ctx* ctx, const mrc_index* index, const mrc_docs* docs, float* sig,
                                            uint64_t* simhash) {
  if (!ctx || !index) return MRC_ERR_INVALID;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != ctx->device) cudaSetDevice(ctx->device);
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, ctx->device};
  mrc::wait_for_index(ctx, index);

  if (!docs || docs->n_docs < 0) return mrc::fail(ctx, MRC_ERR_INVALID, "docs is NULL or n_docs < 0");
  if (docs->n_docs > kMaxDocs)
    return mrc::fail(ctx, MRC_ERR_INVALID,
                     "mrc_signature_noalloc: n_docs " + std::to_string(docs->n_docs) +
                         " exceeds MRC_NOALLOC_MAX_DOCS (" + std::to_string(kMaxDocs) + "); split the batch");
  if (docs->n_docs == 0) return MRC_OK;
  if (!sig && !simhash) return mrc::fail(ctx, MRC_ERR_INVALID, "no output requested");
  if (!on_device(docs->offsets) || !on_device(docs->tokens) || (sig && !on_device(sig)) ||
      (simhash && !on_device(simhash)))
    return mrc::fail(ctx, MRC_ERR_INVALID,
                     "mrc_signature_noalloc: offsets, tokens and outputs must be device memory (it copies nothing)");

  // the call waits for its own stream (list sizes, error word), which a stream capture forbids
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return mrc::fail(ctx, MRC_ERR_UNSUPPORTED, "mrc_signature_noalloc cannot run while its stream is being captured");
  }
  int32_t* scratch = nullptr;
  mrc_status st = scratch_on(ctx, &scratch);
  if (st != MRC_OK) return st;
  int32_t* lists = scratch;
  int32_t* counts = scratch + 2 * kMaxDocs;
  int32_t* err = counts + 32;

  mrc::DocsDev d{};
  d.n_docs = docs->n_docs;
  d.offsets = docs->offsets;
  d.tokens = docs->tokens;
  d.n_tokens = 0;
  d.err = err;
  mrc::SigOut o{};
  o.sig = sig;
  o.simhash = simhash;
  int32_t herr = 0;
  const cudaError_t e = mrc::launch_signature_scratch(ctx, d, index->vocab, index->tinfo, index->rinv, index->k,
                                                      index->params.seed, index->fhash, o, lists, kMaxDocs,
                                                      counts, err, &herr);
  if (e != cudaSuccess) return mrc::cuda_fail(ctx, e, "mrc_signature_noalloc");
  if (herr & mrc::kErrBadOffsets) return mrc::fail(ctx, MRC_ERR_INVALID, "offsets must start at 0 and be non-decreasing");
  if (herr & mrc::kErrTooLong)
    return mrc::fail(ctx, MRC_ERR_UNSUPPORTED, "a document is longer than MRC_MAX_DOC_TOKENS tokens");
  if (herr & mrc::kErrBadToken) return mrc::fail(ctx, MRC_ERR_INVALID, "a token id is outside [0, vocab)");
  if (herr) return mrc::fail(ctx, MRC_ERR_CUDA, "internal error word " + std::to_string(herr));
  return MRC_OK;
}
