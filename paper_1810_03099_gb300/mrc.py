"""Python binding of the C ABI in include/mrc.h (argument marshalling only).

Every function here converts arguments (torch tensors on the GPU, or numpy
arrays / pinned host tensors) to plain pointers and sizes and calls the
library of the same name; all computation happens in the CUDA kernels behind
it. There is no fallback: if libmrc.so is missing or the GPU is absent the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmrc.so")

MRC_OK, MRC_ERR_INVALID, MRC_ERR_OOM, MRC_ERR_CAPACITY = 0, 1, 2, 3
MRC_ERR_CUDA, MRC_ERR_TIMEOUT, MRC_ERR_UNSUPPORTED = 4, 5, 6
SELECT_ALL, SELECT_REGION, SELECT_DF1 = 0, 1, 2
WEIGHT_COUNT, WEIGHT_TFIDF = 0, 1
HASH_SPLITMIX64, HASH_MD5, HASH_SHA1 = 0, 1, 2
GRAM_VOCAB = 17576  # MRC_GRAM_VOCAB: character 3-grams over the 26-letter alphabet
PREC_FP32, PREC_BF16_FP8, PREC_FP16 = 0, 1, 2
MAX_K = 256


class MrcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"mrc status {status}: {message}")
        self.status = status
        self.message = message


class Params(C.Structure):
    _fields_ = [("k", C.c_int32), ("L", C.c_int32), ("select_mode", C.c_int32), ("region_start", C.c_int32),
                ("weighting", C.c_int32), ("precision", C.c_int32), ("tau", C.c_float), ("margin", C.c_float),
                ("hamming_max", C.c_int32), ("feature_hash", C.c_int32), ("seed", C.c_uint64)]


class Pair(C.Structure):
    _fields_ = [("i", C.c_int32), ("j", C.c_int32), ("score", C.c_float)]


class Docs(C.Structure):
    _fields_ = [("n_docs", C.c_int64), ("offsets", C.c_void_p), ("tokens", C.c_void_p)]


class IndexInfo(C.Structure):
    _fields_ = [("n_docs", C.c_int64), ("vocab", C.c_int32), ("k", C.c_int32), ("L_used", C.c_int64),
                ("precision", C.c_int32), ("weighting", C.c_int32), ("kp", C.c_int32), ("reserved", C.c_int32)]


PAIR_DTYPE = np.dtype([("i", np.int32), ("j", np.int32), ("score", np.float32)])

# name -> (restype, argtypes); the exported symbols of include/mrc.h
_SIGNATURES = {
    "mrc_params_default": (None, [C.POINTER(Params)]),
    "mrc_ctx_create": (C.c_int32, [C.c_void_p, C.POINTER(C.c_void_p)]),
    "mrc_ctx_destroy": (None, [C.c_void_p]),
    "mrc_last_error": (C.c_char_p, [C.c_void_p]),
    "mrc_text_grams": (C.c_int32, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                   C.POINTER(C.c_int64)]),
    "mrc_simhash_index_build": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_void_p)]),
    "mrc_simhash_index_match": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                            C.c_int64, C.POINTER(C.c_int64)]),
    "mrc_simhash_index_free": (None, [C.c_void_p]),
    "mrc_build_index": (C.c_int32, [C.c_void_p, C.POINTER(Docs), C.c_int32, C.POINTER(Params), C.POINTER(C.c_void_p)]),
    "mrc_signature": (C.c_int32, [C.c_void_p, C.c_void_p, C.POINTER(Docs), C.c_void_p, C.c_void_p]),
    "mrc_signature_noalloc": (C.c_int32, [C.c_void_p, C.c_void_p, C.POINTER(Docs), C.c_void_p, C.c_void_p]),
    "mrc_match": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_void_p, C.c_int64,
                              C.POINTER(C.c_int64)]),
    "cosine_allpairs": (C.c_int32, [C.c_void_p, C.c_void_p, C.POINTER(Docs), C.c_float, C.c_void_p, C.c_int64,
                                    C.POINTER(C.c_int64)]),
    "simhash_match": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                  C.c_int64, C.POINTER(C.c_int64)]),
    "mrc_match_async": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_float, C.c_void_p,
                                    C.c_int64, C.c_void_p]),
    "cosine_allpairs_async": (C.c_int32, [C.c_void_p, C.c_void_p, C.POINTER(Docs), C.c_float, C.c_void_p,
                                          C.c_int64, C.c_void_p]),
    "simhash_match_async": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_int32,
                                        C.c_void_p, C.c_int64, C.c_void_p]),
    "mrc_ctx_sync": (C.c_int32, [C.c_void_p]),
    "mrc_index_get_info": (C.c_int32, [C.c_void_p, C.POINTER(IndexInfo)]),
    "mrc_index_export": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p]),
    "mrc_index_save": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_char_p]),
    "mrc_index_load": (C.c_int32, [C.c_void_p, C.c_char_p, C.POINTER(C.c_void_p)]),
    "mrc_index_free": (None, [C.c_void_p]),
    "mrc_ctx_set_timing": (C.c_int32, [C.c_void_p, C.c_int32]),
    "mrc_ctx_set_wait_limit": (C.c_int32, [C.c_void_p, C.c_int64]),
    "mrc_ctx_set_test_stall": (C.c_int32, [C.c_void_p, C.c_int32]),
    "mrc_ctx_set_rescoring": (C.c_int32, [C.c_void_p, C.c_int32]),
    "mrc_measure_popc_rate": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "mrc_measure_smem_atomic_rate": (C.c_int32, [C.c_void_p, C.c_void_p]),
    "mrc_ctx_kernel_stat": (C.c_int32, [C.c_void_p, C.c_int32, C.c_char_p, C.POINTER(C.c_int64),
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "mrc_ctx_reset_stats": (None, [C.c_void_p]),
    "mrc_batch_create": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_float, C.c_int64, C.c_int32,
                                     C.POINTER(C.c_void_p)]),
    "mrc_batch_launch": (C.c_int32, [C.c_void_p, C.POINTER(Docs)]),
    "mrc_batch_poll": (C.c_int32, [C.c_void_p]),
    "mrc_batch_wait": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]),
    "mrc_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "mrc_batch_attach_simhash": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int64]),
    "mrc_batch_hamming": (C.c_int32, [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]),
    "mrc_batch_free": (None, [C.c_void_p]),
    "mrc_batch_tune": (C.c_int32, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32]),
    "mrc_batch_kernels": (C.c_int32, [C.c_void_p]),
    "mrc_batch_phase_ns": (C.c_int32, [C.c_void_p, C.c_void_p]),
}

_LIB = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libmrc.so (built by ``__graft_entry__.build()``); raises if it is absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def exported_symbols():
    return sorted(_SIGNATURES)


# ---------------------------------------------------------------------------- marshalling
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check_dtype(x, np_dtype, torch_name):
    if x is None:
        return
    if _is_torch(x):
        if str(x.dtype) != f"torch.{torch_name}":
            raise TypeError(f"expected torch.{torch_name}, got {x.dtype}")
    elif x.dtype != np_dtype:
        raise TypeError(f"expected {np_dtype}, got {x.dtype}")


def _docs(offsets, tokens):
    _check_dtype(offsets, np.int64, "int64")
    _check_dtype(tokens, np.int32, "int32")
    n = int(offsets.shape[0]) - 1
    return Docs(n, _ptr(offsets), _ptr(tokens))


def _on_device(x):
    return _is_torch(x) and x.is_cuda


class Context:
    """A library context bound to the current device and a CUDA stream (torch's current stream by default)."""

    def __init__(self, stream=None):
        self.lib = load_library()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        h = C.c_void_p()
        st = self.lib.mrc_ctx_create(C.c_void_p(stream), C.byref(h))
        if st != MRC_OK:
            raise MrcError(st, "mrc_ctx_create failed (needs a Blackwell sm_103a device)")
        self.handle = h
        self.stream = stream

    def check(self, st):
        if st != MRC_OK:
            raise MrcError(st, self.last_error())

    def sync(self):
        """Wait for the context's stream; raise a device-side error of the stream-ordered calls."""
        self.check(self.lib.mrc_ctx_sync(self.handle))

    def last_error(self) -> str:
        return self.lib.mrc_last_error(self.handle).decode()

    def set_timing(self, on: bool = True):
        self.check(self.lib.mrc_ctx_set_timing(self.handle, 1 if on else 0))

    def set_wait_limit(self, ns: int):
        """Bound of every device-side wait of this context's kernels (nanoseconds)."""
        self.check(self.lib.mrc_ctx_set_wait_limit(self.handle, int(ns)))

    def popc_rate(self) -> float:
        """Measured 32-bit POPC issue rate of this context's device (per second)."""
        out = C.c_double()
        self.check(self.lib.mrc_measure_popc_rate(self.handle, C.byref(out)))
        return out.value

    def smem_atomic_rate(self) -> float:
        """Measured rate of 64-bit shared-memory atomic adds of this context's device (per second)."""
        out = C.c_double()
        self.check(self.lib.mrc_measure_smem_atomic_rate(self.handle, C.byref(out)))
        return out.value

    def set_rescoring(self, on: bool):
        """Off: mrc_match returns the compare's candidates with the compare's own cosine (diagnostics)."""
        self.check(self.lib.mrc_ctx_set_rescoring(self.handle, 1 if on else 0))

    def set_test_stall(self, on: bool):
        """Failure-detection test: this context's compare kernels issue no MMA, so their waits run out."""
        self.check(self.lib.mrc_ctx_set_test_stall(self.handle, 1 if on else 0))

    def kernel_stats(self):
        out = []
        n = self.lib.mrc_ctx_kernel_stat(self.handle, -1, None, None, None, None, None)
        for s in range(max(n, 0)):
            name = C.create_string_buffer(64)
            la, ms, by, fl = C.c_int64(), C.c_double(), C.c_double(), C.c_double()
            self.lib.mrc_ctx_kernel_stat(self.handle, s, name, C.byref(la), C.byref(ms), C.byref(by), C.byref(fl))
            out.append({"name": name.value.decode(), "launches": la.value, "ms": ms.value, "bytes": by.value,
                        "flops": fl.value})
        return out

    def reset_stats(self):
        self.lib.mrc_ctx_reset_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            self.lib.mrc_ctx_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class Index:
    def __init__(self, ctx: Context, handle):
        self.ctx = ctx
        self.handle = handle
        info = IndexInfo()
        ctx.check(ctx.lib.mrc_index_get_info(handle, C.byref(info)))
        self.n_docs, self.vocab, self.k = info.n_docs, info.vocab, info.k
        self.L_used, self.precision, self.weighting, self.kp = info.L_used, info.precision, info.weighting, info.kp

    def free(self):
        if self.handle:
            self.ctx.lib.mrc_index_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


def _pinned_pairs(n: int) -> np.ndarray:
    """A host pair array in page-locked memory (device-to-host copies into it run at full speed).
    The array is a view of a pinned torch tensor, which numpy keeps alive as the view's base."""
    import torch
    try:
        t = torch.empty(max(n, 1) * PAIR_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
    except RuntimeError:  # no device to pin for: plain host memory
        return np.empty(max(n, 1), PAIR_DTYPE)
    return t.numpy().view(PAIR_DTYPE)


class Batch:
    """A graph-captured query pipeline (mrc_batch_*): up to max_docs new documents per launch,
    compared against every document of `index`."""

    def __init__(self, ctx: Context, index: Index, max_docs: int, max_tokens: int, tau: float = 0.9,
                 capacity: int = 1 << 18, tile_n: int = 0):
        self.ctx, self.index = ctx, index
        self.max_docs, self.max_tokens, self.capacity, self.tile_n = max_docs, max_tokens, capacity, tile_n
        h = C.c_void_p()
        ctx.check(ctx.lib.mrc_batch_create(ctx.handle, index.handle, int(max_docs), int(max_tokens), float(tau),
                                           int(capacity), int(tile_n), C.byref(h)))
        self.handle = h
        self._keep = None

    def _check(self, st):
        if st != MRC_OK:
            raise MrcError(st, self.ctx.lib.mrc_batch_last_error(self.handle).decode())

    def launch(self, offsets, tokens):
        """Asynchronous: copy the batch in (host or device buffers) and launch the graph."""
        d = _docs(offsets, tokens)
        self._keep = (offsets, tokens)  # the copies are stream-ordered: keep the inputs alive
        self._check(self.ctx.lib.mrc_batch_launch(self.handle, C.byref(d)))

    def poll(self) -> bool:
        return bool(self.ctx.lib.mrc_batch_poll(self.handle))

    def tune(self, tile_n: int = 0, ring: int = 0, prefetch: int = -1):
        """Set the compare's tile width, streamed-operand ring depth and L2 prefetch distance
        (mrc_batch_tune; re-captures the graph)."""
        self._check(self.ctx.lib.mrc_batch_tune(self.handle, int(tile_n), int(ring), int(prefetch)))
        self.tile_n = int(tile_n)

    def phase_ns(self) -> dict:
        """Phase durations (ns) of the persistent kernel's last launch (mrc_batch_phase_ns)."""
        out = np.zeros(6, np.int64)
        self._check(self.ctx.lib.mrc_batch_phase_ns(self.handle, out.ctypes.data))
        return dict(zip(("list", "signature", "compare", "rescore_probe", "scan", "scatter"), out.tolist()))

    @property
    def kernel_nodes(self) -> int:
        """Kernel nodes of the captured graph (mrc_batch_kernels): 1 with the persistent kernel."""
        return int(self.ctx.lib.mrc_batch_kernels(self.handle))

    def wait(self, out=None, offsets=False):
        """Wait for the last launch; returns (pairs grouped by query position, total) and, with
        offsets=True, also the [n + 1] start of each query's pairs. Without `out` the pairs land
        in a buffer owned by this object and a copy of them is returned."""
        own = out is None
        if own:
            if getattr(self, "_out", None) is None:
                self._out = _pinned_pairs(self.capacity)
            buf = self._out
        else:
            buf = out
        n = 0 if self._keep is None else int(self._keep[0].shape[0]) - 1
        self._last_n = n
        qoff = np.zeros(n + 1, np.int64)
        total = C.c_int64()
        st = self.ctx.lib.mrc_batch_wait(self.handle, _ptr(buf), int(buf.shape[0]), C.byref(total),
                                         qoff.ctypes.data if offsets else None)
        self._keep = None
        self._check(st)
        m = min(int(total.value), buf.shape[0])
        pairs = buf[:m].copy() if own else buf[:m]
        return (pairs, int(total.value), qoff) if offsets else (pairs, int(total.value))

    def totals(self):
        """Wait for the last launch and return its (signature pair, Hamming pair) totals without
        copying pairs (errors are raised as by wait); the pairs can then be copied with wait() /
        hamming() until the next launch."""
        t = C.c_int64()
        self._check(self.ctx.lib.mrc_batch_wait(self.handle, None, 0, C.byref(t), None))
        h = C.c_int64(0)
        if getattr(self, "h_capacity", None):
            self._check(self.ctx.lib.mrc_batch_hamming(self.handle, None, 0, C.byref(h), None))
        return int(t.value), int(h.value)

    def attach_simhash(self, shindex: "SimhashIndex", hamming_max: int | None = None, capacity: int = 1 << 16):
        """Add the Hamming leg: each launch also probes `shindex` with the batch's Simhashes."""
        hm = shindex.hamming_max if hamming_max is None else int(hamming_max)
        self._check(self.ctx.lib.mrc_batch_attach_simhash(self.handle, shindex.handle, hm, int(capacity)))
        self.h_capacity = int(capacity)
        self._shindex = shindex  # the batch keeps the fingerprint index in use

    def hamming(self, out=None, offsets=False):
        """After wait(): the last launch's Hamming pairs (query position, index position, distance),
        grouped by query; with offsets=True also where each query's pairs start. Without `out`
        the pairs land in a buffer owned by this object and a copy of them is returned."""
        n = getattr(self, "_last_n", 0)
        own = out is None
        if own:
            if getattr(self, "_hout", None) is None:
                self._hout = _pinned_pairs(self.h_capacity)
            buf = self._hout
        else:
            buf = out
        qoff = np.zeros(n + 1, np.int64)
        total = C.c_int64()
        self._check(self.ctx.lib.mrc_batch_hamming(self.handle, _ptr(buf), int(buf.shape[0]),
                                                   C.byref(total), qoff.ctypes.data if offsets else None))
        m = min(int(total.value), buf.shape[0])
        pairs = buf[:m].copy() if own else buf[:m]
        return (pairs, int(total.value), qoff) if offsets else (pairs, int(total.value))

    def free(self):
        if getattr(self, "handle", None):
            self.ctx.lib.mrc_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


def params_default(**kw) -> Params:
    p = Params()
    load_library().mrc_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def mrc_text_grams(ctx: Context, text_offsets, text, gram_offsets=None, grams=None):
    """Character 3-grams of raw text: (gram_offsets int64 [n+1], grams int32 [total]) on the
    inputs' side (torch CUDA tensors, or numpy arrays). text: uint8 bytes (numpy/torch) or a
    bytes object; caller buffers, when given, must hold n+1 offsets and n_bytes ids."""
    if isinstance(text, (bytes, bytearray)):
        text = np.frombuffer(text, np.uint8)
    _check_dtype(text_offsets, np.int64, "int64")
    _check_dtype(text, np.uint8, "uint8")
    n = int(text_offsets.shape[0]) - 1
    n_bytes = int(text.shape[0])
    if gram_offsets is None:
        if _on_device(text_offsets):
            import torch
            gram_offsets = torch.empty(n + 1, dtype=torch.int64, device=text_offsets.device)
            grams = torch.empty(max(n_bytes, 1), dtype=torch.int32, device=text_offsets.device)
        else:
            gram_offsets = np.empty(n + 1, np.int64)
            grams = np.empty(max(n_bytes, 1), np.int32)
    total = C.c_int64()
    ctx.check(ctx.lib.mrc_text_grams(ctx.handle, n, _ptr(text_offsets), _ptr(text), _ptr(gram_offsets), _ptr(grams),
                                     int(grams.shape[0]), C.byref(total)))
    return gram_offsets, grams[:total.value]


def mrc_build_index(ctx: Context, offsets, tokens, vocab: int, params: Params | None = None) -> Index:
    params = params or params_default()
    d = _docs(offsets, tokens)
    h = C.c_void_p()
    ctx.check(ctx.lib.mrc_build_index(ctx.handle, C.byref(d), int(vocab), C.byref(params), C.byref(h)))
    return Index(ctx, h)


def mrc_signature(ctx: Context, index: Index, offsets, tokens, sig=None, simhash=None, want_simhash=True):
    """Signatures [n, k] float32 (and Simhash [n] uint64) of new documents; outputs on the inputs' side."""
    n = int(offsets.shape[0]) - 1
    if sig is None:
        if _on_device(tokens):
            import torch
            sig = torch.empty((n, index.k), dtype=torch.float32, device=tokens.device)
            simhash = torch.empty(n, dtype=torch.int64, device=tokens.device) if want_simhash else None
        else:
            sig = np.empty((n, index.k), np.float32)
            simhash = np.empty(n, np.uint64) if want_simhash else None
    d = _docs(offsets, tokens)
    ctx.check(ctx.lib.mrc_signature(ctx.handle, index.handle, C.byref(d), _ptr(sig), _ptr(simhash)))
    return sig, simhash


def mrc_signature_noalloc(ctx: Context, index: Index, offsets, tokens, sig, simhash=None):
    """Signatures into caller-provided device tensors without any device allocation
    (at most NOALLOC_MAX_DOCS documents; every buffer must be device memory)."""
    d = _docs(offsets, tokens)
    ctx.check(ctx.lib.mrc_signature_noalloc(ctx.handle, index.handle, C.byref(d), _ptr(sig), _ptr(simhash)))
    return sig, simhash


NOALLOC_MAX_DOCS = 65536


def _pairs_buf(capacity, device):
    if device is not None:
        import torch
        return torch.empty((max(capacity, 1), 3), dtype=torch.int32, device=device)
    return np.empty(max(capacity, 1), PAIR_DTYPE)


def _pair_call(ctx, fn, capacity, device, grow):
    while True:
        buf = _pairs_buf(capacity, device)
        total = C.c_int64()
        st = fn(buf, capacity, total)
        if st == MRC_ERR_CAPACITY and grow:
            capacity = int(total.value)
            continue
        if st not in (MRC_OK, MRC_ERR_CAPACITY):
            ctx.check(st)
        m = min(int(total.value), capacity)
        return buf[:m], int(total.value)


def pairs_to_numpy(buf):
    """Pairs from a device [m, 3] int32 tensor or a host structured array -> structured numpy array."""
    if isinstance(buf, np.ndarray):
        return buf
    arr = buf.cpu().numpy()
    out = np.empty(arr.shape[0], PAIR_DTYPE)
    out["i"] = arr[:, 0]
    out["j"] = arr[:, 1]
    out["score"] = arr[:, 2].view(np.float32)
    return out


def mrc_match(ctx: Context, index: Index, query_sig=None, tau: float = 0.9, capacity: int = 1 << 20,
              device="cuda", grow=True):
    """Signature pairs with cosine >= tau: all index pairs (query_sig None) or queries x index."""
    nq = 0 if query_sig is None else int(query_sig.shape[0])
    if query_sig is not None:
        _check_dtype(query_sig, np.float32, "float32")

    def fn(buf, cap, total):
        return ctx.lib.mrc_match(ctx.handle, index.handle, _ptr(query_sig), nq, float(tau), _ptr(buf), cap,
                                 C.byref(total))
    return _pair_call(ctx, fn, capacity, device, grow)


def cosine_allpairs(ctx: Context, index: Index, offsets, tokens, tau: float = 0.9, capacity: int = 1 << 20,
                    device="cuda", grow=True):
    """Exact TF-IDF cosine pairs >= tau over all pairs of the given documents."""
    d = _docs(offsets, tokens)

    def fn(buf, cap, total):
        return ctx.lib.cosine_allpairs(ctx.handle, index.handle, C.byref(d), float(tau), _ptr(buf), cap,
                                       C.byref(total))
    return _pair_call(ctx, fn, capacity, device, grow)


def simhash_match(ctx: Context, a, b=None, hamming_max: int = 3, capacity: int = 1 << 20, device="cuda", grow=True):
    """Fingerprint pairs with Hamming distance <= hamming_max (all pairs of a, or a x b)."""
    na = int(a.shape[0])
    nb = 0 if b is None else int(b.shape[0])

    def fn(buf, cap, total):
        return ctx.lib.simhash_match(ctx.handle, _ptr(a), na, _ptr(b), nb, int(hamming_max), _ptr(buf), cap,
                                     C.byref(total))
    return _pair_call(ctx, fn, capacity, device, grow)


class SimhashIndex:
    """Block-table Hamming index over 64-bit fingerprints (mrc_simhash_index_*)."""

    def __init__(self, ctx: Context, handle, n: int, hamming_max: int):
        self.ctx, self.handle, self.n, self.hamming_max = ctx, handle, n, hamming_max

    def free(self):
        if self.handle:
            self.ctx.lib.mrc_simhash_index_free(self.handle)
            self.handle = None


def simhash_index_build(ctx: Context, fps, hamming_max: int = 3) -> SimhashIndex:
    n = int(fps.shape[0])
    h = C.c_void_p()
    ctx.check(ctx.lib.mrc_simhash_index_build(ctx.handle, _ptr(fps), n, int(hamming_max), C.byref(h)))
    return SimhashIndex(ctx, h, n, hamming_max)


def simhash_index_match(ctx: Context, index: SimhashIndex, queries=None, hamming_max: int | None = None,
                        capacity: int = 1 << 20, device="cuda", grow=True):
    """Pairs (query, index position) within hamming_max (default: the build's), or all pairs i < j
    of the index when queries is None; the same pairs as simhash_match."""
    nq = 0 if queries is None else int(queries.shape[0])
    hm = index.hamming_max if hamming_max is None else int(hamming_max)

    def fn(buf, cap, total):
        return ctx.lib.mrc_simhash_index_match(ctx.handle, index.handle, _ptr(queries), nq, hm, _ptr(buf), cap,
                                               C.byref(total))
    return _pair_call(ctx, fn, capacity, device, grow)


def _async_out(pairs, count):
    import torch
    if not (_is_torch(pairs) and pairs.is_cuda and pairs.dtype == torch.int32 and pairs.dim() == 2
            and pairs.shape[1] == 3 and pairs.is_contiguous()):
        raise TypeError("pairs must be a contiguous CUDA int32 tensor of shape [capacity, 3]")
    if not (_is_torch(count) and count.is_cuda and count.dtype == torch.int64 and count.numel() >= 1):
        raise TypeError("count must be a CUDA int64 tensor")
    return int(pairs.shape[0]), _ptr(count)


def mrc_match_async(ctx: Context, index: Index, pairs, count, query_sig=None, tau: float = 0.9):
    """Stream-ordered mrc_match: writes up to pairs.shape[0] pairs and count[0] = total; no wait."""
    cap, pc = _async_out(pairs, count)
    nq = 0 if query_sig is None else int(query_sig.shape[0])
    if query_sig is not None:
        _check_dtype(query_sig, np.float32, "float32")
    ctx.check(ctx.lib.mrc_match_async(ctx.handle, index.handle, _ptr(query_sig), nq, float(tau), _ptr(pairs), cap,
                                      pc))


def cosine_allpairs_async(ctx: Context, index: Index, offsets, tokens, pairs, count, tau: float = 0.9):
    """Stream-ordered cosine_allpairs (one wait, after the head/tail split is known)."""
    cap, pc = _async_out(pairs, count)
    d = _docs(offsets, tokens)
    ctx.check(ctx.lib.cosine_allpairs_async(ctx.handle, index.handle, C.byref(d), float(tau), _ptr(pairs), cap, pc))


def simhash_match_async(ctx: Context, a, pairs, count, b=None, hamming_max: int = 3):
    """Stream-ordered simhash_match."""
    cap, pc = _async_out(pairs, count)
    na = int(a.shape[0])
    nb = 0 if b is None else int(b.shape[0])
    ctx.check(ctx.lib.simhash_match_async(ctx.handle, _ptr(a), na, _ptr(b), nb, int(hamming_max), _ptr(pairs), cap,
                                          pc))


def mrc_index_export(ctx: Context, index: Index):
    """Host copies of the index: raw signatures, Simhash, df, idf, partitions, reference norms."""
    n, k, V = index.n_docs, index.k, index.vocab
    sig = np.empty((n, k), np.float32)
    sh = np.empty(n, np.uint64)
    df = np.empty(V, np.int32)
    idf = np.empty(V, np.float32)
    part = np.empty(V, np.int32)
    rnorm = np.empty(k, np.float64)
    ctx.check(ctx.lib.mrc_index_export(ctx.handle, index.handle, _ptr(sig), _ptr(sh), _ptr(df), _ptr(idf),
                                       _ptr(part), _ptr(rnorm)))
    return {"sig": sig, "simhash": sh, "df": df, "idf": idf, "part": part, "rnorm": rnorm}


def index_simhash(ctx: Context, index: Index, out):
    """The index's Simhash fingerprints copied into ``out`` (device or host, 8 bytes per document)."""
    ctx.check(ctx.lib.mrc_index_export(ctx.handle, index.handle, None, _ptr(out), None, None, None, None))
    return out


def mrc_index_save(ctx: Context, index: Index, path: str):
    ctx.check(ctx.lib.mrc_index_save(ctx.handle, index.handle, path.encode()))


def mrc_index_load(ctx: Context, path: str) -> Index:
    h = C.c_void_p()
    ctx.check(ctx.lib.mrc_index_load(ctx.handle, path.encode(), C.byref(h)))
    return Index(ctx, h)
