"""Python face of the FP64 C oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
use this module. It loads ``oracle/_build/libmrc_oracle.so`` (plain C, double
precision, built from ``mrc_oracle.c``) and strings its functions together in
the order the paper describes the method (Sections III-V):

  token CSR -> term counts -> df -> idf -> weights -> reference partitions
  -> signatures (cosine to each partition) -> signature cosine -> pairs,
  plus the two rivals: exact cosine of the weight vectors, and Simhash with
  Hamming distance.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

MODE_ALL, MODE_REGION, MODE_DF1 = 0, 1, 2
HASH_SPLITMIX64, HASH_MD5, HASH_SHA1 = 0, 1, 2
GRAM_VOCAB = 26 ** 3  # character 3-grams over the case-folded 26-letter alphabet
WEIGHT_COUNT, WEIGHT_TFIDF = 0, 1

_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_vp = C.c_void_p


def _sig(lib):
    i64, i32, f64, u64 = C.c_int64, C.c_int32, C.c_double, C.c_uint64
    spec = {
        "orc_char3grams": (i64, [i64, _i64p, _u8p, _i64p, _i32p]),
        "orc_term_counts": (i64, [i64, _i64p, _i32p, _i64p, _i32p, _i32p]),
        "orc_df": (None, [i64, _i64p, _i32p, i32, _i64p]),
        "orc_idf": (None, [i64, i32, _i64p, _f64p]),
        "orc_weights": (None, [i64, _i32p, _i32p, _vp, _f64p]),
        "orc_select_refs": (i64, [i32, i64, _i64p, i32, i64, i64, i32, _i32p]),
        "orc_ref_norms": (None, [i32, _i32p, i32, _vp, _f64p]),
        "orc_signatures": (None, [i64, _i64p, _i32p, _f64p, _i32p, _vp, _f64p, i32, _f64p]),
        "orc_cos_dense": (f64, [_f64p, _f64p, i32]),
        "orc_cosine_pair": (f64, [_i64p, _i32p, _f64p, i64, i64]),
        "orc_sig_pairs": (i64, [_f64p, i64, i32, f64, _i32p, _i32p, _f64p, i64]),
        "orc_sig_match": (i64, [_f64p, i64, _f64p, i64, i32, f64, _i32p, _i32p, _f64p, i64]),
        "orc_cosine_pairs": (i64, [i64, _i64p, _i32p, _f64p, f64, _i32p, _i32p, _f64p, i64]),
        "orc_splitmix64": (u64, [u64]),
        "orc_term_hash": (u64, [i32, u64]),
        "orc_md5": (None, [_vp, i64, _u8p]),
        "orc_sha1": (None, [_vp, i64, _u8p]),
        "orc_feature_hash": (u64, [i32, u64, i32]),
        "orc_simhash": (None, [i64, _i64p, _i32p, u64, i32, _u64p]),
        "orc_hamming": (i32, [u64, u64]),
        "orc_hamming_pairs": (i64, [_u64p, i64, _vp, i64, i32, _i32p, _i32p, _i32p, i64]),
        "orc_error_stats": (None, [_f64p, _f64p, i64, _f64p]),
        "orc_round_bf16": (f64, [f64]),
        "orc_idf_bf16": (None, [i32, _f64p, _f64p]),
    }
    for name, (res, args) in spec.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIBS: dict[str, C.CDLL] = {}


def load(path: str | None = None) -> C.CDLL:
    """Load (building first if needed) the oracle library; ``path`` selects another build."""
    if path is None:
        path = _build.build()
    path = os.path.abspath(path)
    if path not in _LIBS:
        _LIBS[path] = _sig(C.CDLL(path))
    return _LIBS[path]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """Thin wrappers over the C functions (numpy in, numpy out)."""

    def __init__(self, lib_path: str | None = None):
        self.lib = load(lib_path)

    # ---- Section III: vector space model -------------------------------------------------
    def term_counts(self, offsets, tokens):
        offsets = np.ascontiguousarray(offsets, np.int64)
        tokens = np.ascontiguousarray(tokens, np.int32)
        n = offsets.shape[0] - 1
        cap = max(1, int(offsets[-1]))
        row_ptr = np.zeros(n + 1, np.int64)
        terms = np.zeros(cap, np.int32)
        counts = np.zeros(cap, np.int32)
        nnz = self.lib.orc_term_counts(n, offsets, tokens, row_ptr, terms, counts)
        return row_ptr, terms[:nnz].copy(), counts[:nnz].copy()

    def df(self, row_ptr, terms, vocab):
        out = np.zeros(vocab, np.int64)
        self.lib.orc_df(row_ptr.shape[0] - 1, row_ptr, np.ascontiguousarray(terms, np.int32), vocab, out)
        return out

    def idf(self, n_docs, df):
        df = np.ascontiguousarray(df, np.int64)
        out = np.zeros(df.shape[0], np.float64)
        self.lib.orc_idf(n_docs, df.shape[0], df, out)
        return out

    def round_bf16(self, x):
        return self.lib.orc_round_bf16(float(x))

    def idf_bf16(self, idf):
        idf = _c64(idf)
        out = np.zeros_like(idf)
        self.lib.orc_idf_bf16(idf.shape[0], idf, out)
        return out

    def weights(self, terms, counts, idf=None):
        out = np.zeros(terms.shape[0], np.float64)
        idf = None if idf is None else _c64(idf)
        self.lib.orc_weights(terms.shape[0], terms, counts, _ptr(idf), out)
        return out

    # ---- Section IV: references and signatures -----------------------------------------
    def select_refs(self, df, n_docs, mode, L, start, k):
        df = np.ascontiguousarray(df, np.int64)
        part = np.zeros(df.shape[0], np.int32)
        used = self.lib.orc_select_refs(df.shape[0], n_docs, df, mode, L, start, k, part)
        if used < 0:
            raise ValueError("invalid reference selection")
        return part, int(used)

    def ref_norms(self, part, k, idf=None):
        out = np.zeros(k, np.float64)
        idf = None if idf is None else _c64(idf)
        self.lib.orc_ref_norms(part.shape[0], part, k, _ptr(idf), out)
        return out

    def signatures(self, row_ptr, terms, w, part, idf, rnorm, k):
        n = row_ptr.shape[0] - 1
        out = np.zeros((n, k), np.float64)
        idf = None if idf is None else _c64(idf)
        self.lib.orc_signatures(n, row_ptr, terms, _c64(w), part, _ptr(idf), _c64(rnorm), k, out)
        return out

    def cos_dense(self, a, b):
        a, b = _c64(a), _c64(b)
        return self.lib.orc_cos_dense(a, b, a.shape[0])

    def sig_pairs(self, S, tau, cap=None):
        S = _c64(S)
        n, k = S.shape
        if cap is None:
            cap = self.lib.orc_sig_pairs(S, n, k, tau, np.zeros(1, np.int32), np.zeros(1, np.int32),
                                         np.zeros(1, np.float64), 0)
        pi, pj, ps = np.zeros(max(cap, 1), np.int32), np.zeros(max(cap, 1), np.int32), np.zeros(max(cap, 1))
        tot = self.lib.orc_sig_pairs(S, n, k, tau, pi, pj, ps, cap)
        m = min(tot, cap)
        return tot, pi[:m], pj[:m], ps[:m]

    def sig_match(self, Q, X, tau, cap=None):
        Q, X = _c64(Q), _c64(X)
        z = (np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.float64))
        if cap is None:
            cap = self.lib.orc_sig_match(Q, Q.shape[0], X, X.shape[0], Q.shape[1], tau, *z, 0)
        pi, pj, ps = np.zeros(max(cap, 1), np.int32), np.zeros(max(cap, 1), np.int32), np.zeros(max(cap, 1))
        tot = self.lib.orc_sig_match(Q, Q.shape[0], X, X.shape[0], Q.shape[1], tau, pi, pj, ps, cap)
        m = min(tot, cap)
        return tot, pi[:m], pj[:m], ps[:m]

    # ---- Eq. 1 on the weight vectors: the exact rival -----------------------------------
    def cosine_pair(self, row_ptr, terms, w, i, j):
        return self.lib.orc_cosine_pair(row_ptr, terms, _c64(w), int(i), int(j))

    def cosine_pairs(self, row_ptr, terms, w, tau, cap=None):
        n = row_ptr.shape[0] - 1
        w = _c64(w)
        z = (np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.float64))
        if cap is None:
            cap = self.lib.orc_cosine_pairs(n, row_ptr, terms, w, tau, *z, 0)
        pi, pj, ps = np.zeros(max(cap, 1), np.int32), np.zeros(max(cap, 1), np.int32), np.zeros(max(cap, 1))
        tot = self.lib.orc_cosine_pairs(n, row_ptr, terms, w, tau, pi, pj, ps, cap)
        m = min(tot, cap)
        return tot, pi[:m], pj[:m], ps[:m]

    # ---- Section III: character 3-grams ------------------------------------------------
    def char3grams(self, text_offsets, text):
        """(gram_offsets [n+1] int64, grams [G] int32) of a text CSR (bytes as uint8)."""
        text_offsets = np.ascontiguousarray(text_offsets, np.int64)
        text = np.frombuffer(text, np.uint8) if isinstance(text, (bytes, bytearray)) else np.asarray(text, np.uint8)
        padded = np.zeros(text.shape[0] + 2, np.uint8)  # two zero bytes after the text
        padded[:text.shape[0]] = text
        n = text_offsets.shape[0] - 1
        go = np.zeros(n + 1, np.int64)
        grams = np.zeros(max(int(text_offsets[-1]), 1), np.int32)
        g = self.lib.orc_char3grams(n, text_offsets, padded, go, grams)
        return go, grams[:g]

    # ---- Section III: Simhash ------------------------------------------------------------
    def splitmix64(self, state):
        return int(self.lib.orc_splitmix64(C.c_uint64(int(state) & (2**64 - 1))))

    def term_hash(self, t, seed):
        return int(self.lib.orc_term_hash(int(t), C.c_uint64(int(seed) & (2**64 - 1))))

    def md5(self, msg: bytes) -> bytes:
        out = np.zeros(16, np.uint8)
        self.lib.orc_md5(C.c_char_p(bytes(msg)), len(msg), out)
        return out.tobytes()

    def sha1(self, msg: bytes) -> bytes:
        out = np.zeros(20, np.uint8)
        self.lib.orc_sha1(C.c_char_p(bytes(msg)), len(msg), out)
        return out.tobytes()

    def feature_hash(self, t, seed, mode):
        return int(self.lib.orc_feature_hash(int(t), C.c_uint64(int(seed) & (2**64 - 1)), int(mode)))

    def simhash(self, offsets, tokens, seed, mode=HASH_SPLITMIX64):
        offsets = np.ascontiguousarray(offsets, np.int64)
        n = offsets.shape[0] - 1
        out = np.zeros(n, np.uint64)
        self.lib.orc_simhash(n, offsets, np.ascontiguousarray(tokens, np.int32),
                             C.c_uint64(int(seed) & (2**64 - 1)), int(mode), out)
        return out

    def hamming(self, a, b):
        return int(self.lib.orc_hamming(C.c_uint64(int(a)), C.c_uint64(int(b))))

    def hamming_pairs(self, a, b, hmax, cap=None):
        a = np.ascontiguousarray(a, np.uint64)
        bb = None if b is None else np.ascontiguousarray(b, np.uint64)
        nb = 0 if bb is None else bb.shape[0]
        z = (np.zeros(1, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32))
        if cap is None:
            cap = self.lib.orc_hamming_pairs(a, a.shape[0], _ptr(bb), nb, hmax, *z, 0)
        pi, pj, ph = (np.zeros(max(cap, 1), np.int32) for _ in range(3))
        tot = self.lib.orc_hamming_pairs(a, a.shape[0], _ptr(bb), nb, hmax, pi, pj, ph, cap)
        m = min(tot, cap)
        return tot, pi[:m], pj[:m], ph[:m]

    # ---- Eq. 2 / Eq. 3 ------------------------------------------------------------------
    def error_stats(self, approx, exact):
        approx, exact = _c64(approx), _c64(exact)
        out = np.zeros(4)
        self.lib.orc_error_stats(approx, exact, approx.shape[0], out)
        return {"mae": out[0], "mean": out[1], "var": out[2], "mse": out[3]}


@dataclass
class Params:
    """Method parameters; the defaults are the readings stated in the oracle source."""
    k: int = 8
    L: int = -1  # -1: 32 * k
    mode: int = MODE_REGION
    region_start: int = -1  # -1: first rank with df <= N/100
    weighting: int = WEIGHT_TFIDF
    tau: float = 0.9
    hamming_max: int = 3
    seed: int = 0x1810030990
    bf16: bool = False  # precision form: per-term weights stored as bfloat16
    feature_hash: int = HASH_SPLITMIX64  # Simhash feature hash: HASH_SPLITMIX64, HASH_MD5 or HASH_SHA1

    @property
    def L_eff(self) -> int:
        return 32 * self.k if self.L < 0 else self.L


@dataclass
class OracleIndex:
    params: Params
    n_docs: int
    vocab: int
    df: np.ndarray
    idf: np.ndarray | None  # None under count weighting
    idf_values: np.ndarray  # idf (always computed; the index freezes it)
    part: np.ndarray
    L_used: int
    rnorm: np.ndarray
    row_ptr: np.ndarray
    terms: np.ndarray
    counts: np.ndarray
    w: np.ndarray
    S: np.ndarray
    F: np.ndarray
    extra: dict = field(default_factory=dict)


def build_index(offsets, tokens, vocab, params: Params | None = None, orc: Oracle | None = None) -> OracleIndex:
    """The whole index build in the paper's order (Sections III-IV)."""
    p = params or Params()
    o = orc or Oracle()
    n = int(np.asarray(offsets).shape[0] - 1)
    row_ptr, terms, counts = o.term_counts(offsets, tokens)
    df = o.df(row_ptr, terms, vocab)
    idf_values = o.idf(n, df)
    idf = idf_values if p.weighting == WEIGHT_TFIDF else None
    if idf is not None and p.bf16:
        idf = o.idf_bf16(idf)  # the stored weight table of the precision form
    w = o.weights(terms, counts, idf)
    part, used = o.select_refs(df, n, p.mode, p.L_eff, p.region_start, p.k)
    rnorm = o.ref_norms(part, p.k, idf)
    S = o.signatures(row_ptr, terms, w, part, idf, rnorm, p.k)
    F = o.simhash(offsets, tokens, p.seed, p.feature_hash)
    return OracleIndex(p, n, vocab, df, idf, idf_values, part, used, rnorm, row_ptr, terms, counts, w, S, F)


def signature(index: OracleIndex, offsets, tokens, orc: Oracle | None = None):
    """Signatures and Simhash of new documents against a frozen index (idf, references)."""
    o = orc or Oracle()
    p = index.params
    row_ptr, terms, counts = o.term_counts(offsets, tokens)
    w = o.weights(terms, counts, index.idf)
    S = o.signatures(row_ptr, terms, w, index.part, index.idf, index.rnorm, p.k)
    F = o.simhash(offsets, tokens, p.seed, p.feature_hash)
    return S, F, (row_ptr, terms, w)
