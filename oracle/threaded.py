"""The FP64 oracle run on several host cores, for timing it (test infrastructure only).

The oracle's C functions work document by document and row by row, so disjoint document
ranges and pair-row blocks can run at the same time: each range is one call of the same C
function, made from a thread pool (ctypes releases the interpreter lock for the call), and
the pieces are put back together in document order. No arithmetic differs from the serial
calls in ``oracle.py``: every output value is computed by the same C code on the same inputs,
which ``tests/test_oracle_threaded.py`` checks against the serial oracle.

Pair counts over all pairs i < j of n rows use query x index calls of one row block against
the rows from the block's first row on, keeping j > i; only the block's own triangle is
computed twice.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .oracle import WEIGHT_TFIDF, Oracle, OracleIndex, Params


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - non-Linux hosts
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU's model name (lscpu's, else /proc/cpuinfo's, else the architecture)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip().lower() == "model name":
                return f"{line.split(':', 1)[1].strip()} ({platform.machine()})"
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def _ranges(n, parts):
    parts = max(1, min(parts, n)) if n > 0 else 1
    cuts = [n * p // parts for p in range(parts + 1)]
    return [(cuts[p], cuts[p + 1]) for p in range(parts) if cuts[p + 1] > cuts[p]]


class ThreadedOracle:
    """The oracle's pipeline on `threads` host threads (documents and pair rows split)."""

    def __init__(self, threads: int | None = None, orc: Oracle | None = None):
        self.threads = max(1, int(threads or host_cores()))
        self.o = orc or Oracle()
        self.pool = ThreadPoolExecutor(max_workers=self.threads)

    def close(self):
        self.pool.shutdown(wait=True)

    def _map(self, fn, items):
        if self.threads == 1:
            return [fn(x) for x in items]
        return list(self.pool.map(fn, items))

    # ---- per-document stages ---------------------------------------------------------------
    def term_counts(self, offsets, tokens):
        offsets = np.ascontiguousarray(offsets, np.int64)
        tokens = np.ascontiguousarray(tokens, np.int32)
        n = offsets.shape[0] - 1
        parts = self._map(lambda r: self.o.term_counts(offsets[r[0]:r[1] + 1], tokens), _ranges(n, 4 * self.threads))
        row_ptr = np.zeros(n + 1, np.int64)
        at, d = 0, 0
        for rp, _, _ in parts:
            m = rp.shape[0] - 1
            row_ptr[d + 1:d + m + 1] = rp[1:] + at
            at += int(rp[-1])
            d += m
        terms = np.concatenate([t for _, t, _ in parts]) if parts else np.zeros(0, np.int32)
        counts = np.concatenate([c for _, _, c in parts]) if parts else np.zeros(0, np.int32)
        return row_ptr, terms, counts

    def signatures(self, row_ptr, terms, w, part, idf, rnorm, k):
        n = row_ptr.shape[0] - 1
        out = np.zeros((n, k), np.float64)

        def run(r):
            out[r[0]:r[1]] = self.o.signatures(row_ptr[r[0]:r[1] + 1], terms, w, part, idf, rnorm, k)
        self._map(run, _ranges(n, 4 * self.threads))
        return out

    def simhash(self, offsets, tokens, seed, mode):
        offsets = np.ascontiguousarray(offsets, np.int64)
        n = offsets.shape[0] - 1
        out = np.zeros(n, np.uint64)

        def run(r):
            out[r[0]:r[1]] = self.o.simhash(offsets[r[0]:r[1] + 1], tokens, seed, mode)
        self._map(run, _ranges(n, 4 * self.threads))
        return out

    def build_index(self, offsets, tokens, vocab, params: Params | None = None) -> OracleIndex:
        """oracle.build_index with its per-document stages split over the threads."""
        p = params or Params()
        o = self.o
        n = int(np.asarray(offsets).shape[0] - 1)
        row_ptr, terms, counts = self.term_counts(offsets, tokens)
        df = o.df(row_ptr, terms, vocab)
        idf_values = o.idf(n, df)
        idf = idf_values if p.weighting == WEIGHT_TFIDF else None
        if idf is not None and p.bf16:
            idf = o.idf_bf16(idf)
        w = o.weights(terms, counts, idf)
        part, used = o.select_refs(df, n, p.mode, p.L_eff, p.region_start, p.k)
        rnorm = o.ref_norms(part, p.k, idf)
        S = self.signatures(row_ptr, terms, w, part, idf, rnorm, p.k)
        F = self.simhash(offsets, tokens, p.seed, p.feature_hash)
        return OracleIndex(p, n, vocab, df, idf, idf_values, part, used, rnorm, row_ptr, terms, counts, w, S, F)

    # ---- all pairs i < j -------------------------------------------------------------------
    def _blocks(self, n):
        # row blocks of equal pair work: block b covers rows whose remaining-pair counts sum to
        # about 1 / parts of the triangle
        parts = max(1, 8 * self.threads)
        rem = np.arange(n, 0, -1, dtype=np.float64)  # pairs of row i with rows from i on
        cum = np.concatenate([[0.0], np.cumsum(rem)])
        cuts = np.searchsorted(cum, np.linspace(0, cum[-1], parts + 1)).tolist()
        cuts[0], cuts[-1] = 0, n
        return [(a, b) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]

    def sig_pairs(self, S, tau):
        """(total, i, j, score) of all pairs i < j with signature cosine >= tau, in (i, j) order."""
        S = np.ascontiguousarray(S, np.float64)
        n = S.shape[0]

        def run(r):
            a, b = r
            _, qi, xj, sc = self.o.sig_match(S[a:b], S[a:], tau)
            gi, gj = qi.astype(np.int64) + a, xj.astype(np.int64) + a
            keep = gj > gi
            return gi[keep], gj[keep], sc[keep]
        return self._gather(self._map(run, self._blocks(n)))

    def hamming_pairs(self, F, hmax):
        """(total, i, j, distance) of all pairs i < j with Hamming distance <= hmax, in (i, j) order."""
        F = np.ascontiguousarray(F, np.uint64)
        n = F.shape[0]

        def run(r):
            a, b = r
            _, qi, xj, h = self.o.hamming_pairs(F[a:b], F[a:], hmax)
            gi, gj = qi.astype(np.int64) + a, xj.astype(np.int64) + a
            keep = gj > gi
            return gi[keep], gj[keep], h[keep]
        return self._gather(self._map(run, self._blocks(n)))

    @staticmethod
    def _gather(parts):
        if not parts:
            return 0, np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0)
        gi = np.concatenate([p[0] for p in parts])
        gj = np.concatenate([p[1] for p in parts])
        sc = np.concatenate([p[2] for p in parts])
        order = np.lexsort((gj, gi))
        return int(gi.shape[0]), gi[order], gj[order], sc[order]
