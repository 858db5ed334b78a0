"""Shared pieces of the GPU parity tests: corpora, the oracle side, pair-set comparison."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1810_03099_gb300 import synth


def cuda_or_skip():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def concat(*parts):
    """Concatenate token-CSR corpora given as (offsets, tokens)."""
    offs = [np.zeros(1, np.int64)]
    toks = []
    base = 0
    for o, t in parts:
        offs.append(o[1:] + base)
        toks.append(t)
        base += int(o[-1])
    return np.concatenate(offs), np.concatenate(toks).astype(np.int32)


def csr(docs):
    o = np.zeros(len(docs) + 1, np.int64)
    o[1:] = np.cumsum([len(d) for d in docs])
    t = np.array([x for d in docs for x in d], np.int32) if o[-1] else np.zeros(0, np.int32)
    return o, t


def edge_docs(vocab, seed=3):
    """Degenerate documents: empty, one token, one repeated token, two tokens, a long repeat."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = [int(x) for x in rng.integers(0, vocab, size=8)]
    return [[], [t[0]], [t[1]] * 7, [t[2], t[3]], [t[4]] * 3000, [t[5], t[6], t[6], t[7]] * 200]


def mixed_corpus(n_tiny=600, n_long=24, vocab=5000, seed=None):
    """Short lognormal documents, long log-uniform ones (20..20,000 tokens) and edge cases, mixed."""
    a = synth.make_corpus(synth.SPECS["tiny"].with_(n_docs=n_tiny, vocab=vocab, **({"seed": seed} if seed else {})))
    b = synth.make_corpus(synth.SPECS["batch_queries"].with_(n_docs=n_long, vocab=vocab))
    e = csr(edge_docs(vocab))
    return concat((a.offsets, a.tokens), e, (b.offsets, b.tokens))


def pair_dict(i, j, s):
    return {(int(a), int(b)): float(c) for a, b, c in zip(i, j, s)}


def compare_pairs(gpu, ref, tau, band, score_tol, ref_score=None):
    """gpu, ref: {(i, j): score}. Pairs present on one side only must lie within `band` of tau
    (by the reference score); common pairs must agree within score_tol. Returns a report dict."""
    missing = [p for p in ref if p not in gpu]
    extra = [p for p in gpu if p not in ref]
    bad_missing = [p for p in missing if abs(ref[p] - tau) > band]
    bad_extra = []
    for p in extra:
        s = ref_score(*p) if ref_score else None
        if s is None or abs(s - tau) > band:
            bad_extra.append((p, gpu[p], s))
    worst = 0.0
    for p, s in gpu.items():
        if p in ref:
            worst = max(worst, abs(s - ref[p]))
    assert not bad_missing, f"{len(bad_missing)} pairs missing, e.g. {bad_missing[:5]}"
    assert not bad_extra, f"{len(bad_extra)} extra pairs, e.g. {bad_extra[:5]}"
    assert worst <= score_tol, f"score error {worst} > {score_tol}"
    return {"missing": len(missing), "extra": len(extra), "worst": worst, "n": len(ref)}
