"""Pure-Python brute force of the same definitions, for corpora of a few dozen documents.

Written independently of ``mrc_oracle.c`` (dicts, ``math``, Python integers) so
that the two can be checked against each other. Test infrastructure only.
"""
from __future__ import annotations

import hashlib
import math
import re
from collections import Counter

MASK64 = (1 << 64) - 1


def char3grams(doc: bytes):
    """3-gram ids of one document: letter runs found by a regular expression, lower-cased,
    every window of three letters numbered in base 26."""
    out = []
    for run in re.findall(rb"[A-Za-z]+", doc):
        run = run.lower()
        for i in range(len(run) - 2):
            a, b, c = (x - ord("a") for x in run[i:i + 3])
            out.append((a * 26 + b) * 26 + c)
    return out


def docs_from_csr(offsets, tokens):
    return [list(map(int, tokens[offsets[i]:offsets[i + 1]])) for i in range(len(offsets) - 1)]


def bags(docs):
    return [Counter(d) for d in docs]


def doc_freq(bag_list):
    df = Counter()
    for b in bag_list:
        for t in b:
            df[t] += 1
    return df


def idf_of(n_docs, df_t):
    return math.log((1 + n_docs) / (1 + df_t)) + 1


def select(df, vocab, n_docs, mode, L, start, k):
    """mode 0 = all, 1 = frequency region, 2 = document-frequency-one terms."""
    if mode == 2:
        chosen = [t for t in range(vocab) if df.get(t, 0) == 1][:L]
    else:
        ranked = sorted((t for t in range(vocab) if df.get(t, 0) > 0), key=lambda t: (-df[t], t))
        if mode == 0:
            chosen = ranked
        else:
            if start < 0:
                start = next((q for q, t in enumerate(ranked) if df[t] <= n_docs / 100), len(ranked))
            chosen = ranked[start:start + L]
    parts = [chosen[(p * len(chosen)) // k:((p + 1) * len(chosen)) // k] for p in range(k)]
    return parts


def weight_vec(bag, idf):
    return {t: c * (idf[t] if idf is not None else 1.0) for t, c in bag.items()}


def cosine(u, v):
    num = sum(x * v[t] for t, x in u.items() if t in v)
    nu = math.sqrt(sum(x * x for x in u.values()))
    nv = math.sqrt(sum(x * x for x in v.values()))
    if nu == 0 or nv == 0:
        return 0.0
    return num / (nu * nv)


def cosine_list(a, b):
    return cosine(dict(enumerate(a)), dict(enumerate(b)))


def signature(wvec, parts, idf):
    """Entry p = cosine between the document and partition p (a reference weighted like a document)."""
    out = []
    for part in parts:
        ref = {t: (idf[t] if idf is not None else 1.0) for t in part}
        out.append(cosine(wvec, ref))
    return out


def splitmix64(state):
    z = (state + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def feature_hash(t, seed, mode=0):
    """Mode 0: SplitMix64 of (t xor seed); modes 1 and 2: the first 8 bytes (little-endian) of
    the MD5 / SHA-1 digest of t (4 bytes, little-endian) followed by the seed (8 bytes,
    little-endian), taken from Python's hashlib."""
    if mode == 0:
        return splitmix64((t & 0xFFFFFFFF) ^ seed)
    msg = (t & 0xFFFFFFFF).to_bytes(4, "little") + (seed & MASK64).to_bytes(8, "little")
    dg = (hashlib.md5 if mode == 1 else hashlib.sha1)(msg).digest()
    return int.from_bytes(dg[:8], "little")


def simhash(doc_tokens, seed, mode=0):
    cols = [0] * 64
    for t in doc_tokens:
        h = feature_hash(t, seed, mode)
        for b in range(64):
            cols[b] += 1 if (h >> b) & 1 else -1
    return sum(1 << b for b in range(64) if cols[b] > 0)


def hamming(a, b):
    return bin(a ^ b).count("1")


def pipeline(offsets, tokens, vocab, k, L, mode, start, tfidf, seed, hash_mode=0):
    docs = docs_from_csr(offsets, tokens)
    bl = bags(docs)
    n = len(docs)
    df = doc_freq(bl)
    idf = {t: idf_of(n, df.get(t, 0)) for t in range(vocab)} if tfidf else None
    parts = select(df, vocab, n, mode, L, start, k)
    wv = [weight_vec(b, idf) for b in bl]
    sig = [signature(w, parts, idf) for w in wv]
    fp = [simhash(d, seed, hash_mode) for d in docs]
    return {"df": df, "idf": idf, "parts": parts, "w": wv, "sig": sig, "simhash": fp}
