"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each ``pin_*`` takes an ``Oracle`` and raises ``AssertionError`` on a mismatch.
The same suite runs on the real oracle (all must pass) and on deliberately
broken copies of it (``test_oracle_mutants.py``: at least one must fail for
each planted mistake). What each pin rests on:

* published values (SplitMix64 outputs from state 0; the MD5 test suite of
  RFC 1321 and SHA-1 examples of FIPS 180) and Python's hashlib on messages
  of every length around the padding boundaries;
* closed forms worked by hand (idf values, a count-weighted signature,
  partition cuts of a hand-ranked df list, error statistics);
* invariants the paper's definitions imply (symmetry, cos(x,x)=1, a
  reference's own signature is one-hot, singleton partitions make the
  signature cosine equal the exact cosine (the many-partition limit of
  Section IV), Simhash of one or two terms, Hamming of identical documents);
* brute force on tiny corpora by the independent pure-Python code in
  ``oracle/brute.py``.
"""
from __future__ import annotations

import hashlib
import math
import os
import re
import shlex

import numpy as np

from oracle import brute
from oracle.oracle import MODE_ALL, MODE_DF1, MODE_REGION, Oracle, Params, build_index

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _csr(docs):
    offs = np.zeros(len(docs) + 1, np.int64)
    offs[1:] = np.cumsum([len(d) for d in docs])
    toks = np.array([t for d in docs for t in d], dtype=np.int32)
    return offs, toks


def _tiny_corpus(seed, n_docs=40, vocab=60, lo=1, hi=30, n_dup=3):
    rng = np.random.Generator(np.random.PCG64(seed))
    docs = []
    for i in range(n_docs):
        if i >= n_docs - n_dup:
            docs.append(list(docs[int(rng.integers(0, i - 1))]))
            continue
        n = int(rng.integers(lo, hi + 1))
        # skewed term law so that df spreads over several values
        docs.append([int(x) for x in np.minimum(rng.zipf(1.3, size=n) - 1, vocab - 1)])
    docs[5] = []  # an empty document
    return docs


# ---------------------------------------------------------------- published / hand values
def pin_splitmix64_published(o: Oracle):
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    assert rows
    for state, out in rows:
        got = o.splitmix64(int(state, 16))
        assert got == int(out, 16), (state, hex(got), out)
    # the term hash is one generator step from (t xor seed)
    assert o.term_hash(0, 0) == int(rows[0][1], 16)


def pin_digests_published(o: Oracle):
    with open(os.path.join(GOLDEN, "digests.txt")) as f:
        rows = [shlex.split(ln) for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) >= 8
    for algo, msg, hexd in rows:
        got = (o.md5 if algo == "md5" else o.sha1)(msg.encode())
        assert got.hex() == hexd, (algo, msg, got.hex())


def pin_digests_match_hashlib(o: Oracle):
    """Every message length from 0 to 130 bytes (one, two and three padded blocks, both sides
    of the 56-byte length-field boundary) and a few long ones, against Python's hashlib."""
    rng = np.random.Generator(np.random.PCG64(11))
    for n in list(range(131)) + [191, 192, 1000]:
        m = rng.integers(0, 256, size=n, dtype=np.uint8).tobytes()
        assert o.md5(m) == hashlib.md5(m).digest(), n
        assert o.sha1(m) == hashlib.sha1(m).digest(), n


def pin_feature_hash_modes(o: Oracle):
    """The 12-byte message (term, then seed, little-endian) and the first 8 digest bytes taken
    little-endian, against hashlib; mode 0 is the SplitMix64 step."""
    rng = np.random.Generator(np.random.PCG64(12))
    for t, seed in [(0, 0), (1, 0), (0x7FFFFFFF, 2**64 - 1), (12345, 0x1810030990)] + \
            [(int(rng.integers(0, 2**31)), int(rng.integers(0, 2**63))) for _ in range(20)]:
        msg = t.to_bytes(4, "little") + seed.to_bytes(8, "little")
        assert o.feature_hash(t, seed, 1) == int.from_bytes(hashlib.md5(msg).digest()[:8], "little")
        assert o.feature_hash(t, seed, 2) == int.from_bytes(hashlib.sha1(msg).digest()[:8], "little")
        assert o.feature_hash(t, seed, 0) == o.term_hash(t, seed)


def _text_csr(docs):
    offs = np.zeros(len(docs) + 1, np.int64)
    offs[1:] = np.cumsum([len(d) for d in docs])
    return offs, np.frombuffer(b"".join(docs), np.uint8).copy()


def pin_char3grams_by_hand(o: Oracle):
    # the = (19, 7, 4) -> 19*676 + 7*26 + 4 = 13030; cat = 1371; and = 341; hat = 4751;
    # abc = 28, bcd = 731, aaa = 0, zzz = 17575 (the largest id)
    docs = [b"The cat, AND the hat.", b"", b"ab", b"c", b"abcd", b"a1bc", b"aaa zzz", b"x y z", b"ZzZ\xc3\xa9ab"]
    go, g = o.char3grams(*_text_csr(docs))
    assert go.tolist() == [0, 5, 5, 5, 5, 7, 7, 9, 9, 10]
    assert g.tolist() == [13030, 1371, 341, 13030, 4751, 28, 731, 0, 17575, 17575]


def pin_char3grams_brute_force(o: Oracle):
    """Random byte documents (letters of both cases, separators, UTF-8 bytes) against the
    regular-expression version in brute.py; the count of each document is the sum of
    max(0, m - 2) over its letter runs of length m."""
    rng = np.random.Generator(np.random.PCG64(14))
    alphabet = np.frombuffer(b"abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ  .,\n09@[`{\xc3\xa9\xff", np.uint8)
    docs = [rng.choice(alphabet, size=int(rng.integers(0, 200))).tobytes() for _ in range(60)]
    go, g = o.char3grams(*_text_csr(docs))
    for d, doc in enumerate(docs):
        assert g[go[d]:go[d + 1]].tolist() == brute.char3grams(doc), d
        runs = re.findall(rb"[A-Za-z]+", doc)
        assert go[d + 1] - go[d] == sum(max(0, len(r) - 2) for r in runs)
    assert go[-1] == g.shape[0] and int(g.max()) < 26 ** 3


def pin_idf_closed_form(o: Oracle):
    # idf(t) = ln((1+N)/(1+df)) + 1, worked by hand
    idf = o.idf(3, np.array([1, 3, 0], np.int64))
    assert abs(idf[0] - 1.6931471805599453) < 1e-15  # ln 2 + 1
    assert abs(idf[1] - 1.0) < 1e-15  # df = N
    assert abs(idf[2] - 2.386294361119891) < 1e-15  # ln 4 + 1
    idf = o.idf(9, np.array([2], np.int64))
    assert abs(idf[0] - 2.203972804325936) < 1e-15  # ln(10/3) + 1


def pin_term_counts_by_hand(o: Oracle):
    offs, toks = _csr([[3, 1, 3, 3, 0], [], [7]])
    rp, terms, counts = o.term_counts(offs, toks)
    assert rp.tolist() == [0, 3, 3, 4]
    assert terms.tolist() == [0, 1, 3, 7]
    assert counts.tolist() == [1, 1, 3, 1]


def pin_reference_selection_by_hand(o: Oracle):
    # ranked by df descending then id: t5(7) t1(5) t9(4) t2(3) t3(3) t7(2) t4(1) t6(1); t0, t8 have df 0
    df = np.array([0, 5, 3, 3, 1, 7, 1, 2, 0, 4], np.int64)

    def parts(part, k):
        return [sorted(np.nonzero(part == p)[0].tolist()) for p in range(k)]

    part, used = o.select_refs(df, 100, MODE_ALL, 0, 0, 3)
    assert used == 8 and parts(part, 3) == [[1, 5], [2, 3, 9], [4, 6, 7]]
    part, used = o.select_refs(df, 100, MODE_REGION, 4, 2, 2)
    assert used == 4 and parts(part, 2) == [[2, 9], [3, 7]]
    # default region start with N = 300: first rank with df <= 3 is t2 (rank 3)
    part, used = o.select_refs(df, 300, MODE_REGION, 3, -1, 1)
    assert used == 3 and parts(part, 1) == [[2, 3, 7]]
    part, used = o.select_refs(df, 100, MODE_DF1, 5, 0, 2)
    assert used == 2 and parts(part, 2) == [[4], [6]]


def pin_count_signature_by_hand(o: Oracle):
    # doc = [1, 1, 2], counts weighting, partitions {1} and {2, 3}:
    # s0 = 2 / sqrt(5), s1 = 1 / (sqrt(5) sqrt(2))
    offs, toks = _csr([[1, 1, 2]])
    rp, terms, counts = o.term_counts(offs, toks)
    w = o.weights(terms, counts, None)
    part = np.array([-1, 0, 1, 1], np.int32)
    rn = o.ref_norms(part, 2, None)
    assert abs(rn[0] - 1.0) < 1e-15 and abs(rn[1] - math.sqrt(2.0)) < 1e-15
    S = o.signatures(rp, terms, w, part, None, rn, 2)
    assert abs(S[0, 0] - 2 / math.sqrt(5)) < 1e-15
    assert abs(S[0, 1] - 1 / math.sqrt(10)) < 1e-15


def pin_error_stats_by_hand(o: Oracle):
    st = o.error_stats(np.array([0.5, 0.25, 1.0]), np.array([0.25, 0.5, 1.0]))
    # e = [0.25, -0.25, 0]: MAE 1/6, mean 0, Var = E[e^2] = 1/24
    assert abs(st["mae"] - 1 / 6) < 1e-15 and abs(st["mean"]) < 1e-15
    assert abs(st["var"] - 1 / 24) < 1e-15 and abs(st["mse"] - 1 / 24) < 1e-15


def pin_bf16_rounding_matches_library(o: Oracle):
    """bfloat16 rounding (RNE after FP32) against torch's CPU float32 -> bfloat16 conversion."""
    import torch
    rng = np.random.Generator(np.random.PCG64(9))
    xs = np.concatenate([rng.uniform(0.5, 20.0, 4000), rng.lognormal(0, 3, 4000),
                         [1.0, 1.00390625, 1.005859375, 1.0078125, 2.0 ** -20, 3.0, 17.123456]])
    want = torch.tensor(xs.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([o.round_bf16(x) for x in xs])
    assert np.array_equal(got, want)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert o.round_bf16(1.0 + 2.0 ** -8) == 1.0
    assert o.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6


# ---------------------------------------------------------------- invariants of the definitions
def pin_reference_doc_is_one_hot(o: Oracle):
    """A document made of exactly the terms of partition p has signature e_p
    (partitions are disjoint, and a reference is weighted like a document)."""
    docs = _tiny_corpus(11)
    offs, toks = _csr(docs)
    for weighting in (0, 1):
        idx = build_index(offs, toks, 60, Params(k=4, L=20, mode=MODE_ALL, weighting=weighting), o)
        for p in range(4):
            ref_terms = np.nonzero(idx.part == p)[0].astype(np.int32)
            assert ref_terms.size > 0
            qo = np.array([0, ref_terms.size], np.int64)
            from oracle.oracle import signature
            S, _, _ = signature(idx, qo, ref_terms, o)
            e = np.zeros(4)
            e[p] = 1.0
            assert np.max(np.abs(S[0] - e)) < 1e-12, (weighting, p, S[0])


def pin_singleton_partitions_equal_exact_cosine(o: Oracle):
    """With every term of non-zero df as its own partition (the many-partition
    limit of Section IV), s(d) is d's unit weight vector, so the signature
    cosine equals the exact cosine for every pair."""
    docs = _tiny_corpus(12)
    offs, toks = _csr(docs)
    df = o.df(*o.term_counts(offs, toks)[:2], 60)
    k = int((df > 0).sum())
    for weighting in (0, 1):
        idx = build_index(offs, toks, 60, Params(k=k, mode=MODE_ALL, weighting=weighting), o)
        n = idx.n_docs
        for i in range(n):
            for j in range(n):
                a = o.cos_dense(idx.S[i], idx.S[j])
                b = o.cosine_pair(idx.row_ptr, idx.terms, idx.w, i, j)
                assert abs(a - b) < 1e-12, (i, j, a, b)


def pin_symmetry_and_self_similarity(o: Oracle):
    docs = _tiny_corpus(13)
    offs, toks = _csr(docs)
    idx = build_index(offs, toks, 60, Params(k=6, L=30, mode=MODE_ALL), o)
    n = idx.n_docs
    for i in range(n):
        nz = np.any(idx.S[i] > 0)
        assert abs(o.cos_dense(idx.S[i], idx.S[i]) - (1.0 if nz else 0.0)) < 1e-12
        has = idx.row_ptr[i + 1] > idx.row_ptr[i]
        assert abs(o.cosine_pair(idx.row_ptr, idx.terms, idx.w, i, i) - (1.0 if has else 0.0)) < 1e-12
        for j in range(n):
            assert o.cos_dense(idx.S[i], idx.S[j]) == o.cos_dense(idx.S[j], idx.S[i])
            a = o.cosine_pair(idx.row_ptr, idx.terms, idx.w, i, j)
            b = o.cosine_pair(idx.row_ptr, idx.terms, idx.w, j, i)
            assert abs(a - b) < 1e-15
            assert -1e-15 <= a <= 1 + 1e-12


def pin_scaled_and_disjoint_docs(o: Oracle):
    """Repeating every token of a document leaves its direction unchanged
    (cosine 1); documents with no common term have cosine 0."""
    offs, toks = _csr([[1, 2, 2, 5], [1, 1, 2, 2, 2, 2, 5, 5], [3, 4], [9, 9, 8]])
    rp, terms, counts = o.term_counts(offs, toks)
    for idf in (None, o.idf(4, o.df(rp, terms, 10))):
        w = o.weights(terms, counts, idf)
        assert abs(o.cosine_pair(rp, terms, w, 0, 1) - 1.0) < 1e-14
        assert o.cosine_pair(rp, terms, w, 0, 2) == 0.0
        assert o.cosine_pair(rp, terms, w, 2, 3) == 0.0


def pin_simhash_small_cases(o: Oracle):
    for mode in (0, 1, 2):
        _simhash_small_cases(o, mode)


def _simhash_small_cases(o: Oracle, mode):
    seed = 0x1234
    h = [brute.feature_hash(t, seed, mode) for t in range(4)]
    # one term, any multiplicity: the term's own hash
    offs, toks = _csr([[2], [2, 2, 2], [0, 1], [0, 1, 1], [0, 1, 3], [0, 1, 3], []])
    F = o.simhash(offs, toks, seed, mode)
    assert int(F[0]) == h[2] and int(F[1]) == h[2]
    # two terms once each: a column is positive only where both bits are 1 (a tie gives 0)
    assert int(F[2]) == h[0] & h[1]
    # counts weigh in: term 1 twice beats term 0 once
    assert int(F[3]) == h[1]
    # three terms once each: bitwise majority
    assert int(F[4]) == (h[0] & h[1]) | (h[0] & h[3]) | (h[1] & h[3])
    # identical documents: Hamming 0; an empty document: all column sums 0 -> 0
    assert o.hamming(int(F[4]), int(F[5])) == 0
    assert int(F[6]) == 0


def pin_hamming_textbook(o: Oracle):
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(200):
        a, b = (int(x) for x in rng.integers(0, 2**63, size=2, dtype=np.int64))
        a ^= int(rng.integers(0, 2)) << 63
        assert o.hamming(a, b) == bin(a ^ b).count("1")
    assert o.hamming(0, (1 << 64) - 1) == 64


def pin_pair_emission_rules(o: Oracle):
    """i < j only, inclusive threshold, total count returned beyond capacity."""
    S = np.array([[1.0, 0.0], [1.0, 0.0], [0.0, 1.0], [3.0, 4.0]])
    # cos(s3, s0) = 0.6, cos(s3, s2) = 0.8
    tot, pi, pj, ps = o.sig_pairs(S, 0.8)
    assert tot == 2 and list(zip(pi.tolist(), pj.tolist())) == [(0, 1), (2, 3)]
    assert abs(ps[1] - 0.8) < 1e-15
    tot, pi, pj, ps = o.sig_pairs(S, 0.6)
    assert tot == 4
    tot, pi, pj, ps = o.sig_pairs(S, 0.6, cap=1)
    assert tot == 4 and pi.size == 1
    tot, pi, pj, ph = o.hamming_pairs(np.array([0, 1, 3, 0], np.uint64), None, 1)
    assert tot == 4 and list(zip(pi.tolist(), pj.tolist())) == [(0, 1), (0, 3), (1, 2), (1, 3)]
    tot, _, _, _ = o.hamming_pairs(np.array([0, 1, 3, 0], np.uint64), None, 0)
    assert tot == 1


# ---------------------------------------------------------------- brute force
def pin_brute_force_agreement(o: Oracle):
    for seed, (mode, L, start, k, tfidf) in enumerate([
            (MODE_ALL, 0, 0, 5, True), (MODE_REGION, 24, -1, 4, True), (MODE_REGION, 20, 3, 6, False),
            (MODE_DF1, 9, 0, 3, True)]):
        docs = _tiny_corpus(100 + seed, n_docs=30)
        offs, toks = _csr(docs)
        vocab = 60
        p = Params(k=k, L=L, mode=mode, region_start=start, weighting=1 if tfidf else 0, seed=0xABCDEF + seed,
                   feature_hash=seed % 3)
        idx = build_index(offs, toks, vocab, p, o)
        ref = brute.pipeline(offs, toks, vocab, k, p.L_eff, mode, start, tfidf, p.seed, p.feature_hash)
        for t in range(vocab):
            assert idx.df[t] == ref["df"].get(t, 0)
        if tfidf:
            assert max(abs(idx.idf[t] - ref["idf"][t]) for t in range(vocab)) < 1e-12
        for q, part in enumerate(ref["parts"]):
            assert sorted(np.nonzero(idx.part == q)[0].tolist()) == sorted(part)
        S = np.array(ref["sig"])
        assert np.max(np.abs(idx.S - S)) < 1e-12
        assert [int(x) for x in idx.F] == ref["simhash"]
        n = len(docs)
        for i in range(n):
            for j in range(n):
                c = brute.cosine(ref["w"][i], ref["w"][j])
                assert abs(o.cosine_pair(idx.row_ptr, idx.terms, idx.w, i, j) - c) < 1e-12
                assert abs(o.cos_dense(idx.S[i], idx.S[j]) - brute.cosine_list(ref["sig"][i], ref["sig"][j])) < 1e-12
        # pair sets at a threshold
        tot, pi, pj, _ = o.cosine_pairs(idx.row_ptr, idx.terms, idx.w, 0.5)
        want = {(i, j) for i in range(n) for j in range(i + 1, n) if brute.cosine(ref["w"][i], ref["w"][j]) >= 0.5}
        assert set(zip(pi.tolist(), pj.tolist())) == want and tot == len(want)


def pin_exact_duplicates_found(o: Oracle):
    """Documents copied with zero edits are found by all three methods."""
    docs = _tiny_corpus(21, n_docs=40, n_dup=4)
    offs, toks = _csr(docs)
    idx = build_index(offs, toks, 60, Params(k=5, L=25, mode=MODE_ALL), o)
    dups = []
    for i in range(36, 40):
        j = next(j for j in range(i) if docs[j] == docs[i])
        dups.append((j, i))
    sig = set(zip(*o.sig_pairs(idx.S, 0.9)[1:3]))
    cos = set(zip(*o.cosine_pairs(idx.row_ptr, idx.terms, idx.w, 0.9)[1:3]))
    ham = set(zip(*o.hamming_pairs(idx.F, None, 0)[1:3]))
    for pr in dups:
        if np.any(idx.S[pr[1]] > 0):
            assert pr in sig, pr
        assert pr in cos and pr in ham, pr


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


def run_all(o: Oracle):
    failures = []
    for f in ALL_PINS:
        try:
            f(o)
        except Exception as e:  # noqa: BLE001 - a crash of a mutant counts as a failed pin
            failures.append((f.__name__, repr(e)[:200]))
    return failures
