"""GPU path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: raw signature entries within 2e-6 (FP32 contributions, exact
fixed-point sums); every cosine (signature cosine of Eq. 2, exact cosine of
Eq. 1) within 1e-5 absolute in the FP32 form; Simhash fingerprints and
Hamming pair sets bit-exact; pair sets equal to the oracle's except pairs
whose oracle score lies within 1e-5 of the threshold. Reduced-precision forms:
recall and precision >= 0.99 against the FP64 pair set.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle.oracle import (HASH_MD5, HASH_SHA1, MODE_ALL, MODE_DF1, MODE_REGION, Oracle, Params, build_index,
                           signature)
from paper_1810_03099_gb300 import synth
from tests.gpu_common import compare_pairs, concat, csr, cuda_or_skip, edge_docs, mixed_corpus, pair_dict

pytestmark = pytest.mark.gpu

SIG_TOL = 2e-6
COS_TOL = 1e-5
BAND = 1e-5


@pytest.fixture(scope="module")
def torch():
    return cuda_or_skip()


@pytest.fixture(scope="module")
def M(torch):
    from paper_1810_03099_gb300 import mrc
    return mrc


@pytest.fixture(scope="module")
def ctx(M):
    c = M.Context()
    yield c
    c.close()


@pytest.fixture(scope="module")
def orc():
    return Oracle()


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def mrc_params(M, p: Params, precision=0):
    return M.params_default(k=p.k, L=p.L, select_mode=p.mode, region_start=p.region_start, weighting=p.weighting,
                            precision=precision, tau=p.tau, hamming_max=p.hamming_max, seed=p.seed,
                            feature_hash=p.feature_hash)


PARAM_CASES = [
    Params(k=8),
    Params(k=16, mode=MODE_ALL, weighting=0),
    Params(k=64, mode=MODE_DF1, L=200),
    Params(k=200, mode=MODE_ALL),
    Params(k=33, mode=MODE_REGION, L=500, region_start=40, seed=7),
    Params(k=8, feature_hash=HASH_MD5),
    Params(k=16, mode=MODE_ALL, weighting=0, feature_hash=HASH_SHA1, seed=2**64 - 1),
]


@pytest.fixture(scope="module")
def corpus():
    return mixed_corpus()


@pytest.mark.parametrize("case", range(len(PARAM_CASES)))
def test_index_build_matches_oracle(torch, M, ctx, orc, corpus, case):
    p = PARAM_CASES[case]
    offs, toks = corpus
    V = 5000
    ref = build_index(offs, toks, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, offs), dev(torch, toks), V, mrc_params(M, p))
    ex = M.mrc_index_export(ctx, idx)
    assert np.array_equal(ex["df"].astype(np.int64), ref.df)
    assert np.max(np.abs(ex["idf"] - ref.idf_values) / ref.idf_values) < 1e-6
    assert np.array_equal(ex["part"], ref.part) and idx.L_used == ref.L_used
    assert np.max(np.abs(ex["rnorm"] - ref.rnorm) / np.maximum(ref.rnorm, 1e-300)) < 1e-6
    err = np.abs(ex["sig"].astype(np.float64) - ref.S)
    assert err.max() <= SIG_TOL, (err.max(), np.unravel_index(err.argmax(), err.shape))
    assert np.array_equal(ex["simhash"], ref.F)
    idx.free()


def test_index_build_large_tie_group(torch, M, ctx, orc):
    """20,000 terms that all share df = 5: the REGION selection's band is one tie group larger
    than the device sort holds, so the build selects on the host; the index still matches."""
    n_docs, V = 2000, 20000
    rows = [[] for _ in range(n_docs)]
    for t in range(V):
        for j in range(5):
            rows[(t * 5 + j) % n_docs].append(t)
    offs = np.zeros(n_docs + 1, np.int64)
    offs[1:] = np.cumsum([len(r) for r in rows])
    toks = np.concatenate([np.array(r, np.int32) for r in rows])
    p = Params(k=64)
    ref = build_index(offs, toks, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, offs), dev(torch, toks), V, mrc_params(M, p))
    ex = M.mrc_index_export(ctx, idx)
    assert np.array_equal(ex["part"], ref.part) and idx.L_used == ref.L_used == 2048
    assert np.max(np.abs(ex["rnorm"] - ref.rnorm) / np.maximum(ref.rnorm, 1e-300)) < 1e-6
    assert np.abs(ex["sig"].astype(np.float64) - ref.S).max() <= SIG_TOL
    idx.free()


@pytest.mark.parametrize("p", [Params(k=64, mode=MODE_ALL), Params(k=32, mode=MODE_DF1, L=20000),
                               Params(k=48, mode=MODE_REGION, L=20000), Params(k=16, mode=MODE_DF1, L=300)])
def test_selection_of_wide_bands(torch, M, ctx, orc, p):
    """Selections whose band of df values holds more than the 8,192 terms the small device path
    sorts: ALL ranks 50,589 terms over 339 df values (two radix passes), DF1 takes from a df-1
    group of 12,327 terms, REGION 20,000 terms over many values. The partitions, |R_p| and the
    signatures match the oracle's ranking by (df descending, id ascending)."""
    c = synth.make_corpus(synth.SPECS["tiny"].with_(n_docs=3000, vocab=60000))
    V = c.vocab
    ref = build_index(c.offsets, c.tokens, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), V, mrc_params(M, p))
    ex = M.mrc_index_export(ctx, idx)
    assert idx.L_used == ref.L_used
    assert np.array_equal(ex["part"], ref.part)
    assert np.max(np.abs(ex["rnorm"] - ref.rnorm) / np.maximum(ref.rnorm, 1e-300)) < 1e-6
    assert np.abs(ex["sig"].astype(np.float64) - ref.S).max() <= SIG_TOL
    assert np.array_equal(ex["simhash"], ref.F)
    idx.free()


def test_long_documents_in_groups(torch, M, ctx, orc):
    """800 documents of 2,048 to 8,000 tokens: at least four per CTA, so with 32-bit tables the
    four-warp groups take them, each into 2,048 64-bit slots hashed in two to eight passes. The
    build and the signature pass over tokens match the oracle."""
    c = synth.make_corpus(synth.SPECS["batch_queries"].with_(n_docs=800, vocab=5000, length_min=2048,
                                                              length_max=8000))
    V = c.vocab
    lens = np.diff(c.offsets)
    assert lens.min() >= 2048 and len(lens) >= 4 * 152
    p = Params(k=32, mode=MODE_ALL)  # every term a reference (the default region is empty here)
    ref = build_index(c.offsets, c.tokens, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), V, mrc_params(M, p))
    ex = M.mrc_index_export(ctx, idx)
    assert np.array_equal(ex["df"].astype(np.int64), ref.df)
    assert np.abs(ex["sig"].astype(np.float64) - ref.S).max() <= SIG_TOL
    assert np.array_equal(ex["simhash"], ref.F)
    S_ref, F_ref, _ = signature(ref, c.offsets, c.tokens, orc)
    sig, sh = M.mrc_signature(ctx, idx, dev(torch, c.offsets), dev(torch, c.tokens))
    assert np.abs(sig.cpu().numpy().astype(np.float64) - S_ref).max() <= SIG_TOL
    assert np.array_equal(sh.cpu().numpy().view(np.uint64), F_ref)
    idx.free()


def test_signature_of_new_documents(torch, M, ctx, orc, corpus):
    offs, toks = corpus
    V = 5000
    p = Params(k=24, mode=MODE_ALL)
    ref = build_index(offs, toks, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, offs), dev(torch, toks), V, mrc_params(M, p))
    # queries: a different seed, plus terms the index never saw (df = 0)
    q = synth.make_corpus(synth.SPECS["tiny"].with_(n_docs=300, vocab=V, seed=99))
    qo, qt = concat((q.offsets, q.tokens), csr(edge_docs(V, seed=5)))
    S_ref, F_ref, _ = signature(ref, qo, qt, orc)
    sig, sh = M.mrc_signature(ctx, idx, dev(torch, qo), dev(torch, qt))
    assert np.abs(sig.cpu().numpy().astype(np.float64) - S_ref).max() <= SIG_TOL
    assert np.array_equal(sh.cpu().numpy().view(np.uint64), F_ref)
    # host buffers give the same bits
    sig_h, sh_h = M.mrc_signature(ctx, idx, qo, qt)
    assert np.array_equal(sig_h, sig.cpu().numpy()) and np.array_equal(sh_h, sh.cpu().numpy().view(np.uint64))
    # page-locked host tokens are read in place by the kernels: the same bits again, and an
    # index built from page-locked buffers equals one built from device buffers
    po, pt = torch.from_numpy(qo).pin_memory(), torch.from_numpy(qt).pin_memory()
    sig_p, sh_p = M.mrc_signature(ctx, idx, po, pt)  # host outputs (numpy), ready on return
    assert np.array_equal(sig_p, sig.cpu().numpy()) and np.array_equal(sh_p, sh.cpu().numpy().view(np.uint64))
    idx_p = M.mrc_build_index(ctx, torch.from_numpy(offs).pin_memory(), torch.from_numpy(toks).pin_memory(), V,
                              mrc_params(M, p))
    a, b = M.mrc_index_export(ctx, idx), M.mrc_index_export(ctx, idx_p)
    assert all(np.array_equal(a[key], b[key]) for key in ("df", "sig", "simhash"))
    idx_p.free()
    idx.free()


def test_wide_vocabulary_tables(torch, M, ctx, orc, corpus):
    """A vocabulary of 2^22 term ids is too wide for the 32-bit table slots (21 bits of term id):
    every path (warp, four-warp groups, whole CTA) then hashes into 64-bit slots. The index build
    and the signature pass over tokens still match the oracle, with the mixed corpus's term ids
    spread over the whole vocabulary."""
    offs, toks = corpus
    V = 1 << 22
    toks = ((toks.astype(np.int64) * 838_861 + 12_345) % V).astype(np.int32)  # distinct ids stay distinct
    assert toks.max() >= 1 << 21
    p = Params(k=16)
    ref = build_index(offs, toks, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, offs), dev(torch, toks), V, mrc_params(M, p))
    ex = M.mrc_index_export(ctx, idx)
    assert np.array_equal(ex["df"].astype(np.int64), ref.df)
    assert np.abs(ex["sig"].astype(np.float64) - ref.S).max() <= SIG_TOL
    assert np.array_equal(ex["simhash"], ref.F)
    S_ref, F_ref, _ = signature(ref, offs, toks, orc)
    sig, sh = M.mrc_signature(ctx, idx, dev(torch, offs), dev(torch, toks))
    assert np.abs(sig.cpu().numpy().astype(np.float64) - S_ref).max() <= SIG_TOL
    assert np.array_equal(sh.cpu().numpy().view(np.uint64), F_ref)
    idx.free()


@pytest.mark.parametrize("k,tau", [(8, 0.9), (64, 0.9), (64, 0.6), (130, 0.8)])
def test_match_allpairs_fp32(torch, M, ctx, orc, k, tau):
    c = synth.make_corpus("tiny")
    V = c.vocab
    p = Params(k=k, mode=MODE_ALL if k > 64 else MODE_REGION)
    ref = build_index(c.offsets, c.tokens, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), V, mrc_params(M, p))
    buf, total = M.mrc_match(ctx, idx, None, tau)
    got = M.pairs_to_numpy(buf)
    assert total == got.shape[0]
    assert np.all(got["i"] < got["j"])
    tot, pi, pj, ps = orc.sig_pairs(ref.S, tau)
    rep = compare_pairs(pair_dict(got["i"], got["j"], got["score"]), pair_dict(pi, pj, ps), tau, BAND, COS_TOL,
                        lambda i, j: orc.cos_dense(ref.S[i], ref.S[j]))
    assert rep["n"] == tot
    idx.free()


def test_match_query_fp32(torch, M, ctx, orc):
    c = synth.make_corpus("tiny")
    V = c.vocab
    p = Params(k=16)
    ref = build_index(c.offsets, c.tokens, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), V, mrc_params(M, p))
    # arbitrary non-negative query vectors with exact zeros, and real document signatures
    Q = np.concatenate([synth.random_signatures(300, 16, 11, density=0.3), ref.S[:50].astype(np.float32)])
    Q[7] = 0.0  # an all-zero query matches nothing
    for tau in (0.9, 0.5):
        buf, total = M.mrc_match(ctx, idx, dev(torch, Q), tau)
        got = M.pairs_to_numpy(buf)
        Q64 = Q.astype(np.float64)
        tot, pi, pj, ps = orc.sig_match(Q64, ref.S, tau)
        compare_pairs(pair_dict(got["i"], got["j"], got["score"]), pair_dict(pi, pj, ps), tau, BAND, COS_TOL,
                      lambda i, j: orc.cos_dense(Q64[i], ref.S[j]))
        assert not np.any(got["i"] == 7)
    idx.free()


@pytest.mark.parametrize("precision,k", [(1, 64), (2, 64), (1, 100), (2, 40), (1, 200), (2, 20)])
def test_match_reduced_precision(torch, M, ctx, orc, precision, k):
    """Reduced-precision forms against the FP64 oracle: precision 1 builds its E4M3 compare
    operands from bfloat16 weights, precision 2 compares fp16 signatures; both rescore every
    candidate >= tau - margin in FP32 from the stored FP32-weight signatures. The stored
    signatures match the oracle's to 2e-6; accepted pairs are true pairs (1e-5); the
    low-precision candidate stage may lose a pair only beyond the margin; recall and precision
    against the FP64 pair set >= 0.99."""
    c = synth.make_corpus("tiny")
    V = c.vocab
    p = Params(k=k, mode=MODE_ALL if k > 64 else MODE_REGION)
    ref = build_index(c.offsets, c.tokens, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), V, mrc_params(M, p, precision))
    ex = M.mrc_index_export(ctx, idx)
    assert np.abs(ex["sig"].astype(np.float64) - ref.S).max() <= SIG_TOL
    tau = 0.9
    buf, total = M.mrc_match(ctx, idx, None, tau)
    got = M.pairs_to_numpy(buf)
    tot, pi, pj, ps = orc.sig_pairs(ref.S, tau)
    gd, od = pair_dict(got["i"], got["j"], got["score"]), pair_dict(pi, pj, ps)
    for pr, sc in gd.items():  # every accepted pair is a true pair (FP32 rescoring)
        o = od.get(pr, orc.cos_dense(ref.S[pr[0]], ref.S[pr[1]]))
        assert o >= tau - BAND and abs(sc - o) <= COS_TOL, (pr, sc, o)
    missed = [pr for pr, o in od.items() if pr not in gd and o > tau + BAND]
    assert len(missed) <= 0.01 * max(len(od), 1), (len(missed), len(od))
    # the spec bar of the reduced-precision forms: recall and precision >= 0.99 against
    # the plain FP64 oracle's pair set
    o64 = set(zip(pi.tolist(), pj.tolist()))
    g = set(gd)
    recall, prec = len(g & o64) / max(len(o64), 1), len(g & o64) / max(len(g), 1)
    assert recall >= 0.99 and prec >= 0.99, (recall, prec, len(o64), len(g))
    idx.free()


def test_precision_form_vs_fp64_at_20k_documents(torch, M, ctx, orc):
    """The precision form on 20,000 documents of the million-document recipe (2^18 terms,
    Zipf 1.05, median 300 tokens, 5 % near-duplicates) against the plain FP64 oracle: recall
    and precision of the pair set >= 0.99 for the bf16 + FP8 form and the FP32 form; every
    reported score within 1e-5 of its FP64 cosine (FP32 rescoring); the per-stage errors
    (signature entries with bfloat16 weights, the FP8 compare's cosine of its candidates) stay
    within their derived bounds, and the FP8 compare keeps every FP64 pair as a candidate."""
    from oracle.threaded import ThreadedOracle
    c = synth.make_corpus("precision", n_docs=20000)
    V = c.vocab
    to = ThreadedOracle(orc=orc)
    plain = to.build_index(c.offsets, c.tokens, V, Params(k=64))
    t64, qi, qj, _ = to.sig_pairs(plain.S, 0.9)
    to.close()
    o64 = set(zip(qi.tolist(), qj.tolist()))
    assert t64 > 50  # the recipe's near-duplicates alone give pairs
    nrm = np.linalg.norm(plain.S, axis=1)
    U = np.divide(plain.S, nrm[:, None], out=np.zeros_like(plain.S), where=nrm[:, None] > 0)
    offs, toks = dev(torch, c.offsets), dev(torch, c.tokens)
    for precision in (1, 0):
        idx = M.mrc_build_index(ctx, offs, toks, V, M.params_default(k=64, precision=precision))
        ex = M.mrc_index_export(ctx, idx)
        got = M.pairs_to_numpy(M.mrc_match(ctx, idx, None, 0.9)[0])
        ctx.set_rescoring(False)
        cand = M.pairs_to_numpy(M.mrc_match(ctx, idx, None, 0.9)[0])
        ctx.set_rescoring(True)
        idx.free()
        g = set(zip(got["i"].tolist(), got["j"].tolist()))
        recall, prec = len(g & o64) / len(o64), len(g & o64) / max(len(g), 1)
        assert recall >= 0.99 and prec >= 0.99, (precision, recall, prec)
        s64 = np.einsum("ij,ij->i", U[got["i"]], U[got["j"]])
        assert np.abs(got["score"] - s64).max() <= COS_TOL
        # stage 1: signature entries (each <= 1); bfloat16 weights (relative rounding <= 2^-9)
        # enter the numerator and both norms twice each, so an entry moves by <= 4 * 2^-9
        sig_err = np.abs(ex["sig"].astype(np.float64) - plain.S).max()
        assert sig_err <= (4 * 2.0 ** -9 if precision == 1 else SIG_TOL), sig_err
        # stage 2: no FP64 pair lost by the compare; its cosine within the fp16 form's proven
        # bound (2e-3), and for E4M3 (3-bit mantissas, 2^-4 relative per entry) within 0.05
        c64 = np.einsum("ij,ij->i", U[cand["i"]], U[cand["j"]])
        cmp_err = np.abs(cand["score"] - c64).max()
        assert cmp_err <= (0.05 if precision == 1 else 2e-3), cmp_err
        assert o64 <= set(zip(cand["i"].tolist(), cand["j"].tolist()))


@pytest.mark.parametrize("tau,weighting", [(0.5, 1), (0.9, 1), (0.7, 0)])
def test_cosine_allpairs(torch, M, ctx, orc, tau, weighting):
    offs, toks = mixed_corpus(n_tiny=1500, n_long=12)
    V = 5000
    p = Params(k=8, weighting=weighting)
    ref = build_index(offs, toks, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, offs), dev(torch, toks), V, mrc_params(M, p))
    buf, total = M.cosine_allpairs(ctx, idx, dev(torch, offs), dev(torch, toks), tau)
    got = M.pairs_to_numpy(buf)
    tot, pi, pj, ps = orc.cosine_pairs(ref.row_ptr, ref.terms, ref.w, tau)
    rep = compare_pairs(pair_dict(got["i"], got["j"], got["score"]), pair_dict(pi, pj, ps), tau, BAND, COS_TOL,
                        lambda i, j: orc.cosine_pair(ref.row_ptr, ref.terms, ref.w, i, j))
    assert rep["n"] == tot and tot > 0
    idx.free()


def test_cosine_allpairs_candidate_overflow_takes_tail_walk(torch, M, ctx, orc):
    """tau = 0: every one of the 4.5 M pairs of 3,000 documents is a candidate of the bound-pruned
    path, more than its 2^22-entry buffer, so the call falls back to the exhaustive tail walk.
    The total must be the oracle's (every pair) and the pairs written must carry the oracle's
    cosine."""
    c = synth.make_corpus("tiny", n_docs=3000)
    V = c.vocab
    p = Params(k=8)
    ref = build_index(c.offsets, c.tokens, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), V, mrc_params(M, p))
    n = c.n_docs
    buf, total = M.cosine_allpairs(ctx, idx, dev(torch, c.offsets), dev(torch, c.tokens), 0.0, capacity=1 << 20,
                                   grow=False)
    assert total == n * (n - 1) // 2
    got = M.pairs_to_numpy(buf)
    assert got.shape[0] == 1 << 20
    rng = np.random.Generator(np.random.PCG64(5))
    for x in rng.choice(got.shape[0], 500, replace=False).tolist():
        i, j, s = int(got["i"][x]), int(got["j"][x]), float(got["score"][x])
        assert i < j and abs(s - orc.cosine_pair(ref.row_ptr, ref.terms, ref.w, i, j)) <= COS_TOL
    # tau = 0.6 on the same documents (bound-pruned path) against the oracle
    a = M.pairs_to_numpy(M.cosine_allpairs(ctx, idx, dev(torch, c.offsets), dev(torch, c.tokens), 0.6)[0])
    tot, pi, pj, ps = orc.cosine_pairs(ref.row_ptr, ref.terms, ref.w, 0.6)
    compare_pairs(pair_dict(a["i"], a["j"], a["score"]), pair_dict(pi, pj, ps), 0.6, BAND, COS_TOL,
                  lambda i, j: orc.cosine_pair(ref.row_ptr, ref.terms, ref.w, i, j))
    idx.free()


@pytest.mark.parametrize("n_docs,tau", [(20, 0.0), (60, 0.1)])
def test_cosine_allpairs_long_documents_and_no_head(torch, M, ctx, orc, n_docs, tau):
    """Few documents, most of them long (log-uniform 20..20,000 tokens). With N = 20 the head cut
    max(32, N/8) exceeds every df, so the bound-pruned GEMM has no head columns at all; with a
    low tau nearly every pair is a candidate, and the long documents' tail lists (thousands of
    terms) take the CTA-level verification in several hash-partitioned passes."""
    b = synth.make_corpus(synth.SPECS["batch_queries"].with_(n_docs=n_docs, vocab=5000, seed=41))
    e = csr(edge_docs(5000))
    offs, toks = concat((b.offsets, b.tokens), e)
    V = 5000
    p = Params(k=8)
    ref = build_index(offs, toks, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, offs), dev(torch, toks), V, mrc_params(M, p))
    buf, total = M.cosine_allpairs(ctx, idx, dev(torch, offs), dev(torch, toks), tau)
    got = M.pairs_to_numpy(buf)
    tot, pi, pj, ps = orc.cosine_pairs(ref.row_ptr, ref.terms, ref.w, tau)
    rep = compare_pairs(pair_dict(got["i"], got["j"], got["score"]), pair_dict(pi, pj, ps), tau, BAND, COS_TOL,
                        lambda i, j: orc.cosine_pair(ref.row_ptr, ref.terms, ref.w, i, j))
    assert rep["n"] == tot and tot > 0
    idx.free()


@pytest.mark.parametrize("mode", [HASH_MD5, HASH_SHA1])
def test_paper_feature_hashes_queries_reload(torch, M, ctx, orc, corpus, mode, tmp_path):
    """MD5 / SHA-1 Simhash features (Section III): fingerprints of new documents (allocating and
    no-allocation calls, also after a save / load round trip, which recomputes the feature
    table) equal the oracle's bit for bit, and so do the Hamming pair sets."""
    offs, toks = corpus
    V = 5000
    p = Params(k=8, feature_hash=mode, seed=0x0123456789ABCDEF)
    ref = build_index(offs, toks, V, p, orc)
    idx = M.mrc_build_index(ctx, dev(torch, offs), dev(torch, toks), V, mrc_params(M, p))
    assert np.array_equal(M.mrc_index_export(ctx, idx)["simhash"], ref.F)
    q = synth.make_corpus(synth.SPECS["tiny"].with_(n_docs=300, vocab=V, seed=98))
    qo, qt = concat((q.offsets, q.tokens), csr(edge_docs(V, seed=6)))
    _, F_ref, _ = signature(ref, qo, qt, orc)
    path = str(tmp_path / "md5.mrcidx")
    M.mrc_index_save(ctx, idx, path)
    idx2 = M.mrc_index_load(ctx, path)
    for x in (idx, idx2):
        _, sh = M.mrc_signature(ctx, x, dev(torch, qo), dev(torch, qt))
        assert np.array_equal(sh.cpu().numpy().view(np.uint64), F_ref)
        n = qo.shape[0] - 1
        sig = torch.empty((n, p.k), dtype=torch.float32, device="cuda")
        sh2 = torch.empty(n, dtype=torch.int64, device="cuda")
        M.mrc_signature_noalloc(ctx, x, dev(torch, qo), dev(torch, qt), sig, sh2)
        assert np.array_equal(sh2.cpu().numpy().view(np.uint64), F_ref)
    # a different mode gives different fingerprints (the table is the one asked for)
    assert not np.array_equal(ref.F, build_index(offs, toks, V, Params(k=8, seed=p.seed), orc).F)
    buf, total = M.simhash_match(ctx, dev(torch, F_ref.view(np.int64)), dev(torch, ref.F.view(np.int64)), 3)
    got = M.pairs_to_numpy(buf)
    tot, pi, pj, ph = orc.hamming_pairs(F_ref, ref.F, 3)
    assert total == tot
    assert sorted(zip(got["i"].tolist(), got["j"].tolist(), got["score"].astype(int).tolist())) == sorted(
        zip(pi.tolist(), pj.tolist(), ph.tolist()))
    idx2.free()
    idx.free()


def test_simhash_match_bit_exact(torch, M, ctx, orc):
    c = synth.make_corpus("tiny")
    ref_F = orc.simhash(c.offsets, c.tokens, 0x1810030990)
    for hmax in (0, 3, 6):
        buf, total = M.simhash_match(ctx, dev(torch, ref_F.view(np.int64)), None, hmax)
        got = M.pairs_to_numpy(buf)
        tot, pi, pj, ph = orc.hamming_pairs(ref_F, None, hmax)
        assert total == tot
        assert sorted(zip(got["i"].tolist(), got["j"].tolist(), got["score"].astype(int).tolist())) == sorted(
            zip(pi.tolist(), pj.tolist(), ph.tolist()))
    # query x index with planted near copies, ragged sizes
    X = synth.random_fingerprints(5003, 21, n_near=800, max_flip=4)
    Q = np.concatenate([X[-300:], synth.random_fingerprints(77, 22)])
    buf, total = M.simhash_match(ctx, dev(torch, Q.view(np.int64)), dev(torch, X.view(np.int64)), 4)
    got = M.pairs_to_numpy(buf)
    tot, pi, pj, ph = orc.hamming_pairs(Q, X, 4)
    assert total == tot and tot >= 300
    assert sorted(zip(got["i"].tolist(), got["j"].tolist())) == sorted(zip(pi.tolist(), pj.tolist()))


def test_host_buffers_same_results(torch, M, ctx):
    c = synth.make_corpus("tiny", n_docs=700)
    V = c.vocab
    p = M.params_default(k=16)
    a = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), V, p)
    b = M.mrc_build_index(ctx, c.offsets, c.tokens, V, p)
    ea, eb = M.mrc_index_export(ctx, a), M.mrc_index_export(ctx, b)
    assert np.array_equal(ea["sig"], eb["sig"]) and np.array_equal(ea["simhash"], eb["simhash"])
    ga = M.pairs_to_numpy(M.mrc_match(ctx, a, None, 0.8)[0])
    gb = M.mrc_match(ctx, b, None, 0.8, device=None)[0]
    assert sorted(ga.tolist()) == sorted(gb.tolist())
    ca = M.pairs_to_numpy(M.cosine_allpairs(ctx, a, dev(torch, c.offsets), dev(torch, c.tokens), 0.6)[0])
    cb = M.cosine_allpairs(ctx, b, c.offsets, c.tokens, 0.6, device=None)[0]
    assert sorted(ca.tolist()) == sorted(cb.tolist())
    a.free()
    b.free()


def test_errors_and_capacity(torch, M, ctx):
    c = synth.make_corpus("tiny", n_docs=300)
    V = c.vocab
    bad = c.tokens.copy()
    bad[17] = V + 3
    with pytest.raises(M.MrcError) as e:
        M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, bad), V, M.params_default())
    assert e.value.status == M.MRC_ERR_INVALID
    with pytest.raises(M.MrcError) as e:
        M.mrc_build_index(ctx, c.offsets, c.tokens, V, M.params_default(k=0))
    assert e.value.status == M.MRC_ERR_INVALID
    idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), V, M.params_default(k=8))
    full, total = M.mrc_match(ctx, idx, None, 0.5)
    assert total > 10
    part, total2 = M.mrc_match(ctx, idx, None, 0.5, capacity=10, grow=False)
    assert total2 == total and part.shape[0] == 10
    fullset = {tuple(r) for r in M.pairs_to_numpy(full)[["i", "j"]].tolist()}
    assert {tuple(r) for r in M.pairs_to_numpy(part)[["i", "j"]].tolist()} <= fullset
    idx.free()


def test_save_load_roundtrip(torch, M, ctx, tmp_path):
    c = synth.make_corpus("tiny", n_docs=500)
    for prec in (0, 1, 2):
        idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), c.vocab,
                                M.params_default(k=32, precision=prec))
        path = str(tmp_path / f"idx{prec}.bin")
        M.mrc_index_save(ctx, idx, path)
        idx2 = M.mrc_index_load(ctx, path)
        e1, e2 = M.mrc_index_export(ctx, idx), M.mrc_index_export(ctx, idx2)
        for key in ("sig", "simhash", "df", "idf", "part"):
            assert np.array_equal(e1[key], e2[key]), key
        p1 = sorted(M.pairs_to_numpy(M.mrc_match(ctx, idx, None, 0.9)[0]).tolist())
        p2 = sorted(M.pairs_to_numpy(M.mrc_match(ctx, idx2, None, 0.9)[0]).tolist())
        assert p1 == p2
        q, _ = M.mrc_signature(ctx, idx2, dev(torch, c.offsets), dev(torch, c.tokens))
        assert np.array_equal(q.cpu().numpy(), e1["sig"])
        idx.free()
        idx2.free()
