"""Parity at the benchmark's full size and launch configuration (news20: 18,846 documents,
60,000 terms, k = 64, tau = 0.9, Hamming <= 3), through the C ABI.

Signatures and Simhash are compared for every document. Pair sets are compared on a seeded
sample of rows: for each sampled row i the oracle scores every pair (i, j > i) one by one,
and the GPU's pairs of row i must match except within 1e-5 of the threshold. Every emitted
pair's score is checked against the oracle.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, Params, build_index
from paper_1810_03099_gb300 import synth
from tests.gpu_common import cuda_or_skip

pytestmark = pytest.mark.gpu

K, TAU, HMAX = 64, 0.9, 3
SAMPLE_ROWS = 40


@pytest.fixture(scope="module")
def setup():
    torch = cuda_or_skip()
    from paper_1810_03099_gb300 import mrc
    c = synth.cached_corpus("news20")
    orc = Oracle()
    ref = build_index(c.offsets, c.tokens, c.vocab, Params(k=K, tau=TAU, hamming_max=HMAX), orc)
    ctx = mrc.Context()
    o = torch.from_numpy(c.offsets).cuda()
    t = torch.from_numpy(c.tokens).cuda()
    idx = mrc.mrc_build_index(ctx, o, t, c.vocab, mrc.params_default(k=K, tau=TAU, hamming_max=HMAX))
    rows = np.sort(np.random.Generator(np.random.PCG64(77)).choice(c.n_docs - 1, SAMPLE_ROWS, replace=False))
    yield {"torch": torch, "mrc": mrc, "c": c, "orc": orc, "ref": ref, "ctx": ctx, "o": o, "t": t, "idx": idx,
           "rows": rows}
    idx.free()
    ctx.close()


def _row_check(got, rows, n, score_fn, tau):
    by_row = {}
    for i, j, s in zip(got["i"].tolist(), got["j"].tolist(), got["score"].tolist()):
        by_row.setdefault(i, {})[j] = s
    for i in rows.tolist():
        want = {}
        for j in range(i + 1, n):
            s = score_fn(i, j)
            if s >= tau or abs(s - tau) <= 1e-5:
                want[j] = s
        have = by_row.get(i, {})
        for j, s in want.items():
            if j not in have:
                assert abs(s - tau) <= 1e-5, (i, j, s)
        for j, s in have.items():
            assert j in want, (i, j, s)
            assert abs(s - want[j]) <= 1e-5, (i, j, s, want[j])


def test_fullsize_signatures_and_simhash(setup):
    m, ctx, idx, ref = setup["mrc"], setup["ctx"], setup["idx"], setup["ref"]
    ex = m.mrc_index_export(ctx, idx)
    assert np.abs(ex["sig"].astype(np.float64) - ref.S).max() <= 2e-6
    assert np.array_equal(ex["simhash"], ref.F)
    assert np.array_equal(ex["part"], ref.part)


def test_fullsize_signature_match(setup):
    m, ctx, idx, ref, orc = setup["mrc"], setup["ctx"], setup["idx"], setup["ref"], setup["orc"]
    got = m.pairs_to_numpy(m.mrc_match(ctx, idx, None, TAU)[0])
    for i, j, s in zip(got["i"], got["j"], got["score"]):
        assert abs(s - orc.cos_dense(ref.S[i], ref.S[j])) <= 1e-5
    _row_check(got, setup["rows"], ref.S.shape[0], lambda i, j: orc.cos_dense(ref.S[i], ref.S[j]), TAU)


def test_fullsize_simhash_match(setup):
    m, ctx, torch, ref, orc = setup["mrc"], setup["ctx"], setup["torch"], setup["ref"], setup["orc"]
    F = torch.from_numpy(ref.F.view(np.int64)).cuda()
    got = m.pairs_to_numpy(m.simhash_match(ctx, F, None, HMAX)[0])
    have = set(zip(got["i"].tolist(), got["j"].tolist()))
    n = ref.F.shape[0]
    for i in setup["rows"].tolist() + list(range(0, n, 997)):
        tot, _, pj, _ = orc.hamming_pairs(ref.F[i:i + 1], ref.F[i + 1:], HMAX)
        want = {(i, i + 1 + int(j)) for j in pj}
        assert {p for p in have if p[0] == i} == want
    for i, j, h in zip(got["i"][:2000], got["j"][:2000], got["score"][:2000]):
        assert orc.hamming(int(ref.F[i]), int(ref.F[j])) == int(h)


def test_fullsize_exact_cosine(setup):
    m, ctx, ref, orc = setup["mrc"], setup["ctx"], setup["ref"], setup["orc"]
    got = m.pairs_to_numpy(m.cosine_allpairs(ctx, setup["idx"], setup["o"], setup["t"], TAU)[0])
    assert got.shape[0] > 0
    for i, j, s in zip(got["i"], got["j"], got["score"]):
        assert abs(s - orc.cosine_pair(ref.row_ptr, ref.terms, ref.w, i, j)) <= 1e-5
    _row_check(got, setup["rows"], ref.S.shape[0],
               lambda i, j: orc.cosine_pair(ref.row_ptr, ref.terms, ref.w, i, j), TAU)


def test_large_allpairs_signature_match():
    """300,000 documents (FP32 form, k = 64): the fp16 compare operand (38 MB) is larger than the
    compare kernel keeps to one L2-resident sweep, so row blocks are dealt to the CTAs round
    robin. Sampled rows (spread over the whole triangle, including the last row blocks) are
    scored by the oracle against every later document; every emitted pair of a sample is
    checked against the oracle's cosine."""
    torch = cuda_or_skip()
    from paper_1810_03099_gb300 import mrc
    c = synth.cached_corpus("precision", n_docs=300_000, length_median=150.0)
    orc = Oracle()
    ref = build_index(c.offsets, c.tokens, c.vocab, Params(k=K, tau=TAU), orc)
    n = ref.S.shape[0]
    with mrc.Context() as ctx:
        idx = mrc.mrc_build_index(ctx, torch.from_numpy(c.offsets).cuda(), torch.from_numpy(c.tokens).cuda(), c.vocab,
                                  mrc.params_default(k=K, tau=TAU))
        buf, total = mrc.mrc_match(ctx, idx, None, TAU, capacity=1 << 24)
        got = mrc.pairs_to_numpy(buf)
        idx.free()
    assert total == got.shape[0] > 0
    rng = np.random.Generator(np.random.PCG64(78))
    rows = np.unique(np.concatenate([rng.choice(n - 1, 24, replace=False), [0, 1, n - 2, n - 3, n - 129, n - 300]]))
    by_row, rowset = {}, set(rows.tolist())
    for i, j, s in zip(got["i"].tolist(), got["j"].tolist(), got["score"].tolist()):
        if i in rowset:
            by_row.setdefault(i, {})[j] = s
    for i in rows.tolist():
        _, _, pj, ps = orc.sig_match(ref.S[i:i + 1], ref.S[i + 1:], TAU - 1e-5)
        want = {i + 1 + int(j): float(s) for j, s in zip(pj, ps)}
        have = by_row.get(i, {})
        for j, s in want.items():
            if j not in have:
                assert abs(s - TAU) <= 1e-5, (i, j, s)
        for j, s in have.items():
            assert j in want, (i, j, s)
            assert abs(s - want[j]) <= 1e-5, (i, j, s, want[j])
    for x in rng.choice(got.shape[0], min(2000, got.shape[0]), replace=False).tolist():
        i, j, s = int(got["i"][x]), int(got["j"][x]), float(got["score"][x])
        assert i < j and abs(s - orc.cos_dense(ref.S[i], ref.S[j])) <= 1e-5


def test_fullsize_simhash_index():
    """The block-table Hamming index at the fingerprint-index benchmark's size (10,000,000
    fingerprints, Hamming <= 3): sampled queries and sampled rows of the all-pairs search, each
    against the oracle's brute-force pairs of that query or row."""
    torch = cuda_or_skip()
    from paper_1810_03099_gb300 import mrc
    orc = Oracle()
    n = 10_000_000
    X = synth.random_fingerprints(n, 51, n_near=100_000, max_flip=4)
    rng = np.random.Generator(np.random.PCG64(52))
    near = rng.choice(np.arange(n - 100_000, n), 8, replace=False)
    Q = np.concatenate([X[near] ^ np.uint64(1 << 9), synth.random_fingerprints(8, 53)])
    ctx = mrc.Context()
    sidx = mrc.simhash_index_build(ctx, torch.from_numpy(X.view(np.int64)).cuda(), HMAX)
    got = mrc.pairs_to_numpy(mrc.simhash_index_match(ctx, sidx, torch.from_numpy(Q.view(np.int64)).cuda())[0])
    _, pi, pj, ph = orc.hamming_pairs(Q, X, HMAX)
    assert sorted(zip(got["i"].tolist(), got["j"].tolist(), got["score"].astype(int).tolist())) == \
        sorted(zip(pi.tolist(), pj.tolist(), ph.tolist()))
    assert len(pi) >= 8
    # all pairs of the index: the pairs of sampled rows i (with j > i)
    allp = mrc.pairs_to_numpy(mrc.simhash_index_match(ctx, sidx, capacity=1 << 22)[0])
    rows = np.concatenate([X.shape[0] - 100_000 - 1 - np.arange(4), near[:4]])
    for i in rows.tolist():
        i = int(i)
        mine = sorted((int(j), int(s)) for a, j, s in zip(allp["i"], allp["j"], allp["score"]) if a == i)
        _, _, rj, rh = orc.hamming_pairs(X[i:i + 1], X[i + 1:], HMAX)
        assert mine == sorted(zip((rj + i + 1).tolist(), rh.tolist())), i
    sidx.free()
    ctx.close()
