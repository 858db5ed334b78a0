"""Stream-ordered pair calls (mrc_match_async, cosine_allpairs_async, simhash_match_async,
mrc_ctx_sync): the same kernels as the synchronous calls, so the same pair sets, with the pair
count left on the device and device-side errors reported by mrc_ctx_sync."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1810_03099_gb300 import synth
from tests.gpu_common import cuda_or_skip

pytestmark = pytest.mark.gpu


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


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def triples(M, buf):
    p = M.pairs_to_numpy(buf)
    return sorted(zip(p["i"].tolist(), p["j"].tolist(), p["score"].tolist()))


def run_async(torch, M, ctx, call, cap):
    pairs = torch.empty((cap, 3), dtype=torch.int32, device="cuda")
    count = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    call(pairs, count)
    ctx.sync()
    total = int(count.item())
    return pairs[:min(total, cap)], total


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_match_async_equals_sync(torch, M, ctx, precision):
    c = synth.make_corpus("tiny", n_docs=1500)
    idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), c.vocab,
                            M.params_default(k=64, precision=precision))
    ref, tot = M.mrc_match(ctx, idx, None, 0.7)
    got, tot2 = run_async(torch, M, ctx, lambda p, n: M.mrc_match_async(ctx, idx, p, n, None, 0.7), tot + 10)
    assert tot2 == tot and triples(M, got) == triples(M, ref)
    # queries, and a pair buffer smaller than the total: the count is still the total
    Q = synth.random_signatures(200, 64, 5, density=0.5)
    refq, totq = M.mrc_match(ctx, idx, dev(torch, Q), 0.5)
    gotq, totq2 = run_async(torch, M, ctx, lambda p, n: M.mrc_match_async(ctx, idx, p, n, dev(torch, Q), 0.5),
                            max(totq // 2, 1))
    assert totq2 == totq
    assert set(triples(M, gotq)) <= set(triples(M, refq))
    idx.free()


def test_simhash_and_cosine_async_equal_sync(torch, M, ctx):
    c = synth.make_corpus("tiny", n_docs=900)
    idx = M.mrc_build_index(ctx, dev(torch, c.offsets), dev(torch, c.tokens), c.vocab, M.params_default(k=16))
    F = M.mrc_index_export(ctx, idx)["simhash"].view(np.int64)
    ref, tot = M.simhash_match(ctx, dev(torch, F), None, 5)
    got, tot2 = run_async(torch, M, ctx, lambda p, n: M.simhash_match_async(ctx, dev(torch, F), p, n, None, 5),
                          tot + 1)
    assert tot2 == tot and triples(M, got) == triples(M, ref)
    # host input (copied before the call returns)
    got, tot3 = run_async(torch, M, ctx, lambda p, n: M.simhash_match_async(ctx, F, p, n, F[:50], 5), tot + 100)
    ref, tot4 = M.simhash_match(ctx, F, F[:50], 5)
    assert tot3 == tot4 and triples(M, got) == triples(M, ref)
    ref, tot = M.cosine_allpairs(ctx, idx, dev(torch, c.offsets), dev(torch, c.tokens), 0.6)
    got, tot2 = run_async(torch, M, ctx, lambda p, n: M.cosine_allpairs_async(
        ctx, idx, dev(torch, c.offsets), dev(torch, c.tokens), p, n, 0.6), tot + 1)
    assert tot2 == tot and triples(M, got) == triples(M, ref)
    idx.free()


def test_async_candidate_overflow_reported(torch, M, ctx):
    """1,500 identical documents: every one of the 1,124,250 pairs is a candidate of the E4M3
    compare, more than the 2^20-entry candidate buffer. The synchronous call grows the buffer and
    repeats; the stream-ordered call keeps what fits and mrc_ctx_sync reports MRC_ERR_CAPACITY."""
    n, doc = 1500, np.arange(40, dtype=np.int32) * 7
    offsets = np.arange(n + 1, dtype=np.int64) * doc.size
    tokens = np.tile(doc, n)
    idx = M.mrc_build_index(ctx, dev(torch, offsets), dev(torch, tokens), 400,
                            M.params_default(k=8, precision=1, select_mode=0))  # every term
    _, tot = M.mrc_match(ctx, idx, None, 0.9, capacity=16, grow=False)
    assert tot == n * (n - 1) // 2
    pairs = torch.empty((16, 3), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    M.mrc_match_async(ctx, idx, pairs, count, None, 0.9)
    with pytest.raises(M.MrcError) as e:
        ctx.sync()
    assert e.value.status == M.MRC_ERR_CAPACITY
    assert 0 < int(count.item()) <= 1 << 20
    ctx.sync()  # the error was cleared by the previous sync
    idx.free()


def test_async_argument_errors(torch, M, ctx):
    c = synth.make_corpus("tiny", n_docs=100)
    idx = M.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, M.params_default(k=8))
    with pytest.raises(TypeError):
        M.mrc_match_async(ctx, idx, np.zeros((4, 3), np.int32), torch.zeros(1, dtype=torch.int64, device="cuda"))
    # device pairs but a host count: refused by the library
    pairs = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    hc = np.zeros(1, np.int64)
    st = ctx.lib.mrc_match_async(ctx.handle, idx.handle, None, 0, 0.9, pairs.data_ptr(), 4, hc.ctypes.data)
    assert st == M.MRC_ERR_INVALID
    ctx.sync()
    idx.free()
