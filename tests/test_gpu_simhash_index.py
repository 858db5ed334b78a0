"""Block-table Hamming index (mrc_simhash_index_*) against the oracle's brute-force Hamming
pairs: the same pair set with the same distances, each pair once, for all-pairs and
query x index searches, several distances, skewed buckets and degenerate inputs."""
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


@pytest.fixture(scope="module")
def orc():
    from oracle.oracle import Oracle
    return Oracle()


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def triples(M, buf):
    p = M.pairs_to_numpy(buf)
    return sorted(zip(p["i"].tolist(), p["j"].tolist(), p["score"].astype(int).tolist()))


def oracle_triples(orc, a, b, h):
    _, pi, pj, ph = orc.hamming_pairs(a, b, h)
    return sorted(zip(pi.tolist(), pj.tolist(), ph.tolist()))


def skewed_fingerprints(n, seed):
    """Near copies that agree on several blocks (one flipped bit in block 0, 1, 2 or 3, two flips
    in two blocks), hundreds of exact duplicates, and words that share one 16-bit block value."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = rng.integers(0, 2**63, size=n // 4, dtype=np.int64).astype(np.uint64) * np.uint64(2) + np.uint64(1)
    out = [base]
    for shift in (0, 17, 33, 49):
        out.append(base[: n // 16] ^ np.uint64(1 << shift))
    out.append(base[: n // 32] ^ np.uint64((1 << 3) | (1 << 40)))
    out.append(np.full(300, base[0], np.uint64))
    same_block = rng.integers(0, 2**63, size=500, dtype=np.int64).astype(np.uint64) & ~np.uint64(0xFFFF)
    out.append(same_block | np.uint64(0x1234))
    return np.concatenate(out)


@pytest.mark.parametrize("h", [0, 1, 3, 5, 8])
def test_all_pairs_equal_brute_force(torch, M, ctx, orc, h):
    X = synth.random_fingerprints(6001, 31 + h, n_near=1500, max_flip=h + 2)
    sidx = M.simhash_index_build(ctx, dev(torch, X), h)
    got = triples(M, M.simhash_index_match(ctx, sidx)[0])
    assert got == oracle_triples(orc, X, None, h) and len(got) > 0
    sidx.free()


def test_query_search_skewed_and_lower_distance(torch, M, ctx, orc):
    X = skewed_fingerprints(8000, 5)
    rng = np.random.Generator(np.random.PCG64(6))
    Q = np.concatenate([X[rng.choice(X.shape[0], 400, replace=False)] ^ np.uint64(1 << 20),
                        synth.random_fingerprints(333, 7)])
    sidx = M.simhash_index_build(ctx, dev(torch, X), 3)
    for h in (3, 2, 0):
        got = triples(M, M.simhash_index_match(ctx, sidx, dev(torch, Q), h)[0])
        assert got == oracle_triples(orc, Q, X, h)
    got = triples(M, M.simhash_index_match(ctx, sidx)[0])
    assert got == oracle_triples(orc, X, None, 3)
    # host queries and host pairs
    got = M.simhash_index_match(ctx, sidx, Q, 3, device=None)[0]
    assert sorted(zip(got["i"].tolist(), got["j"].tolist(), got["score"].astype(int).tolist())) == \
        oracle_triples(orc, Q, X, 3)
    with pytest.raises(M.MrcError) as e:
        M.simhash_index_match(ctx, sidx, dev(torch, Q), 4)
    assert e.value.status == M.MRC_ERR_INVALID
    sidx.free()


def test_degenerate_inputs_and_sixteen_blocks(torch, M, ctx, orc):
    X = synth.random_fingerprints(3000, 9, n_near=900, max_flip=16)
    sidx = M.simhash_index_build(ctx, dev(torch, X), 15)  # 16 blocks of 4 bits
    got = triples(M, M.simhash_index_match(ctx, sidx, dev(torch, X[:200]), 15)[0])
    assert got == oracle_triples(orc, X[:200], X, 15)
    sidx.free()
    empty = M.simhash_index_build(ctx, np.zeros(0, np.uint64), 3)
    assert M.simhash_index_match(ctx, empty)[1] == 0
    assert M.simhash_index_match(ctx, empty, dev(torch, X[:5]))[1] == 0
    empty.free()
    one = M.simhash_index_build(ctx, X[:1], 3)
    assert M.simhash_index_match(ctx, one)[1] == 0
    assert triples(M, M.simhash_index_match(ctx, one, dev(torch, X[:1]))[0]) == [(0, 0, 0)]
    one.free()
    with pytest.raises(M.MrcError):
        M.simhash_index_build(ctx, X, 16)


def test_large_index_query_search(torch, M, ctx, orc):
    """A 100,000-fingerprint index searched by 500 queries (near copies and random words)."""
    X = synth.random_fingerprints(100_000, 11, n_near=20_000, max_flip=4)
    rng = np.random.Generator(np.random.PCG64(12))
    Q = X[rng.choice(X.shape[0], 500, replace=False)].copy()
    Q[::2] ^= np.uint64(0b1011 << 30)
    sidx = M.simhash_index_build(ctx, dev(torch, X), 3)
    got = triples(M, M.simhash_index_match(ctx, sidx, dev(torch, Q), 3)[0])
    assert got == oracle_triples(orc, Q, X, 3) and len(got) >= 250
    sidx.free()


def test_capacity_overflow_keeps_a_subset_and_reports_the_total(torch, M, ctx, orc):
    X = skewed_fingerprints(8000, 5)
    want = oracle_triples(orc, X, None, 3)
    sidx = M.simhash_index_build(ctx, dev(torch, X), 3)
    for cap in (0, 1, 1000):
        buf, total = M.simhash_index_match(ctx, sidx, capacity=cap, grow=False)
        assert total == len(want)
        got = triples(M, buf) if cap > 0 else []
        assert len(got) == min(cap, len(want)) and set(got) <= set(want)
    # host pairs grown to the total
    got = M.simhash_index_match(ctx, sidx, capacity=16, device=None)[0]
    assert sorted(zip(got["i"].tolist(), got["j"].tolist(), got["score"].astype(int).tolist())) == want
    sidx.free()
