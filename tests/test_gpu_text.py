"""Character 3-grams of raw text (mrc_text_grams) against the oracle: bit-exact offsets and ids
on synthetic NEWS20-shaped text, at tile boundaries, on unaligned and host buffers, with
capacity overflow and invalid offsets, and the whole path from text to pairs."""
from __future__ import annotations

import numpy as np
import pytest

from oracle.oracle import GRAM_VOCAB, MODE_ALL, MODE_DF1, Params, build_index
from paper_1810_03099_gb300 import synth
from tests.gpu_common import compare_pairs, cuda_or_skip, pair_dict

pytestmark = pytest.mark.gpu

TILE = 8192  # bytes per CTA of the 3-gram kernel: boundary cases are placed around multiples of it


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
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def text_csr(docs):
    offs = np.zeros(len(docs) + 1, np.int64)
    offs[1:] = np.cumsum([len(d) for d in docs])
    return offs, np.frombuffer(b"".join(docs), np.uint8).copy()


def boundary_docs():
    """Documents whose boundaries and letter runs straddle tile edges: a 20,000-letter run, runs
    ending 1-3 bytes before and after multiples of the tile, empty and 1-2 byte documents at
    tile edges, separators only, upper case and UTF-8 bytes."""
    rng = np.random.Generator(np.random.PCG64(21))
    letters = np.frombuffer(b"abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ", np.uint8)
    docs = [bytes(rng.choice(letters, size=TILE - 1)), b"", b"ab", b"c", bytes(rng.choice(letters, size=3)),
            bytes(rng.choice(letters, size=20000)), b" .,\n\t7", b"", b"x"]
    # pad so that the next document starts exactly on a tile edge, then one that ends on the next
    used = sum(len(d) for d in docs)
    docs.append(bytes(rng.choice(letters, size=(-used) % TILE)))
    docs.append(bytes(rng.choice(letters, size=TILE)))
    docs.append(b"Ab\xc3\xa9cdE-fgh")
    docs += [bytes(rng.choice(letters, size=int(rng.integers(0, 5)))) for _ in range(300)]
    return docs


def check_grams(M, ctx, orc, torch, offs, text, device=True, shift=0):
    go_ref, g_ref = orc.char3grams(offs, text)
    if device:
        t = dev(torch, np.concatenate([np.zeros(shift, np.uint8), text]))[shift:]
        go, g = M.mrc_text_grams(ctx, dev(torch, offs), t)
        go, g = go.cpu().numpy(), g.cpu().numpy()
    else:
        go, g = M.mrc_text_grams(ctx, offs, text)
    assert np.array_equal(go, go_ref)
    assert np.array_equal(g, g_ref)
    return go_ref, g_ref


def test_text_grams_synthetic_text(torch, M, ctx, orc):
    tc = synth.make_text_corpus("tiny", n_docs=700)
    go, g = check_grams(M, ctx, orc, torch, tc.offsets, tc.text)
    assert g.shape[0] > tc.n_bytes // 3 and int(g.max()) < GRAM_VOCAB


@pytest.mark.parametrize("shift", [0, 1, 3, 8])
def test_text_grams_tile_boundaries_and_alignment(torch, M, ctx, orc, shift):
    offs, text = text_csr(boundary_docs())
    assert offs[10] % TILE == 0
    check_grams(M, ctx, orc, torch, offs, text, shift=shift)


def test_text_grams_host_buffers_and_degenerate_inputs(torch, M, ctx, orc):
    offs, text = text_csr(boundary_docs())
    check_grams(M, ctx, orc, torch, offs, text, device=False)
    # every document empty; no documents; a single short document
    for docs in ([b"", b"", b""], [b"ab"], [b"abc"]):
        check_grams(M, ctx, orc, torch, *text_csr(docs))
    go, g = M.mrc_text_grams(ctx, np.zeros(1, np.int64), np.zeros(0, np.uint8))
    assert go.tolist() == [0] and g.shape[0] == 0


def test_text_grams_capacity_and_invalid_offsets(torch, M, ctx, orc):
    offs, text = text_csr(boundary_docs())
    go_ref, g_ref = orc.char3grams(offs, text)
    cap = g_ref.shape[0] // 2
    go = torch.empty(offs.shape[0], dtype=torch.int64, device="cuda")
    g = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(M.MrcError) as e:
        M.mrc_text_grams(ctx, dev(torch, offs), dev(torch, text), go, g)
    assert e.value.status == M.MRC_ERR_CAPACITY
    assert np.array_equal(go.cpu().numpy(), go_ref) and np.array_equal(g.cpu().numpy(), g_ref[:cap])
    for bad in ([0, 10, 5, 20], [1, 10, 20], [0, 30, 20]):
        bo = np.array(bad, np.int64)
        t = np.frombuffer(b"abcdefghijklmnopqrstuvwxyz0123456789", np.uint8)[:bad[-1]].copy()
        with pytest.raises(M.MrcError) as e:
            M.mrc_text_grams(ctx, dev(torch, bo), dev(torch, t))
        assert e.value.status == M.MRC_ERR_INVALID
    ctx.sync()


def test_text_to_pairs_matches_oracle(torch, M, ctx, orc):
    """Text -> 3-grams -> index -> signature and Simhash pairs, against the oracle run on the
    oracle's own 3-grams of the same text."""
    tc = synth.make_text_corpus("tiny", n_docs=1500)
    go_ref, g_ref = orc.char3grams(tc.offsets, tc.text)
    go, g = M.mrc_text_grams(ctx, dev(torch, tc.offsets), dev(torch, tc.text))
    # every 3-gram of the corpus as the reference (selection ALL): 3-grams are dense, so the
    # default REGION band (df <= N/100) holds only a few dozen of them on this text
    p = Params(k=32, mode=MODE_ALL)
    ref = build_index(go_ref, g_ref, GRAM_VOCAB, p, orc)
    idx = M.mrc_build_index(ctx, go, g, GRAM_VOCAB, M.params_default(k=32, select_mode=MODE_ALL))
    ex = M.mrc_index_export(ctx, idx)
    assert np.array_equal(ex["df"].astype(np.int64), ref.df)
    assert np.array_equal(ex["simhash"], ref.F)
    assert np.abs(ex["sig"].astype(np.float64) - ref.S).max() <= 2e-6
    tot, pi, pj, _ = orc.hamming_pairs(ref.F, None, 3)
    buf, total = M.simhash_match(ctx, dev(torch, ex["simhash"].view(np.int64)), None, 3)
    got = M.pairs_to_numpy(buf)
    assert total == tot and sorted(zip(got["i"].tolist(), got["j"].tolist())) == sorted(zip(pi.tolist(), pj.tolist()))
    # signature pairs: the oracle's set (apart from scores within 1e-5 of tau), and the
    # near-duplicates of the text among them
    tot, pi, pj, ps = orc.sig_pairs(ref.S, 0.9)
    got = M.pairs_to_numpy(M.mrc_match(ctx, idx, None, 0.9)[0])
    compare_pairs(pair_dict(got["i"], got["j"], got["score"]), pair_dict(pi, pj, ps), 0.9, 1e-5, 1e-5,
                  lambda i, j: orc.cos_dense(ref.S[i], ref.S[j]))
    have = set(zip(got["i"].tolist(), got["j"].tolist()))
    dups = np.nonzero(tc.words.dup_src >= 0)[0]
    found = sum((int(tc.words.dup_src[i]), int(i)) in have for i in dups)
    assert found >= 0.9 * len(dups)
    idx.free()


def test_text_grams_news20_sized_text(torch, M, ctx, orc):
    """The NEWS20-shaped text (18,846 documents, about 55 MB) through the same launch shape the
    benchmark times, every id compared."""
    tc = synth.make_text_corpus("news20")
    check_grams(M, ctx, orc, torch, tc.offsets, tc.text)


def test_study_error_statistics_match_oracle(torch, M, ctx, orc):
    """The reference-selection study's statistic (Eq. 2, Eq. 3: MAE and variance of the signature
    cosine against the exact cosine over all pairs), from the GPU's all-pair lists (tau = -1 for
    signatures, 0 for the exact cosine), equals the oracle's on 300 text documents."""
    m = 300
    tc = synth.make_text_corpus("tiny", n_docs=m)
    go_ref, g_ref = orc.char3grams(tc.offsets, tc.text)
    for mode, k, L in ((MODE_ALL, 60, -1), (MODE_DF1, 30, 500)):
        ref = build_index(go_ref, g_ref, GRAM_VOCAB, Params(k=k, mode=mode, L=L), orc)
        _, pi, pj, ps = orc.sig_pairs(ref.S, -1.0)
        _, ci, cj, cs = orc.cosine_pairs(ref.row_ptr, ref.terms, ref.w, 0.0)
        assert pi.shape[0] == ci.shape[0] == m * (m - 1) // 2
        ost = orc.error_stats(ps, cs)  # both lists in row-major (i, j) order
        go, g = M.mrc_text_grams(ctx, dev(torch, tc.offsets), dev(torch, tc.text))
        idx = M.mrc_build_index(ctx, go, g, GRAM_VOCAB, M.params_default(k=k, select_mode=mode, L=L))
        sig = M.pairs_to_numpy(M.mrc_match(ctx, idx, None, -1.0, capacity=m * m)[0])
        ex = M.pairs_to_numpy(M.cosine_allpairs(ctx, idx, go, g, 0.0, capacity=m * m)[0])
        order_s = np.lexsort((sig["j"], sig["i"]))
        order_e = np.lexsort((ex["j"], ex["i"]))
        assert np.array_equal(sig["i"][order_s], pi) and np.array_equal(sig["j"][order_s], pj)
        assert np.array_equal(ex["i"][order_e], ci) and np.array_equal(ex["j"][order_e], cj)
        e = sig["score"][order_s].astype(np.float64) - ex["score"][order_e].astype(np.float64)
        assert abs(np.abs(e).mean() - ost["mae"]) < 1e-5
        assert abs(e.var() - ost["var"]) < 1e-5
        idx.free()
