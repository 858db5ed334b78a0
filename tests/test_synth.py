"""The seeded generator: deterministic, shaped as specified, near-duplicates as planned."""
import numpy as np

from paper_1810_03099_gb300 import synth


def test_deterministic_and_shaped():
    a = synth.make_corpus("tiny")
    b = synth.make_corpus("tiny")
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.tokens, b.tokens)
    assert a.n_docs == 2000 and a.offsets[0] == 0 and a.offsets[-1] == a.tokens.shape[0]
    lens = a.lengths()
    assert lens.min() >= 5 and lens.max() <= 10000
    assert 80 < np.median(lens) < 180  # lognormal median 120
    assert a.tokens.min() >= 0 and a.tokens.max() < 5000
    c = synth.make_corpus("tiny", seed=7)
    assert not np.array_equal(a.tokens[:1000], c.tokens[:1000])


def test_near_duplicates():
    c = synth.make_corpus("tiny")
    dups = np.nonzero(c.dup_src >= 0)[0]
    assert len(dups) == 100  # 5 % of 2000
    for i in dups[:50]:
        j = c.dup_src[i]
        assert j < i
        a, b = c.doc(int(i)), c.doc(int(j))
        assert a.shape == b.shape
        diff = int((a != b).sum())
        assert diff <= c.edits[i] and c.edits[i] >= 1
        assert c.edits[i] <= max(1, round(0.10 * b.shape[0]))


def test_exact_duplicates_with_zero_edits():
    spec = synth.SPECS["tiny"].with_(n_docs=200, edit_lo=0.0, edit_hi=0.0)
    c = synth.make_corpus(spec)
    for i in np.nonzero(c.dup_src >= 0)[0]:
        assert np.array_equal(c.doc(int(i)), c.doc(int(c.dup_src[i])))


def test_loguniform_lengths():
    c = synth.make_corpus("batch_queries", n_docs=400)
    lens = c.lengths()
    assert lens.min() >= 20 and lens.max() <= 20000
    # log-uniform: about a third of the mass below 20 * 10
    assert 0.2 < np.mean(lens < 200) < 0.5


def test_fingerprints_and_signatures_helpers():
    f = synth.random_fingerprints(100, 3, n_near=20, max_flip=3)
    assert f.dtype == np.uint64 and f.shape == (100,)
    s = synth.random_signatures(10, 8, 4)
    assert s.dtype == np.float32 and (s >= 0).all() and (s == 0).any()


def test_text_corpus_is_seeded_and_well_formed():
    a = synth.make_text_corpus("tiny", n_docs=300)
    b = synth.make_text_corpus("tiny", n_docs=300)
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.text, b.text)
    assert a.offsets[0] == 0 and np.all(np.diff(a.offsets) > 0) and a.offsets[-1] == a.n_bytes
    # every document ends with a separator byte; letters of both cases and UTF-8 bytes occur
    seps = set(b" \n,.'-7\t")
    assert all(a.text[e - 1] in seps for e in a.offsets[1:].tolist())
    assert (a.text >= ord("A")).any() and ((a.text >= ord("A")) & (a.text <= ord("Z"))).any()
    assert (a.text == 0xC3).any()
    # a near-duplicate's text is its source's word sequence with a few words replaced
    i = int(np.nonzero(a.words.dup_src >= 0)[0][0])
    assert a.words.edits[i] >= 1
