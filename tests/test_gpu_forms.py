"""Batching and serving forms, through the C ABI.

* A graph-captured batch gives the pair set of the oracle (query x index, FP32 form:
  equal except within 1e-5 of tau) and exactly what the eager path (mrc_signature then
  mrc_match) gives, padded or not, with either compare tile width.
* A served request's pairs are bit-identical alone and in the mix of a continuous batch.
* Admission by free device memory: a fake low free-memory figure admits fewer slots.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle, Params, build_index, signature
from paper_1810_03099_gb300 import synth
from tests.gpu_common import cuda_or_skip, pair_dict

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = cuda_or_skip()
    from paper_1810_03099_gb300 import mrc
    c = synth.make_corpus(synth.SPECS["tiny"].with_(n_docs=3000))
    ctx = mrc.Context()
    orc = Oracle()
    yield {"torch": torch, "mrc": mrc, "c": c, "ctx": ctx, "orc": orc}
    ctx.close()


def _queries(c, n, seed):
    q = synth.make_corpus(synth.SPECS["tiny"].with_(n_docs=n, vocab=c.vocab, seed=seed, dup_frac=0.0))
    # half of the queries are copies (with edits) of index documents, so that matches exist
    rng = np.random.Generator(np.random.PCG64(seed))
    docs = [q.doc(i).copy() for i in range(n)]
    for i in range(0, n, 2):
        src = c.doc(int(rng.integers(0, c.n_docs))).copy()
        if src.size > 4:
            src[rng.integers(0, src.size)] = int(rng.integers(0, c.vocab))
        docs[i] = src
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum([d.size for d in docs])
    return offs, np.concatenate(docs).astype(np.int32)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_matches_oracle_and_eager(env, precision):
    mrc, ctx, c, orc, torch = env["mrc"], env["ctx"], env["c"], env["orc"], env["torch"]
    p = Params(k=32)  # stored signatures and rescoring use FP32 weights in every form
    ref = build_index(c.offsets, c.tokens, c.vocab, p, orc)
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=32, precision=precision))
    qo, qt = _queries(c, 100, 5)
    tau = 0.9
    # eager path
    sig, _ = mrc.mrc_signature(ctx, idx, qo, qt)
    eager = mrc.pairs_to_numpy(mrc.mrc_match(ctx, idx, sig, tau, device=None)[0])
    eset = sorted(eager.tolist())
    Sq, _, _ = signature(ref, qo, qt, orc)
    tot, pi, pj, ps = orc.sig_match(Sq, ref.S, tau)
    od = pair_dict(pi, pj, ps)
    assert tot > 20
    for max_docs, tile in ((100, 0), (128, 128), (256, 256)):
        b = mrc.Batch(ctx, idx, max_docs, 200000, tau, capacity=1 << 16, tile_n=tile)
        assert b.kernel_nodes == 1  # the whole pipeline is one persistent kernel
        for _ in range(2):  # replays are repeatable
            b.launch(qo, qt)
            got, total = b.wait()
            assert total == got.shape[0]
            assert sorted(got.tolist()) == eset
        b.free()
    gd = pair_dict(eager["i"], eager["j"], eager["score"])
    for pr, sc in gd.items():
        o = od.get(pr, orc.cos_dense(Sq[pr[0]], ref.S[pr[1]]))
        assert o >= tau - 1e-5 and abs(sc - o) <= 1e-5
    missed = [pr for pr, o in od.items() if pr not in gd and o > tau + 1e-5]
    assert len(missed) <= (0 if precision == 0 else 0.01 * len(od))
    # against the FP64 pair set: recall and precision >= 0.99
    g, o = set(gd), set(od)
    assert len(g & o) >= 0.99 * len(o) and len(g & o) >= 0.99 * len(g)
    idx.free()


@pytest.mark.parametrize("precision", [0, 1])
def test_persistent_batch_every_document_path_hamming_and_errors(env, precision):
    """The one-kernel batch on documents of every signature-pass path (empty; short, one warp;
    long, a whole CTA; 9,000 and 20,000 tokens, several hashing passes) gives the eager calls'
    signature pairs (same scores), the fingerprint index's Hamming pairs, and per-query offsets
    that delimit each query's pairs. Offsets that decrease are reported (MRC_ERR_INVALID) and the
    next launch is correct again; so is a launch of fewer documents than the one before."""
    mrc, ctx, c, torch = env["mrc"], env["ctx"], env["c"], env["torch"]
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=64, precision=precision))
    fps = mrc.index_simhash(ctx, idx, torch.empty(c.n_docs, dtype=torch.int64, device="cuda"))
    shx = mrc.simhash_index_build(ctx, fps, 3)
    n = 90
    qo, qt = _queries(c, n, 23)
    docs = [qt[qo[i]:qo[i + 1]].copy() for i in range(n)]
    rng = np.random.Generator(np.random.PCG64(41))
    docs[1] = np.zeros(0, np.int32)
    docs[3] = rng.integers(0, c.vocab, 3000).astype(np.int32)
    d7 = c.doc(7)
    docs[5] = np.tile(d7, 20000 // max(d7.size, 1) + 1)[:20000].astype(np.int32)  # index document 7, repeated
    docs[8] = rng.integers(0, c.vocab, 9000).astype(np.int32)
    docs[11] = c.doc(11).copy()  # an exact copy: Hamming distance 0
    offs = np.zeros(n + 1, np.int64)
    offs[1:] = np.cumsum([d.size for d in docs])
    toks = np.concatenate(docs).astype(np.int32)

    def eager(o, t):
        sig, sh = mrc.mrc_signature(ctx, idx, o, t)
        sp = mrc.pairs_to_numpy(mrc.mrc_match(ctx, idx, sig, 0.9, device=None)[0])
        hp = mrc.pairs_to_numpy(mrc.simhash_index_match(ctx, shx, torch.from_numpy(sh.view(np.int64)).cuda(),
                                                        3, device=None)[0])
        return sorted(sp.tolist()), sorted(hp.tolist())

    want_s, want_h = eager(offs, toks)
    assert len(want_s) > 20 and len(want_h) > 0
    b = mrc.Batch(ctx, idx, 128, 80000, 0.9, capacity=1 << 16)
    b.attach_simhash(shx, 3, 1 << 16)
    assert b.kernel_nodes == 1

    def check(o, t, ws, wh):
        b.launch(o, t)
        got, total, qoff = b.wait(offsets=True)
        hp, htot, hqoff = b.hamming(offsets=True)
        assert sorted(got.tolist()) == ws and total == len(ws)
        assert sorted(hp.tolist()) == wh and htot == len(wh)
        for pairs, off in ((got, qoff), (hp, hqoff)):
            assert off[0] == 0 and off[-1] == len(pairs) and np.all(np.diff(off) >= 0)
            for q in range(len(off) - 1):
                assert np.all(pairs["i"][off[q]:off[q + 1]] == q)

    check(offs, toks, want_s, want_h)
    ph = b.phase_ns()  # the persistent kernel's phases, timed on the device
    assert len(ph) == 6 and all(v >= 0 for v in ph.values()) and ph["compare"] > 0
    bad = offs.copy()
    bad[4] = bad[2] - 1  # document 3 ends before it starts
    b.launch(bad, toks)
    with pytest.raises(mrc.MrcError) as ei:
        b.wait()
    assert ei.value.status == mrc.MRC_ERR_INVALID
    check(offs, toks, want_s, want_h)
    m = 17  # fewer documents than the launch before
    ws, wh = eager(offs[:m + 1], toks[:offs[m]])
    check(offs[:m + 1], toks[:offs[m]], ws, wh)
    b.free()
    shx.free()
    idx.free()


def test_batch_runner_buckets_and_autotune(env, tmp_path):
    mrc, ctx, c = env["mrc"], env["ctx"], env["c"]
    from paper_1810_03099_gb300 import batching
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=32))
    qo, qt = _queries(c, 300, 9)
    batches = batching.make_batches(qo, qt, [1, 7, 64, 200, 33], seed=3)
    knobs = batching.autotune(ctx, idx, 64, 64 * 5000, batches[2][:2], reps=1, cache=str(tmp_path / "t.json"),
                              rings=(0, 3), prefetches=(0, 8))
    assert knobs["tile_n"] in (128, 256) and knobs["ring"] in (0, 3) and knobs["prefetch"] in (0, 8)
    assert batching.autotune(ctx, idx, 64, 64 * 5000, batches[2][:2], cache=str(tmp_path / "t.json")) == knobs
    runner = batching.BatchRunner(ctx, idx, 0.9, max_docs=256, max_doc_tokens=5000, autotune=False)
    for offs, toks, pick in batches:
        got, total = runner.run(offs, toks)
        sig, _ = mrc.mrc_signature(ctx, idx, offs, toks)
        want = mrc.pairs_to_numpy(mrc.mrc_match(ctx, idx, sig, 0.9, device=None)[0])
        assert sorted(got.tolist()) == sorted(want.tolist())
    runner.free()
    idx.free()


def test_serving_alone_equals_mix(env):
    mrc, ctx, c = env["mrc"], env["ctx"], env["c"]
    from paper_1810_03099_gb300 import serving
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=32))
    qo, qt = _queries(c, 400, 13)
    docs = [qt[qo[i]:qo[i + 1]] for i in range(400)]
    arrivals = synth.poisson_arrivals(200000.0, 400, seed=21)
    srv = serving.Server(ctx, idx, 0.9, micro_batch=32, deadline_s=2e-4, slots=3, max_doc_tokens=5000)
    mixed = srv.run(docs, arrivals)
    rep = serving.latency_report(mixed, srv.wall_s)
    assert rep["requests"] == 400 and rep["p99_ms"] >= rep["p50_ms"] > 0
    alone = serving.Server(ctx, idx, 0.9, micro_batch=1, deadline_s=0.0, slots=1, max_doc_tokens=5000)
    single = alone.run(docs[:120], np.zeros(120))
    for a, b in zip(mixed[:120], single):  # bit-identical scores
        assert sorted(zip(a.pairs["j"].tolist(), a.pairs["score"].tolist())) == \
            sorted(zip(b.pairs["j"].tolist(), b.pairs["score"].tolist()))
    assert sum(len(r.pairs) for r in mixed) > 50
    # results in a small ring of pinned memory: regions are reused and the requests that still
    # view them get copies first; every request keeps its pairs
    ring = max(32, sum(len(r.pairs) for r in mixed) // 4)
    small = serving.Server(ctx, idx, 0.9, micro_batch=32, deadline_s=2e-4, slots=3, max_doc_tokens=5000,
                           result_pairs=ring)
    again = small.run(docs, arrivals)
    assert small.ring.evicted > 0
    for a, b in zip(mixed, again):
        assert sorted(zip(a.pairs["j"].tolist(), a.pairs["score"].tolist())) == \
            sorted(zip(b.pairs["j"].tolist(), b.pairs["score"].tolist()))
    small.free()
    srv.free()
    alone.free()
    idx.free()


def test_serving_admission_by_free_memory(env):
    mrc, ctx, c = env["mrc"], env["ctx"], env["c"]
    from paper_1810_03099_gb300 import serving
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=32))
    foot = serving.slot_footprint(idx, 32, 32 * 5000, 1 << 16)
    s = serving.Server(ctx, idx, micro_batch=32, slots=8, max_doc_tokens=5000, hbm_fraction=1.0,
                       free_bytes=3 * foot + 1)
    assert s.admitted_slots == 3
    s.free()
    with pytest.raises(MemoryError):
        serving.Server(ctx, idx, micro_batch=32, slots=8, max_doc_tokens=5000, hbm_fraction=1.0, free_bytes=foot - 1)
    idx.free()


def test_serving_signature_and_hamming_pairs_match_oracle(env):
    """The serving form with its Hamming leg: against a resident index (FP16 signatures) and a
    block-table index of its Simhashes, every served request gets its signature pairs (the
    oracle's query x index pair set, equal except within 1e-5 of tau; scores within 1e-5) and
    its Hamming pairs (bit-exact: the oracle's fingerprints of the request against the index's,
    distance <= 3)."""
    mrc, ctx, c, orc, torch = env["mrc"], env["ctx"], env["c"], env["orc"], env["torch"]
    from paper_1810_03099_gb300 import serving
    p = Params(k=32)
    ref = build_index(c.offsets, c.tokens, c.vocab, p, orc)
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=32, precision=2))
    fps = mrc.index_simhash(ctx, idx, torch.empty(c.n_docs, dtype=torch.int64, device="cuda"))
    shx = mrc.simhash_index_build(ctx, fps, 3)
    n = 240
    qo, qt = _queries(c, n, 17)
    docs = [qt[qo[i]:qo[i + 1]] for i in range(n)]
    srv = serving.Server(ctx, idx, 0.9, micro_batch=32, deadline_s=2e-4, slots=3, max_doc_tokens=5000,
                         simhash_index=shx, hamming_max=3)
    reqs = srv.run(docs, synth.poisson_arrivals(100000.0, n, seed=5))
    Sq, Fq, _ = signature(ref, qo, qt, orc)
    tot, pi, pj, ps = orc.sig_match(Sq, ref.S, 0.9)
    od = pair_dict(pi, pj, ps)
    gd = {(r.rid, int(j)): float(s) for r in reqs for j, s in zip(r.pairs["j"], r.pairs["score"])}
    for pr, sc in gd.items():
        o = od.get(pr, orc.cos_dense(Sq[pr[0]], ref.S[pr[1]]))
        assert o >= 0.9 - 1e-5 and abs(sc - o) <= 1e-5, (pr, sc, o)
    assert all(pr in gd for pr, o in od.items() if o > 0.9 + 1e-5)
    htot, hi, hj, hh = orc.hamming_pairs(Fq, ref.F, 3)
    want = sorted(zip(hi.tolist(), hj.tolist(), hh.tolist()))
    got = sorted((r.rid, int(j), int(s)) for r in reqs for j, s in zip(r.hamming["j"], r.hamming["score"]))
    assert got == want and htot > 20
    assert tot > 20
    srv.free()
    shx.free()
    idx.free()
