"""The threaded driver of the oracle (used to time it on all host cores) gives exactly the
serial oracle's results: same index arrays, same pair lists in the same order."""
import numpy as np

from oracle.oracle import Oracle, Params, build_index
from oracle.threaded import ThreadedOracle, cpu_model, host_cores
from paper_1810_03099_gb300 import synth


def test_threaded_oracle_equals_serial():
    c = synth.make_corpus("tiny", n_docs=700)
    orc = Oracle()
    p = Params(k=16)
    ref = build_index(c.offsets, c.tokens, c.vocab, p, orc)
    t = ThreadedOracle(threads=4, orc=orc)
    try:
        got = t.build_index(c.offsets, c.tokens, c.vocab, p)
        for name in ("row_ptr", "terms", "counts", "df", "part", "w", "S", "F"):
            assert np.array_equal(getattr(got, name), getattr(ref, name)), name
        tot, pi, pj, ps = orc.sig_pairs(ref.S, 0.8)
        tt, gi, gj, gs = t.sig_pairs(ref.S, 0.8)
        assert tt == tot and np.array_equal(gi, pi) and np.array_equal(gj, pj) and np.array_equal(gs, ps)
        tot, hi, hj, hh = orc.hamming_pairs(ref.F, None, 8)
        tt, gi, gj, gh = t.hamming_pairs(ref.F, 8)
        assert tt == tot and np.array_equal(gi, hi) and np.array_equal(gj, hj) and np.array_equal(gh, hh)
    finally:
        t.close()
    assert host_cores() >= 1 and isinstance(cpu_model(), str)
