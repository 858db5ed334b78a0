"""The serving form's ring of result memory (host logic, no GPU): regions handed out in order
and wrapping around; a request's pairs stay its own whatever later batches overwrite."""
import numpy as np

from paper_1810_03099_gb300 import mrc, serving


class _Req:
    pass


def test_ring_keeps_every_held_request_intact():
    rng = np.random.default_rng(1)
    ring = serving._Ring(100, "pairs")
    held = []
    for batch in range(3000):
        m = int(rng.integers(0, 70))
        start = ring.take(m)
        assert start is not None and 0 <= start and start + m <= ring.n
        ring.buf["i"][start:start + m] = batch  # the batch's DMA into its region
        reqs = [_Req() for _ in range(3)]
        for r in reqs:
            r.pairs = ring.buf[start:start + m]
            r.batch = batch
        ring.keep(start, m, reqs)
        held += reqs
        if batch % 7 == 0:
            held = held[len(held) // 2:]  # the caller drops some requests (freed by refcount)
        for r in held[-40:]:
            assert np.all(r.pairs["i"] == r.batch)
    assert all(np.all(r.pairs["i"] == r.batch) for r in held)
    assert ring.evicted > 0
    assert ring.take(101) is None  # larger than the arena: the caller copies it on its own


def test_ring_skips_dropped_requests():
    ring = serving._Ring(10, "pairs")
    a = ring.take(6)
    r = _Req()
    r.pairs = ring.buf[a:a + 6]
    ring.keep(a, 6, [r])
    del r
    ring.take(8)  # overlaps the dropped request's region: nothing to copy
    assert ring.evicted == 0
    assert mrc.PAIR_DTYPE.itemsize == 12
