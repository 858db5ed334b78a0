"""Bounded device waits (failure detection): a compare kernel whose waits cannot be met stops
after the context's wait limit, the call reports MRC_ERR_TIMEOUT, and the same context then
runs normal calls with the right results.

The waits are made to run out on purpose without faulting or hanging the GPU: with the
context's test stall on, the tensor-core compare kernels issue no MMA, so their TMA producer and
epilogue warps wait for results that never come. Each kernel then lets its own copies land,
frees its tensor memory and returns.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

from paper_1810_03099_gb300 import synth
from tests.gpu_common import cuda_or_skip

pytestmark = pytest.mark.gpu

LIMIT_NS = 50_000_000  # 50 ms


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _triples(M, buf):
    p = M.pairs_to_numpy(buf)
    return sorted(zip(p["i"].tolist(), p["j"].tolist(), p["score"].tolist()))


def _expect_timeout(M, fn):
    t0 = time.perf_counter()
    with pytest.raises(M.MrcError) as ei:
        fn()
    assert ei.value.status == M.MRC_ERR_TIMEOUT, ei.value
    return time.perf_counter() - t0


@pytest.mark.parametrize("precision", [0, 1])
def test_expired_waits_report_timeout_and_context_recovers(precision):
    torch = cuda_or_skip()
    from paper_1810_03099_gb300 import mrc as M

    c = synth.make_corpus("tiny", n_docs=1500)
    offs, toks = _dev(torch, c.offsets), _dev(torch, c.tokens)
    with M.Context() as ref_ctx:
        ref_idx = M.mrc_build_index(ref_ctx, offs, toks, c.vocab, M.params_default(k=64, precision=precision))
        ref_sig = _triples(M, M.mrc_match(ref_ctx, ref_idx, None, 0.7)[0])
        ref_cos = _triples(M, M.cosine_allpairs(ref_ctx, ref_idx, offs, toks, 0.5)[0])
        ref_idx.free()
    with M.Context() as ctx:
        idx = M.mrc_build_index(ctx, offs, toks, c.vocab, M.params_default(k=64, precision=precision))
        ctx.set_wait_limit(LIMIT_NS)
        ctx.set_test_stall(True)
        # one-K-block resident compare (signature match) and the streaming head GEMM (exact cosine)
        dt = _expect_timeout(M, lambda: M.mrc_match(ctx, idx, None, 0.7, grow=False))
        assert dt < 30.0
        _expect_timeout(M, lambda: M.cosine_allpairs(ctx, idx, offs, toks, 0.5, grow=False))
        # stream-ordered form: the timeout is reported by mrc_ctx_sync
        pairs = torch.empty((1 << 16, 3), dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int64, device="cuda")
        M.mrc_match_async(ctx, idx, pairs, count, None, 0.7)
        _expect_timeout(M, ctx.sync)
        # the context is still usable: normal calls give the results of a fresh context
        ctx.set_test_stall(False)
        ctx.set_wait_limit(4_000_000_000)
        assert _triples(M, M.mrc_match(ctx, idx, None, 0.7)[0]) == ref_sig
        assert _triples(M, M.cosine_allpairs(ctx, idx, offs, toks, 0.5)[0]) == ref_cos
        idx.free()
    torch.cuda.synchronize()


def test_wait_limit_rejects_out_of_range_values():
    cuda_or_skip()
    from paper_1810_03099_gb300 import mrc as M

    with M.Context() as ctx:
        for bad in (0, -5, 600_000_000_001):
            with pytest.raises(M.MrcError) as ei:
                ctx.set_wait_limit(bad)
            assert ei.value.status == M.MRC_ERR_INVALID
        ctx.set_wait_limit(1)
        ctx.set_wait_limit(600_000_000_000)
