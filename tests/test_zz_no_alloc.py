"""mrc_signature_noalloc: signatures without device allocation, checked against mrc_signature.

The entry point serves callers that cannot allocate device memory on their
request path (a process whose memory manager already holds the GPU's free
memory, or code that must not call cudaMalloc/cudaFree because they
synchronise the device and can fail under memory pressure). It takes its
scratch from a fixed device array inside the library. This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

from paper_1810_03099_gb300 import synth
from tests.gpu_common import concat, csr, cuda_or_skip, edge_docs

pytestmark = pytest.mark.gpu

SIG_TOL = 2e-6  # the tolerance of the signature parity tests


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_mrc_signature_on_two_calls():
    torch = cuda_or_skip()
    from paper_1810_03099_gb300 import mrc

    V = 5000
    base = synth.make_corpus(synth.SPECS["tiny"].with_(n_docs=800, vocab=V))
    with mrc.Context() as ctx:
        idx = mrc.mrc_build_index(ctx, _dev(torch, base.offsets), _dev(torch, base.tokens), V,
                                  mrc.params_default(k=24, select_mode=mrc.SELECT_ALL))
        # two different batches in a row: short and long documents, edge cases
        q1 = synth.make_corpus(synth.SPECS["tiny"].with_(n_docs=500, vocab=V, seed=31))
        q2 = synth.make_corpus(synth.SPECS["batch_queries"].with_(n_docs=40, vocab=V))
        batches = [concat((q1.offsets, q1.tokens), csr(edge_docs(V, seed=2))), (q2.offsets, q2.tokens)]
        for call, (offs, toks) in enumerate(batches):
            o, t = _dev(torch, offs), _dev(torch, toks)
            ref_sig, ref_sh = mrc.mrc_signature(ctx, idx, o, t)
            n = offs.shape[0] - 1
            sig = torch.full((n, idx.k), -1.0, dtype=torch.float32, device="cuda")
            sh = torch.zeros(n, dtype=torch.int64, device="cuda")
            free_before = torch.cuda.mem_get_info()[0]
            mrc.mrc_signature_noalloc(ctx, idx, o, t, sig, sh)
            torch.cuda.synchronize()
            # the first call on a device may load the library's device code (which creates the
            # fixed array); from then on a call takes no device memory at all
            if call > 0:
                assert torch.cuda.mem_get_info()[0] >= free_before
            assert float((sig - ref_sig).abs().max()) <= SIG_TOL
            assert torch.equal(sh, ref_sh)
        idx.free()


def test_noalloc_rejects_oversized_and_host_inputs():
    torch = cuda_or_skip()
    from paper_1810_03099_gb300 import mrc

    V = 1000
    base = synth.make_corpus(synth.SPECS["tiny"].with_(n_docs=100, vocab=V))
    with mrc.Context() as ctx:
        idx = mrc.mrc_build_index(ctx, _dev(torch, base.offsets), _dev(torch, base.tokens), V,
                                  mrc.params_default(k=8))
        n = mrc.NOALLOC_MAX_DOCS + 1
        offs = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
        toks = torch.zeros(1, dtype=torch.int32, device="cuda")
        sig = torch.empty((n, 8), dtype=torch.float32, device="cuda")
        with pytest.raises(mrc.MrcError) as e:
            mrc.mrc_signature_noalloc(ctx, idx, offs, toks, sig)
        assert e.value.status == mrc.MRC_ERR_INVALID and "MRC_NOALLOC_MAX_DOCS" in e.value.message
        host_sig = np.empty((base.n_docs, 8), np.float32)
        with pytest.raises(mrc.MrcError) as e:
            mrc.mrc_signature_noalloc(ctx, idx, base.offsets, base.tokens, host_sig)
        assert e.value.status == mrc.MRC_ERR_INVALID
        idx.free()
