"""Batched queries against a resident signature index (the batching form).

Batches of new documents (here 1-512 documents of 20-20,000 tokens) are each
compared with every index document through one graph-captured pipeline launch
(``mrc_batch_*`` in the C ABI). Batch sizes vary, so pipelines are captured per
size bucket (powers of two up to ``max_docs``) and a batch is padded to its
bucket. The compare tile width of each bucket comes from the autotuner.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

from . import mrc

HERE = os.path.dirname(os.path.abspath(__file__))
TUNE_CACHE = os.path.join(HERE, "_build", "autotune.json")


def bucket_of(n: int, max_docs: int) -> int:
    b = 1
    while b < n:
        b <<= 1
    return min(b, max_docs)


def autotune_tile(ctx, index, bucket: int, max_tokens: int, sample, reps: int = 5, cache: str | None = TUNE_CACHE,
                  candidates=(128, 256)) -> int:
    """Time each compare tile width on a sample batch (offsets, tokens) and return the fastest.
    Results are cached by (GPU, index size, k, precision, bucket)."""
    import torch
    key = f"{torch.cuda.get_device_name()}|N{index.n_docs}|k{index.k}|p{index.precision}|b{bucket}"
    table = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if key in table:
        return int(table[key]["tile_n"])
    offs, toks = sample
    timings = {}
    for tn in candidates:
        b = mrc.Batch(ctx, index, bucket, max_tokens, capacity=1 << 16, tile_n=tn)
        b.launch(offs, toks)
        b.wait()
        t0 = time.perf_counter()
        for _ in range(reps):
            b.launch(offs, toks)
            b.wait()
        timings[tn] = (time.perf_counter() - t0) / reps
        b.free()
    best = min(timings, key=timings.get)
    table[key] = {"tile_n": best, "seconds": {str(k): v for k, v in timings.items()}}
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = f"{cache}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return best


class BatchRunner:
    """Runs batches of new documents against `index`, one graph launch per batch."""

    def __init__(self, ctx, index, tau: float = 0.9, max_docs: int = 512, max_doc_tokens: int = 20000,
                 capacity: int = 1 << 18, autotune: bool = True):
        self.ctx, self.index, self.tau = ctx, index, tau
        self.max_docs, self.max_doc_tokens, self.capacity = max_docs, max_doc_tokens, capacity
        self.autotune = autotune
        self.pipes: dict[int, mrc.Batch] = {}
        self.tiles: dict[int, int] = {}

    def pipe(self, bucket: int, sample=None) -> mrc.Batch:
        if bucket not in self.pipes:
            max_tokens = bucket * self.max_doc_tokens
            tn = 0
            if self.autotune and sample is not None:
                tn = autotune_tile(self.ctx, self.index, bucket, max_tokens, sample)
            self.tiles[bucket] = tn
            self.pipes[bucket] = mrc.Batch(self.ctx, self.index, bucket, max_tokens, self.tau, self.capacity, tn)
        return self.pipes[bucket]

    def prepare(self, batches):
        """Capture (and tune) the pipeline of every bucket the batches need."""
        for offs, toks in batches:
            n = offs.shape[0] - 1
            self.pipe(bucket_of(n, self.max_docs), (offs, toks))

    def run(self, offsets, tokens):
        """One batch: returns (pairs, total)."""
        n = offsets.shape[0] - 1
        if n > self.max_docs:
            raise ValueError("batch larger than max_docs")
        p = self.pipe(bucket_of(n, self.max_docs), (offsets, tokens))
        p.launch(offsets, tokens)
        return p.wait()

    def free(self):
        for p in self.pipes.values():
            p.free()
        self.pipes.clear()


def make_batches(pool_offsets, pool_tokens, sizes, seed: int):
    """Batches drawn (with replacement, seeded) from a pool of query documents; each batch is
    a contiguous token CSR in pinned-ready numpy arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_pool = pool_offsets.shape[0] - 1
    lens = np.diff(pool_offsets)
    out = []
    for sz in sizes:
        pick = rng.integers(0, n_pool, size=int(sz))
        offs = np.zeros(int(sz) + 1, np.int64)
        np.cumsum(lens[pick], out=offs[1:])
        toks = np.concatenate([pool_tokens[pool_offsets[i]:pool_offsets[i + 1]] for i in pick]).astype(np.int32)
        out.append((offs, toks, pick))
    return out
