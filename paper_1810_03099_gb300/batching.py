"""Batched queries against a resident signature index (the batching form).

Batches of new documents (here 1-512 documents of 20-20,000 tokens) are each
compared with every index document through one graph-captured pipeline launch
(``mrc_batch_*`` in the C ABI; for k <= 64 one persistent kernel per batch). Batch
sizes vary, so pipelines are captured per size bucket (powers of two up to
``max_docs``); a batch runs in its bucket's pipeline, whose compare covers the
bucket's rows. The compare's tile width, streamed-operand ring depth and L2 prefetch
distance of each bucket come from the autotuner.
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


# The autotuner's search space: compare tile width, depth of the compare's streamed-operand
# ring (0 = as deep as shared memory allows) and L2 prefetch distance in index tiles.
TILES = (128, 256)
RINGS = (0, 3, 6)
PREFETCHES = (0, 8, 24)


def autotune(ctx, index, bucket: int, max_tokens: int, sample, reps: int = 5, cache: str | None = TUNE_CACHE,
             tiles=TILES, rings=RINGS, prefetches=PREFETCHES) -> dict:
    """Time every (tile width, ring depth, prefetch distance) on a sample batch (offsets, tokens)
    and return the fastest as {"tile_n", "ring", "prefetch"}. Results are cached by (GPU, index
    size, k, precision, bucket)."""
    import torch
    key = f"{torch.cuda.get_device_name()}|N{index.n_docs}|k{index.k}|p{index.precision}|b{bucket}"
    table = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
    if key in table and "ring" in table[key]:
        return {k: int(table[key][k]) for k in ("tile_n", "ring", "prefetch")}
    offs, toks = sample
    timings = {}
    for tn in tiles:
        b = mrc.Batch(ctx, index, bucket, max_tokens, capacity=1 << 16, tile_n=tn)
        for ring in rings:
            for pf in prefetches:
                b.tune(tn, ring, pf)
                b.launch(offs, toks)
                b.wait()
                t0 = time.perf_counter()
                for _ in range(reps):
                    b.launch(offs, toks)
                    b.wait()
                timings[(tn, ring, pf)] = (time.perf_counter() - t0) / reps
        b.free()
    best = min(timings, key=timings.get)
    table[key] = {"tile_n": best[0], "ring": best[1], "prefetch": best[2],
                  "seconds": {f"{t}/{r}/{p}": v for (t, r, p), v in timings.items()}}
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tmp = f"{cache}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return {"tile_n": best[0], "ring": best[1], "prefetch": best[2]}


class BatchRunner:
    """Runs batches of new documents against `index`, one graph launch per batch."""

    def __init__(self, ctx, index, tau: float = 0.9, max_docs: int = 512, max_doc_tokens: int = 20000,
                 capacity: int = 1 << 18, autotune: bool = True):
        self.ctx, self.index, self.tau = ctx, index, tau
        self.max_docs, self.max_doc_tokens, self.capacity = max_docs, max_doc_tokens, capacity
        self.autotune = autotune
        self.pipes: dict[int, mrc.Batch] = {}
        self.tuning: dict[int, dict] = {}

    def pipe(self, bucket: int, sample=None) -> mrc.Batch:
        if bucket not in self.pipes:
            max_tokens = bucket * self.max_doc_tokens
            knobs = {"tile_n": 0, "ring": 0, "prefetch": -1}
            if self.autotune and sample is not None:
                knobs = autotune(self.ctx, self.index, bucket, max_tokens, sample)
            self.tuning[bucket] = knobs
            b = mrc.Batch(self.ctx, self.index, bucket, max_tokens, self.tau, self.capacity, knobs["tile_n"])
            if knobs["ring"] != 0 or knobs["prefetch"] != -1:
                b.tune(knobs["tile_n"], knobs["ring"], knobs["prefetch"])
            self.pipes[bucket] = b
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
