"""Continuous-batching server over a device-resident signature index (the serving form).

New documents arrive one by one (Poisson arrivals in the benchmark). A single
host loop
  * admits arrived requests into a queue;
  * dispatches a micro-batch (up to ``micro_batch`` documents, or whatever has
    waited ``deadline_s``) to any free pipeline slot: each slot is a
    graph-captured ``mrc_batch`` with its own stream, so batches launched while
    others are still on the GPU overlap on the device;
  * completes slots as their GPU work finishes (non-blocking polls) and stamps
    every request's latency (completion minus arrival). A finished batch's pairs go by
    one DMA straight into a ring of pinned host memory, and each request's pairs are a view
    of its slice; before a ring region is reused, the requests still viewing it get copies.
With a block-table fingerprint index of the resident documents' Simhashes, every slot also
matches its requests' Simhashes against it (Hamming pairs per request, beside the
signature pairs).
The number of slots is admitted against free HBM at start-up: a slot is only
created while its device footprint fits in ``hbm_fraction`` of the free memory.
Each document's result does not depend on the other documents of its batch
(per-document signature pass, per-pair compare and rescoring), so a request's
pairs are the same alone and in the mix.
"""
from __future__ import annotations

import collections
import time
import weakref
from dataclasses import dataclass, field

import numpy as np

from . import mrc


@dataclass
class Request:
    rid: int
    tokens: np.ndarray
    arrival: float
    done: float = -1.0
    pairs: np.ndarray = field(default_factory=lambda: np.empty(0, mrc.PAIR_DTYPE))  # (i, j, score) rows
    hamming: np.ndarray = field(default_factory=lambda: np.empty(0, mrc.PAIR_DTYPE))  # (i, j, distance) rows


def slot_footprint(index, max_docs: int, max_tokens: int, capacity: int) -> int:
    """Device bytes of one pipeline slot (inputs, operands, candidates, pairs, workspace)."""
    k = index.k
    op = max_docs * (64 if k <= 64 else k) * 2
    cand = max(4 * capacity, 1 << 16) * 12
    ws = max_docs * 8 * 4 + 64 * 1024
    grouped = 12 * capacity + 16 * max_docs + 8
    return 8 * (max_docs + 1) + 4 * max_tokens + 4 * max_docs * k + op + 4 * max_docs + cand + 12 * capacity + ws + grouped


class _Ring:
    """Pinned host arena for batch results, handed out in order and wrapping around. A region
    about to be overwritten first gives the requests still viewing it (held elsewhere) their
    own copies."""

    def __init__(self, n_pairs: int, attr: str):
        self.buf = mrc._pinned_pairs(n_pairs)
        self.n, self.head, self.attr = self.buf.shape[0], 0, attr
        self.live: collections.deque = collections.deque()  # (start, end, requests)
        self.evicted = 0  # requests given their own copies

    def take(self, m: int):
        """A view of m free slots (None if m exceeds the arena)."""
        if m > self.n:
            return None
        start = self.head if self.head + m <= self.n else 0
        end = start + m
        keep = collections.deque()
        for a, b, refs in self.live:  # every region the new one overlaps (the tail left at a wrap too)
            if a < end and start < b:
                for w in refs:
                    r = w()
                    if r is not None:  # still held by the caller
                        setattr(r, self.attr, getattr(r, self.attr).copy())
                        self.evicted += 1
            else:
                keep.append((a, b, refs))
        self.live = keep
        self.head = end
        return start

    def keep(self, start: int, m: int, reqs):
        if m:
            self.live.append((start, start + m, [weakref.ref(r) for r in reqs]))


class Server:
    def __init__(self, ctx, index, tau: float = 0.9, micro_batch: int = 128, deadline_s: float = 1e-3,
                 slots: int = 4, max_doc_tokens: int = 10000, capacity: int = 1 << 16, hbm_fraction: float = 0.5,
                 tile_n: int = 0, free_bytes: int | None = None, simhash_index=None, hamming_max: int | None = None,
                 hamming_capacity: int = 1 << 16, result_pairs: int = 1 << 24):
        import torch
        self.ctx, self.index, self.tau = ctx, index, tau
        self.micro_batch, self.deadline_s = micro_batch, deadline_s
        self.max_tokens = micro_batch * max_doc_tokens
        self.capacity = capacity
        free = torch.cuda.mem_get_info()[0] if free_bytes is None else free_bytes
        foot = slot_footprint(index, micro_batch, self.max_tokens, capacity)
        self.admitted_slots = int(max(0, min(slots, (hbm_fraction * free) // foot)))
        if self.admitted_slots < 1:
            raise MemoryError("not enough free device memory for one pipeline slot")
        self.slots = [mrc.Batch(ctx, index, micro_batch, self.max_tokens, tau, capacity, tile_n)
                      for _ in range(self.admitted_slots)]
        self.hamming = simhash_index is not None
        if self.hamming:  # each slot also matches its requests' Simhashes against the resident ones
            for b in self.slots:
                b.attach_simhash(simhash_index, hamming_max, hamming_capacity)
        self.busy: list[list[Request] | None] = [None] * len(self.slots)
        # pinned rings for the results (result_pairs pairs; the Hamming ring a quarter of that)
        self.ring = _Ring(result_pairs, "pairs")
        self.hring = _Ring(max(result_pairs // 4, 1), "hamming") if self.hamming else None
        # pinned staging per slot (stream-ordered copies read them until the batch finishes)
        self.h_off = [torch.empty(micro_batch + 1, dtype=torch.int64).pin_memory() for _ in self.slots]
        self.h_tok = [torch.empty(self.max_tokens, dtype=torch.int32).pin_memory() for _ in self.slots]

    def _launch(self, s: int, reqs: list[Request]):
        lens = np.array([r.tokens.shape[0] for r in reqs], np.int64)
        off = self.h_off[s].numpy()[:len(reqs) + 1]
        off[0] = 0
        np.cumsum(lens, out=off[1:])
        tok = self.h_tok[s].numpy()
        if off[-1]:
            tok[:off[-1]] = np.concatenate([r.tokens for r in reqs])
        self.slots[s].launch(self.h_off[s][:len(reqs) + 1], self.h_tok[s][:int(off[-1])])
        self.busy[s] = reqs

    def _fetch(self, ring, total, copy):
        """One result kind of a finished batch into its ring: (pairs view, query offsets)."""
        start = ring.take(total)
        if start is None:  # larger than the whole arena: a copy of its own
            pairs, _, qoff = copy(None, True)
            return pairs, qoff, None
        pairs, _, qoff = copy(ring.buf[start:start + total], True)
        return pairs, qoff, start

    def _complete(self, s: int, now: float):
        # the pipeline returns the batch's pairs grouped by request, with each request's start
        b, reqs = self.slots[s], self.busy[s]
        tot, htot = b.totals()
        pairs, qoff, at = self._fetch(self.ring, min(tot, self.capacity), lambda o, f: b.wait(out=o, offsets=f))
        if self.hamming:
            hp, hoff, hat = self._fetch(self.hring, min(htot, b.h_capacity), lambda o, f: b.hamming(out=o, offsets=f))
        for q, r in enumerate(reqs):
            r.done = now
            r.pairs = pairs[qoff[q]:qoff[q + 1]]
            if self.hamming:
                r.hamming = hp[hoff[q]:hoff[q + 1]]
        if at is not None:
            self.ring.keep(at, len(pairs), reqs)
        if self.hamming and hat is not None:
            self.hring.keep(hat, len(hp), reqs)
        self.busy[s] = None

    def run(self, docs: list[np.ndarray], arrivals: np.ndarray) -> list[Request]:
        """Serve documents arriving at the given times (seconds from start); returns the requests."""
        reqs = [Request(i, d, float(a)) for i, (d, a) in enumerate(zip(docs, arrivals))]
        queue: list[Request] = []
        nxt = 0
        finished = 0
        t0 = time.perf_counter()
        while finished < len(reqs):
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                queue.append(reqs[nxt])
                nxt += 1
            for s in range(len(self.slots)):
                if self.busy[s] is not None and self.slots[s].poll():
                    n = len(self.busy[s])
                    self._complete(s, time.perf_counter() - t0)
                    finished += n
            if queue:
                due = len(queue) >= self.micro_batch or (now - queue[0].arrival) >= self.deadline_s or nxt == len(reqs)
                if due:
                    for s in range(len(self.slots)):
                        if self.busy[s] is None and queue:
                            take, queue = queue[:self.micro_batch], queue[self.micro_batch:]
                            self._launch(s, take)
        self.wall_s = time.perf_counter() - t0
        return reqs

    def free(self):
        for b in self.slots:
            b.free()


def latency_report(reqs: list[Request], wall_s: float) -> dict:
    lat = np.array([r.done - r.arrival for r in reqs])
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "max_ms": float(lat.max() * 1e3),
            "docs_per_s": len(reqs) / wall_s}
