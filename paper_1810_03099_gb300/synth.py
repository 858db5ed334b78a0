"""Seeded synthetic corpora shaped like the paper's workloads.

This module produces inputs only. It holds none of the method's arithmetic (no
weighting, no signatures, no hashing of terms): it draws token-id documents and
hands the same arrays to the CUDA path and to the CPU oracle.

A token id stands for one character 3-gram of the paper's vector space model
(Section III). The paper evaluates on NEWS20 (~18.8k Usenet posts, 20 groups,
Section V); that corpus is not available here, so topic-mixture corpora with
Zipf term laws stand in for it:

* each of ``n_topics`` topics is a truncated Zipf(s) law over its own seeded
  permutation of the vocabulary;
* each document draws a topic mixture from Dirichlet(alpha) and a length from a
  lognormal (or log-uniform) law, then draws its tokens from the mixture;
* a fraction of documents are near-duplicates: copies of a random earlier
  document with a uniform 1-10 % of token positions replaced by fresh draws
  from the source document's mixture.

Output layout is a token CSR: ``offsets:int64[N+1]``, ``tokens:int32[T]``.
"""
from __future__ import annotations

import dataclasses
import os
from dataclasses import dataclass

import numpy as np

BASE_SEED = 1810030990


@dataclass(frozen=True)
class CorpusSpec:
    name: str
    n_docs: int
    vocab: int
    zipf_s: float
    n_topics: int
    alpha: float
    length_law: str  # "lognormal" | "loguniform"
    length_median: float  # lognormal median
    length_sigma: float  # lognormal sigma
    length_min: int
    length_max: int
    dup_frac: float
    edit_lo: float
    edit_hi: float
    seed: int

    def with_(self, **kw) -> "CorpusSpec":
        return dataclasses.replace(self, **kw)


# Workload shapes. Sizes follow the five workloads the method is measured on:
# the tiny plain case, the NEWS20-shaped corpus, the one-million-document
# precision corpus, batched queries of 20-20,000 tokens, and serving arrivals.
SPECS = {
    "tiny": CorpusSpec("tiny", 2000, 5000, 1.1, 10, 0.1, "lognormal", 120.0, 1.0, 5, 10000,
                       0.05, 0.01, 0.10, BASE_SEED + 0),
    "news20": CorpusSpec("news20", 18846, 60000, 1.1, 20, 0.1, "lognormal", 150.0, 1.0, 5, 10000,
                         0.05, 0.01, 0.10, BASE_SEED + 1),
    "precision": CorpusSpec("precision", 1_000_000, 1 << 18, 1.05, 20, 0.1, "lognormal", 300.0, 1.0,
                            5, 10000, 0.05, 0.01, 0.10, BASE_SEED + 2),
    "batch_queries": CorpusSpec("batch_queries", 512, 1 << 18, 1.05, 20, 0.1, "loguniform", 0.0, 0.0,
                                20, 20000, 0.0, 0.0, 0.0, BASE_SEED + 3),
    "serving": CorpusSpec("serving", 10_000_000, 1 << 18, 1.05, 20, 0.1, "lognormal", 300.0, 1.0,
                          5, 10000, 0.05, 0.01, 0.10, BASE_SEED + 4),
}


@dataclass
class Corpus:
    spec: CorpusSpec
    offsets: np.ndarray  # int64[N+1]
    tokens: np.ndarray  # int32[T]
    dup_src: np.ndarray  # int64[N]; -1 or the index of the copied document
    edits: np.ndarray  # int32[N]; substituted token positions of a near-duplicate

    @property
    def n_docs(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def vocab(self) -> int:
        return int(self.spec.vocab)

    @property
    def n_tokens(self) -> int:
        return int(self.tokens.shape[0])

    def doc(self, i: int) -> np.ndarray:
        return self.tokens[self.offsets[i]:self.offsets[i + 1]]

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets)

    def subset(self, idx) -> "Corpus":
        """Documents ``idx`` (in that order) as a new corpus; dup links are dropped."""
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths()[idx]
        offs = np.zeros(idx.shape[0] + 1, dtype=np.int64)
        np.cumsum(lens, out=offs[1:])
        toks = np.empty(int(offs[-1]), dtype=np.int32)
        for n, i in enumerate(idx):
            toks[offs[n]:offs[n + 1]] = self.doc(int(i))
        return Corpus(self.spec, offs, toks, np.full(idx.shape[0], -1, np.int64),
                      np.zeros(idx.shape[0], np.int32))


class _Alias:
    """Vose alias table: O(1) draws from a fixed discrete law."""

    def __init__(self, p: np.ndarray):
        n = p.shape[0]
        q = p * (n / p.sum())
        prob = np.zeros(n, dtype=np.float64)
        alias = np.zeros(n, dtype=np.int64)
        small = list(np.nonzero(q < 1.0)[0][::-1])
        large = list(np.nonzero(q >= 1.0)[0][::-1])
        q = q.tolist()
        while small and large:
            s = small.pop()
            g = large.pop()
            prob[s] = q[s]
            alias[s] = g
            q[g] = (q[g] + q[s]) - 1.0
            (small if q[g] < 1.0 else large).append(g)
        for g in large:
            prob[g] = 1.0
        for s in small:
            prob[s] = 1.0
        self.prob = prob
        self.prob32 = prob.astype(np.float32)
        self.alias = alias
        self.n = n

    def draw(self, rng: np.random.Generator, size: int) -> np.ndarray:
        i = rng.integers(0, self.n, size=size, dtype=np.int64)
        u = rng.random(size, dtype=np.float32)
        return np.where(u < self.prob32[i], i, self.alias[i])


def _lengths(spec: CorpusSpec, rng: np.random.Generator, n: int) -> np.ndarray:
    if spec.length_law == "lognormal":
        x = rng.lognormal(mean=np.log(spec.length_median), sigma=spec.length_sigma, size=n)
    elif spec.length_law == "loguniform":
        x = np.exp(rng.uniform(np.log(spec.length_min), np.log(spec.length_max), size=n))
    else:
        raise ValueError(spec.length_law)
    return np.clip(np.rint(x), spec.length_min, spec.length_max).astype(np.int64)


def _draw_terms(rng, zipf: _Alias, perms: np.ndarray, topics: np.ndarray) -> np.ndarray:
    ranks = zipf.draw(rng, topics.shape[0])
    return perms.reshape(-1)[topics.astype(np.int64) * perms.shape[1] + ranks]


def make_corpus(spec: CorpusSpec | str, n_docs: int | None = None, seed: int | None = None) -> Corpus:
    """Draw a corpus. ``n_docs``/``seed`` override the spec (smaller parity cases)."""
    if isinstance(spec, str):
        spec = SPECS[spec]
    if n_docs is not None:
        spec = spec.with_(n_docs=int(n_docs))
    if seed is not None:
        spec = spec.with_(seed=int(seed))
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    N, V, K = spec.n_docs, spec.vocab, spec.n_topics

    ranks = np.arange(1, V + 1, dtype=np.float64)
    zipf = _Alias(ranks ** (-spec.zipf_s))
    perms = np.stack([rng.permutation(V) for _ in range(K)]).astype(np.int32)
    theta = rng.dirichlet(np.full(K, spec.alpha), size=N)
    lens = _lengths(spec, rng, N)

    # near-duplicate plan: dup i copies an earlier document src[i]
    n_dup = int(round(spec.dup_frac * N)) if N > 1 else 0
    dup_src = np.full(N, -1, dtype=np.int64)
    if n_dup:
        dups = np.sort(rng.choice(np.arange(1, N), size=n_dup, replace=False))
        src = (rng.random(n_dup) * dups).astype(np.int64)  # uniform in [0, i)
        dup_src[dups] = src
        for i, j in zip(dups.tolist(), src.tolist()):
            lens[i] = lens[j]
            theta[i] = theta[j]

    offsets = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    T = int(offsets[-1])
    tokens = np.empty(T, dtype=np.int32)

    # base documents, in chunks of about 2^24 tokens: every token draws its topic from its
    # document's mixture (inverse CDF over the mixture) and then its term from that topic
    chunk = 1 << 24
    cum = np.cumsum(theta, axis=1).astype(np.float32)
    cum[:, -1] = 2.0  # every draw falls at or below the last topic
    d0 = 0
    while d0 < N:
        d1 = int(np.searchsorted(offsets, offsets[d0] + chunk, side="right")) - 1
        d1 = min(max(d1, d0 + 1), N)
        ln = lens[d0:d1]
        u = rng.random(int(offsets[d1] - offsets[d0]), dtype=np.float32)
        topics = np.zeros(u.shape[0], dtype=np.int32)
        for z in range(K - 1):
            topics += u > np.repeat(cum[d0:d1, z], ln)
        tokens[offsets[d0]:offsets[d1]] = _draw_terms(rng, zipf, perms, topics)
        d0 = d1

    edits = np.zeros(N, dtype=np.int32)
    if n_dup:
        for i in np.nonzero(dup_src >= 0)[0].tolist():
            j = int(dup_src[i])
            src_tok = tokens[offsets[j]:offsets[j + 1]]
            n = src_tok.shape[0]
            f = rng.uniform(spec.edit_lo, spec.edit_hi) if spec.edit_hi > 0 else 0.0
            n_edit = int(round(f * n))
            if spec.edit_hi > 0:
                n_edit = max(1, min(n, n_edit))
            new = src_tok.copy()
            if n_edit:
                pos = rng.choice(n, size=n_edit, replace=False)
                tz = rng.choice(K, size=n_edit, p=theta[j])
                new[pos] = _draw_terms(rng, zipf, perms, tz.astype(np.int64))
            tokens[offsets[i]:offsets[i + 1]] = new
            edits[i] = n_edit
    return Corpus(spec, offsets, tokens, dup_src, edits)


# ---------------------------------------------------------------------------------------------
# Raw text (input of the character 3-gram front end)

# Approximate relative letter frequencies of English text (a..z), so that the drawn words give
# a skewed 3-gram law: a few 3-grams common, most rare, as in the paper's corpus statistics.
_LETTER_FREQ = np.array([8.2, 1.5, 2.8, 4.3, 12.7, 2.2, 2.0, 6.1, 7.0, 0.15, 0.8, 4.0, 2.4, 6.7, 7.5, 1.9,
                         0.1, 6.0, 6.3, 9.1, 2.8, 1.0, 2.4, 0.15, 2.0, 0.07])
# Single-byte separators between words and their probabilities: space, newline, comma, full
# stop, apostrophe, hyphen, a digit, tab.
_SEPARATORS = np.frombuffer(b" \n,.'-7\t", np.uint8)
_SEP_P = np.array([0.80, 0.05, 0.04, 0.04, 0.02, 0.02, 0.02, 0.01])


@dataclass
class TextCorpus:
    words: Corpus  # the word-id documents the text renders (dup links included)
    offsets: np.ndarray  # int64[N+1] byte offsets
    text: np.ndarray  # uint8[B]

    @property
    def n_docs(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_bytes(self) -> int:
        return int(self.text.shape[0])

    def doc(self, i: int) -> bytes:
        return self.text[self.offsets[i]:self.offsets[i + 1]].tobytes()


def _lexicon(n_words: int, rng: np.random.Generator):
    """Seeded word list: lengths 1 + Poisson(4) (at most 15 letters), letters drawn by English
    letter frequency; 1 % of the words carry a two-byte UTF-8 letter (0xC3 0xA9) inside."""
    lens = np.minimum(1 + rng.poisson(4.0, size=n_words), 15).astype(np.int64)
    accent = rng.random(n_words) < 0.01
    lens_b = lens + 2 * (accent & (lens >= 2))
    offs = np.zeros(n_words + 1, np.int64)
    np.cumsum(lens_b, out=offs[1:])
    letters = (rng.choice(26, size=int(offs[-1]), p=_LETTER_FREQ / _LETTER_FREQ.sum()) + ord("a")).astype(np.uint8)
    for w in np.nonzero(accent & (lens >= 2))[0].tolist():
        at = int(offs[w]) + 1
        letters[at:at + 2] = (0xC3, 0xA9)
    return offs, letters


def make_text_corpus(spec: CorpusSpec | str = "news20", n_docs: int | None = None, seed: int | None = None,
                     words_median: float = 300.0) -> TextCorpus:
    """Raw text shaped like NEWS20 posts: documents of words drawn as ``make_corpus`` draws
    terms (topic mixtures over Zipf laws, lognormal lengths with median ``words_median`` words,
    near-duplicates with 1-10 % of the words replaced), each word rendered from a seeded
    lexicon, 10 % capitalised, followed by one separator byte."""
    if isinstance(spec, str):
        spec = SPECS[spec]
    spec = spec.with_(length_median=float(words_median))
    c = make_corpus(spec, n_docs=n_docs, seed=seed)
    rng = np.random.Generator(np.random.PCG64(c.spec.seed + 7919))
    lex_offs, lex = _lexicon(c.vocab, rng)
    w = c.tokens.astype(np.int64)
    wl = lex_offs[w + 1] - lex_offs[w]
    out_len = wl + 1
    starts = np.zeros(w.shape[0] + 1, np.int64)
    np.cumsum(out_len, out=starts[1:])
    B = int(starts[-1])
    text = np.empty(B, np.uint8)
    # every output byte: the word occurrence it belongs to and its position inside the word
    occ = np.repeat(np.arange(w.shape[0], dtype=np.int64), out_len)
    pos = np.arange(B, dtype=np.int64) - starts[occ]
    is_sep = pos == wl[occ]
    body = ~is_sep
    text[body] = lex[lex_offs[w[occ[body]]] + pos[body]]
    text[is_sep] = _SEPARATORS[rng.choice(_SEPARATORS.shape[0], size=w.shape[0], p=_SEP_P)]
    cap = np.nonzero(rng.random(w.shape[0]) < 0.10)[0]
    first = starts[cap]
    text[first] = np.where((text[first] >= ord("a")) & (text[first] <= ord("z")), text[first] - 32, text[first])
    offsets = starts[c.offsets]
    return TextCorpus(c, offsets, text)


def cached_corpus(name: str, cache_dir: str | None = None, **kw) -> Corpus:
    """``make_corpus`` with an on-disk .npz cache (large workloads take a while to draw)."""
    spec = SPECS[name]
    if kw:
        spec = spec.with_(**kw)
    cache_dir = cache_dir or os.environ.get("MRC_CORPUS_CACHE",
                                            os.path.join(os.path.dirname(__file__), "..", "_build", "corpora"))
    key = (f"{spec.name}_{spec.n_docs}_{spec.seed}_{spec.vocab}_{spec.length_law}_{spec.length_median}_"
           f"{spec.length_sigma}_{spec.dup_frac}.npz")
    path = os.path.join(cache_dir, key)
    if os.path.exists(path):
        z = np.load(path)
        return Corpus(spec, z["offsets"], z["tokens"], z["dup_src"], z["edits"])
    c = make_corpus(spec)
    os.makedirs(cache_dir, exist_ok=True)
    tmp = path + f".tmp{os.getpid()}.npz"
    np.savez(tmp, offsets=c.offsets, tokens=c.tokens, dup_src=c.dup_src, edits=c.edits)
    os.replace(tmp, path)
    return c


def query_batch_sizes(n_batches: int = 4096, lo: int = 1, hi: int = 512, seed: int = BASE_SEED + 5) -> np.ndarray:
    """Batch sizes of the batched-query workload: uniform integers in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(lo, hi + 1, size=n_batches)


def poisson_arrivals(rate_per_s: float, n: int, seed: int = BASE_SEED + 6) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process with the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))


def random_signatures(n: int, k: int, seed: int, density: float = 0.5) -> np.ndarray:
    """Non-negative float32 [n, k] test vectors with exact zeros (signature-shaped inputs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.random((n, k)).astype(np.float32)
    x[rng.random((n, k)) > density] = 0.0
    return x


def random_fingerprints(n: int, seed: int, n_near: int = 0, max_flip: int = 4) -> np.ndarray:
    """uint64[n] random 64-bit words; the last ``n_near`` are copies of earlier words
    with 0..max_flip random bits flipped (so Hamming matches exist)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.integers(0, np.iinfo(np.uint64).max, size=n, dtype=np.uint64, endpoint=True)
    for t in range(n - n_near, n):
        if t <= 0:
            continue
        src = int(rng.integers(0, t))
        v = int(x[src])
        for b in rng.choice(64, size=int(rng.integers(0, max_flip + 1)), replace=False).tolist():
            v ^= 1 << b
        x[t] = np.uint64(v)
    return x


@dataclass
class DeviceCorpus:
    """A corpus whose token CSR lives on a CUDA device (torch tensors)."""
    spec: CorpusSpec
    offsets: "object"  # torch.int64 [N+1] on the device
    tokens: "object"  # torch.int32 [T] on the device
    dup_src: np.ndarray  # [N]: -1 or the original the near-duplicate was copied from

    @property
    def n_docs(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def vocab(self) -> int:
        return int(self.spec.vocab)

    @property
    def n_tokens(self) -> int:
        return int(self.tokens.shape[0])

    def host_subset(self, idx) -> Corpus:
        """Documents ``idx`` copied to the host as a ``Corpus`` (for CPU checks)."""
        import torch
        idx = np.asarray(idx, dtype=np.int64)
        offs_h = self.offsets.cpu().numpy()
        lens = offs_h[idx + 1] - offs_h[idx]
        new = np.zeros(idx.shape[0] + 1, np.int64)
        np.cumsum(lens, out=new[1:])
        pos = torch.from_numpy(np.repeat(offs_h[idx] - new[:-1], lens) + np.arange(int(new[-1]))).to(self.tokens.device)
        toks = self.tokens[pos].cpu().numpy()
        return Corpus(self.spec, new, toks, np.full(idx.shape[0], -1, np.int64), np.zeros(idx.shape[0], np.int32))


def make_corpus_device(spec: CorpusSpec | str, device="cuda", n_docs: int | None = None,
                       seed: int | None = None) -> DeviceCorpus:
    """Draw a large corpus directly into device memory.

    Same recipe as ``make_corpus`` (topic mixtures, Zipf topics, lengths, near-duplicates),
    with a different random stream: mixtures, lengths and the duplicate plan come from
    the seeded NumPy generator; per-token topic and term draws and the duplicates' edits
    from a seeded torch generator on the device. A near-duplicate copies its original's
    root (the first document of a copy chain) before its own edits.
    """
    import torch
    if isinstance(spec, str):
        spec = SPECS[spec]
    if n_docs is not None:
        spec = spec.with_(n_docs=int(n_docs))
    if seed is not None:
        spec = spec.with_(seed=int(seed))
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    N, V, K = spec.n_docs, spec.vocab, spec.n_topics
    dev = torch.device(device)
    ranks = np.arange(1, V + 1, dtype=np.float64)
    zipf = _Alias(ranks ** (-spec.zipf_s))
    perms = np.stack([rng.permutation(V) for _ in range(K)]).astype(np.int32)
    theta = rng.dirichlet(np.full(K, spec.alpha), size=N).astype(np.float32)
    lens = _lengths(spec, rng, N)
    n_dup = int(round(spec.dup_frac * N)) if N > 1 else 0
    dup_src = np.full(N, -1, dtype=np.int64)
    edit_f = np.zeros(N, np.float32)
    if n_dup:
        dups = np.sort(rng.choice(np.arange(1, N), size=n_dup, replace=False))
        dup_src[dups] = (rng.random(n_dup) * dups).astype(np.int64)
        root = dup_src.copy()
        while True:  # follow copy chains to their first document
            nxt = np.where(root >= 0, dup_src[np.maximum(root, 0)], -1)
            upd = (root >= 0) & (nxt >= 0)
            if not upd.any():
                break
            root[upd] = nxt[upd]
        lens[dups] = lens[root[dups]]
        theta[dups] = theta[root[dups]]
        edit_f[dups] = rng.uniform(spec.edit_lo, spec.edit_hi, size=n_dup)
    offsets = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    T = int(offsets[-1])

    g = torch.Generator(device=dev)
    g.manual_seed(spec.seed)
    d_perm = torch.from_numpy(perms.reshape(-1)).to(dev)
    d_prob = torch.from_numpy(zipf.prob32).to(dev)
    d_alias = torch.from_numpy(zipf.alias).to(dev)
    d_cum = torch.from_numpy(np.cumsum(theta, axis=1)).to(dev)
    d_cum[:, -1] = 2.0
    d_lens = torch.from_numpy(lens).to(dev)
    d_off = torch.from_numpy(offsets).to(dev)
    tokens = torch.empty(T, dtype=torch.int32, device=dev)

    def draw_terms(docs_of_tok):
        u = torch.rand(docs_of_tok.shape[0], generator=g, device=dev)
        topic = torch.zeros(docs_of_tok.shape[0], dtype=torch.int64, device=dev)
        for z in range(K - 1):
            topic += (u > d_cum[docs_of_tok, z]).to(torch.int64)
        i = torch.randint(0, V, (docs_of_tok.shape[0],), generator=g, device=dev)
        a = torch.rand(docs_of_tok.shape[0], generator=g, device=dev)
        r = torch.where(a < d_prob[i], i, d_alias[i])
        return d_perm[topic * V + r].to(torch.int32)

    chunk = 1 << 27
    d0 = 0
    while d0 < N:
        d1 = int(np.searchsorted(offsets, offsets[d0] + chunk, side="right")) - 1
        d1 = min(max(d1, d0 + 1), N)
        docs_of = torch.repeat_interleave(torch.arange(d0, d1, device=dev), d_lens[d0:d1])
        tokens[offsets[d0]:offsets[d1]] = draw_terms(docs_of)
        d0 = d1
    if n_dup:
        dd = torch.from_numpy(dups).to(dev)
        rr = torch.from_numpy(root[dups]).to(dev)
        dl = d_lens[dd]
        within = torch.arange(int(dl.sum().item()), device=dev) - torch.repeat_interleave(
            torch.cumsum(dl, 0) - dl, dl)
        dst = torch.repeat_interleave(d_off[dd], dl) + within
        src = torch.repeat_interleave(d_off[rr], dl) + within
        tokens[dst] = tokens[src]
        f = torch.repeat_interleave(torch.from_numpy(edit_f[dups]).to(dev), dl)
        edit = torch.rand(dst.shape[0], generator=g, device=dev) < f
        pos = dst[edit]
        if pos.numel():
            tokens[pos] = draw_terms(torch.repeat_interleave(dd, dl)[edit])
    return DeviceCorpus(spec, d_off, tokens, dup_src)
