"""Benchmark of the Multi-reference Cosine hot path on one GB300 (replicas on N GPUs).

Headline step (the million-document precision workload: 1,000,000 synthetic documents, 2^18
hashed terms, Zipf(1.05) topic mixtures, lognormal lengths with median 300, 5 % near-duplicates;
k = 64 references, tau = 0.9, Hamming <= 3): one pass of the whole hot path over the corpus,
  index build (term counts, TF-IDF with bfloat16 weights, reference selection, signatures,
  fused Simhash, unit-length E4M3 operands) -> all-pairs signature compare on the tensor cores
  in FP8 E4M3 with FP32 accumulation at tau - 0.02 -> FP32 rescoring of every candidate ->
  block-table Hamming index over the Simhashes -> all Simhash pairs within distance 3.
The same step in the plain FP32 form (fp32 weights, fp16 compare at the proven bound
tau - 2e-3, FP32 rescoring) runs on the same corpus for the forms' ratio.

value = documents/s of the precision-form step with inputs resident in HBM; e2e = the same step
through the C ABI with the corpus in page-locked host memory (the kernels read its tokens in
place) and both pair lists read back into page-locked host memory within the step. The line
also carries: the FP32 form's docs/s and the ratio, signature pairs/s, recall / precision and
per-stage errors of both forms against the FP64 oracle on a seeded 20,000-document subset, the
serving form's p50 / p99 latency at arrival rates from 10k to 500k docs/s against a
10-million-document index, the NEWS20-shaped step with the exact cosine, per-kernel rooflines,
and the oracle's own speed on one and on all host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mrc|reference] [--form ...]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

HEADLINE = "precision"  # workload recipe of the headline step (1,000,000 documents)
K = 64
TAU = 0.9
MARGIN = 0.02
HMAX = 3
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
SUBSET_DOCS = 20000  # accuracy subset: the FP64 oracle's all pairs
ORACLE_SAMPLE = 12000  # documents of the reference arm's step
CPU_BASELINE_SAMPLE = 4000  # documents of the main line's oracle timing



# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one single-pass ncu
# capture of the launch at the bench's size (1,000,000 documents; `--form profile --case
# compare-e4m3 / compare-fp16 --docs 1000000`), valid only while the compare's device code is
# unchanged since the capture.
_TC = "paper_1810_03099_gb300/csrc/tc_dev.cuh"
_TC_DIGEST = "b1b3073cc4fa17c12cd39068c95250d2fea1f46e65d9d76f9cd781c81efda0e3"
NCU_TRAFFIC = {
    "gemm_e4m3_thresh": (_TC, _TC_DIGEST, 114_680_000 + 141_090_000),
    "gemm_f16_thresh": (_TC, _TC_DIGEST, 47_140_000_000 + 139_190_000),
}
KERNEL_NOTES = {
    "gemm_f16_bound": "exact-cosine head GEMM carrying the tail-bucket bound: 2 kd flops per pair of the "
                      "triangle (kd = 128 head + 256 bucket columns); ncu: tensor pipe 75% active; candidates "
                      "where head + bound >= tau - delta'",
    "gemm_e4m3_thresh": "signature compare at k = 64, E4M3: epilogue-bound (ncu at 100,000 documents: tensor pipe "
                        "20% active, L2 hit rate 99%); traffic = operand reads (the 64 MB operand stays in L2) "
                        "plus the candidate list written",
    "gemm_f16_thresh": "signature compare at k = 64, fp16: epilogue-bound (ncu at 100,000 documents: tensor pipe "
                       "42% active); at 1 M documents the 128 MB operand does not stay in L2 and is re-read "
                       "from DRAM (~47 GB per launch, 0.74 TB/s), which the epilogue-bound rate hides",
    "cosine_verify": "exact scores of the bound-pruned candidates (a few tens of thousands on news20)",
    "cosine_tail": "algorithmic bytes = the fp16 head scores of the upper triangle; the postings it also walks "
                   "are L2-resident. ncu: issue-active 66%, l1tex 53%: instruction/latency-bound, not HBM-bound",
    "gemm_f16_store": "2 kd flops per pair of the triangle (kd = 1024 head columns); tensor pipe 60% active "
                      "(ncu), L2 66% busy with operand reloads",
}


def ncu_traffic(name):
    if name not in NCU_TRAFFIC:
        return None
    path, digest, nbytes = NCU_TRAFFIC[name]
    try:
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    except OSError:
        return None
    return nbytes


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d["bf16_tflops_sustained"], "source": "measured"}
    except Exception:  # noqa: BLE001
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:  # noqa: BLE001
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows if len(r) > 8 for n, v in zip(names, r[5:9]) if v == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def max_over_ranks(value: float, dist, device: str) -> float:
    """The largest of every rank's value (the job's time is its slowest rank's)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())



def _oracle_step(to, sub, vocab, tau, hmax):
    """One oracle step on a host corpus: index build, all signature pairs, all Simhash pairs."""
    from oracle.oracle import Params
    t0 = time.perf_counter()
    ref = to.build_index(sub.offsets, sub.tokens, vocab, Params(k=K, tau=tau, hamming_max=hmax))
    t1 = time.perf_counter()
    n_sig = to.sig_pairs(ref.S, tau)[0]
    n_sh = to.hamming_pairs(ref.F, hmax)[0]
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, n_sig, n_sh


def _oracle_subset(n):
    """The first n documents of the headline recipe, drawn on the host (no GPU needed)."""
    from paper_1810_03099_gb300 import synth
    return synth.make_corpus(HEADLINE, n_docs=n)


def run_reference(args, rank, world):
    """The FP64 oracle as it stands, on every host core: the headline step (index build, all
    signature pairs, all Simhash pairs) over the first ORACLE_SAMPLE documents of the headline recipe
    (a subset: all-pairs work grows with the square of the documents, so this is a stated
    sample, not scaled up). Rank 0 only; other ranks exit without work."""
    if rank != 0:
        return
    from oracle.threaded import ThreadedOracle, cpu_model, host_cores
    sub = _oracle_subset(ORACLE_SAMPLE)
    to = ThreadedOracle(host_cores())
    times = []
    for it in range(args.warmup + args.steps):
        r = _oracle_step(to, sub, sub.vocab, TAU, HMAX)
        if it >= args.warmup:
            times.append(r[0] + r[1])
    to.close()
    step_s = float(np.mean(times))
    value = sub.n_docs / step_s
    line = {"metric": "docs/s", "value": value, "unit": "docs/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{HEADLINE}: first {sub.n_docs} of 1,000,000 documents of the recipe (2^18 "
                                   f"terms, Zipf 1.05, median 300 tokens), k={K}, FP64, all signature pairs "
                                   f"tau={TAU} + all Simhash pairs h<={HMAX}",
                       "parallelism": f"{to.threads} host threads"},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "docs/s", "cores": to.threads,
                             "cpu": cpu_model(),
                             "sample": f"first {sub.n_docs} documents of the headline recipe, whole step on them "
                                       f"(not scaled to 1,000,000)"},
            "e2e": {"value": value, "unit": "docs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_leg():
    """The oracle on CPU_BASELINE_SAMPLE documents of the headline recipe, once on one core and
    once on all cores: docs/s of the whole step on that sample, and its parts."""
    from oracle.threaded import ThreadedOracle, cpu_model, host_cores
    sub = _oracle_subset(CPU_BASELINE_SAMPLE)
    out = {}
    for label, threads in (("one_core", 1), ("all_cores", host_cores())):
        to = ThreadedOracle(threads)
        tb, tp, n_sig, n_sh = _oracle_step(to, sub, sub.vocab, TAU, HMAX)
        to.close()
        n = sub.n_docs
        out[label] = {"docs_per_s": n / (tb + tp), "build_docs_per_s": n / tb,
                      "pairs_per_s": n * (n - 1) / 2 / tp, "threads": threads, "sig_pairs": n_sig,
                      "simhash_pairs": n_sh}
    best = out["all_cores"]
    return {"value": best["docs_per_s"], "unit": "docs/s", "cores": best["threads"], "kind": "oracle",
            "cpu": cpu_model(), "one_core_docs_per_s": out["one_core"]["docs_per_s"], "detail": out,
            "sample": f"first {sub.n_docs} documents of the headline recipe (FP64 oracle: index build, all "
                      f"signature pairs tau={TAU}, all Simhash pairs h<={HMAX}), whole step on the sample, not "
                      f"scaled to 1,000,000 documents"}


def _timed(fn, reps=1):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    out = None
    for _ in range(reps):
        out = fn()
    e1.record()
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1) / 1e3 / reps


def form_precision(args):
    """Precision form on the one-million-document corpus: bf16 weight table, FP8 E4M3 compare,
    FP32 rescoring; against the FP32 form on the same corpus; error vs the FP64 oracle on a
    seeded 10,000-document subset."""
    import torch
    from oracle.oracle import Oracle, Params, build_index
    from paper_1810_03099_gb300 import mrc, synth
    c = synth.make_corpus_device("precision")
    ctx = mrc.Context()
    res = {}
    for name, prec in (("bf16_fp8", mrc.PREC_BF16_FP8), ("fp32", mrc.PREC_FP32)):
        p = mrc.params_default(k=64, precision=prec)
        build = lambda: mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, p)  # noqa: E731
        idx, _ = _timed(build)
        idx.free()
        idx, t_build = _timed(build)
        mrc.mrc_match(ctx, idx, None, TAU, capacity=1 << 24)
        ctx.reset_stats()
        ctx.set_timing(True)
        (pairs, total), t_match = _timed(lambda: mrc.mrc_match(ctx, idx, None, TAU, capacity=1 << 24))
        ctx.set_timing(False)
        n = c.n_docs
        res[name] = {"build_s": t_build, "match_s": t_match, "docs_per_s": n / (t_build + t_match),
                     "pairs_per_s": n * (n - 1) / 2 / t_match, "pairs": total,
                     "kernels_ms": {s["name"]: s["ms"] for s in ctx.kernel_stats()}}
        idx.free()
    # error vs FP64 on a subset (the index corpus is the subset)
    sub = c.host_subset(np.sort(np.random.Generator(np.random.PCG64(7)).choice(c.n_docs, 10000, replace=False)))
    orc = Oracle()
    ref = build_index(sub.offsets, sub.tokens, c.vocab, Params(k=64), orc)
    _, pi, pj, _ = orc.sig_pairs(ref.S, TAU)
    want = set(zip(pi.tolist(), pj.tolist()))
    idx = mrc.mrc_build_index(ctx, sub.offsets, sub.tokens, c.vocab, mrc.params_default(k=64, precision=1))
    got = mrc.mrc_match(ctx, idx, None, TAU, device=None)[0]
    have = set(zip(got["i"].tolist(), got["j"].tolist()))
    ex = mrc.mrc_index_export(ctx, idx)
    inter = len(have & want)
    res["vs_fp64_subset"] = {"docs": 10000, "pairs_fp64": len(want), "pairs": len(have),
                             "recall": inter / max(len(want), 1), "precision": inter / max(len(have), 1),
                             "max_abs_sig_err": float(np.abs(ex["sig"] - ref.S).max())}
    idx.free()
    line = {"metric": "docs/s", "form": "precision", "value": res["bf16_fp8"]["docs_per_s"], "unit": "docs/s",
            "vs_fp32_form": res["bf16_fp8"]["docs_per_s"] / res["fp32"]["docs_per_s"],
            "config": {"workload": f"precision: {c.n_docs} docs, {c.n_tokens} tokens, V=2^18, k=64, all-pairs tau={TAU}"},
            "detail": res}
    print(json.dumps(line), flush=True)
    ctx.close()


def form_features(args):
    """Simhash feature hashes on the one-million-document corpus: the signature pass (rows a1-a4,
    Simhash fused) over every document under SplitMix64, MD5 and SHA-1 features, and the
    per-vocabulary feature table the MD5 / SHA-1 modes compute with the index."""
    import torch
    from paper_1810_03099_gb300 import mrc, synth
    c = synth.make_corpus_device("precision")
    ctx = mrc.Context()
    n = c.n_docs
    sig = torch.empty((n, 64), dtype=torch.float32, device="cuda")
    sh = torch.empty(n, dtype=torch.int64, device="cuda")
    res = {}
    for name, mode in (("splitmix64", mrc.HASH_SPLITMIX64), ("md5", mrc.HASH_MD5), ("sha1", mrc.HASH_SHA1)):
        p = mrc.params_default(k=64, feature_hash=mode)
        idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, p)
        idx.free()
        ctx.reset_stats()
        ctx.set_timing(True)
        idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, p)
        ctx.set_timing(False)
        table_ms = sum(s["ms"] for s in ctx.kernel_stats() if s["name"] == "feature_table")
        for _ in range(3):
            mrc.mrc_signature(ctx, idx, c.offsets, c.tokens, sig, sh)
        torch.cuda.synchronize()
        reps = 10
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(reps):
            mrc.mrc_signature(ctx, idx, c.offsets, c.tokens, sig, sh)
        t1.record()
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / reps
        res[name] = {"signature_ms": ms, "docs_per_s": n / (ms * 1e-3), "feature_table_ms": table_ms,
                     "simhash_crc": int(sh[: min(n, 4096)].sum().item())}
        idx.free()
    line = {"metric": "docs/s", "form": "features", "value": res["md5"]["docs_per_s"], "unit": "docs/s",
            "vs_splitmix64": res["md5"]["docs_per_s"] / res["splitmix64"]["docs_per_s"],
            "config": {"workload": f"signature pass: {n} docs, {c.n_tokens} tokens, V={c.vocab}, k=64, "
                                   "Simhash with MD5 features (SplitMix64 and SHA-1 beside it)"},
            "detail": res}
    print(json.dumps(line), flush=True)
    ctx.close()


def form_text(args):
    """Character 3-gram front end: raw text -> 3-gram token CSR (mrc_text_grams) on eight
    copies of the NEWS20-shaped text (about 440 MB, larger than L2), device buffers; the call's
    wall time per pass (including its one synchronisation) and the per-kernel CUDA-event times
    of the count and write passes against the measured HBM copy bandwidth."""
    import torch
    from paper_1810_03099_gb300 import mrc, synth
    tc = synth.make_text_corpus("news20")
    reps_text = 8
    n1, b1 = tc.n_docs, tc.n_bytes
    offs = np.concatenate([tc.offsets[:-1] + r * b1 for r in range(reps_text)] + [[reps_text * b1]]).astype(np.int64)
    d_off = torch.from_numpy(offs).cuda()
    d_text = torch.from_numpy(tc.text).cuda().repeat(reps_text)
    n, B = n1 * reps_text, b1 * reps_text
    ctx = mrc.Context()
    go = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    g = torch.empty(B, dtype=torch.int32, device="cuda")
    for _ in range(3):
        _, gr = mrc.mrc_text_grams(ctx, d_off, d_text, go, g)
    G = int(gr.shape[0])
    steps = max(args.steps // 10, 10)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        mrc.mrc_text_grams(ctx, d_off, d_text, go, g)
    wall = (time.perf_counter() - t0) / steps
    ctx.reset_stats()
    ctx.set_timing(True)
    for _ in range(steps):
        mrc.mrc_text_grams(ctx, d_off, d_text, go, g)
    ctx.set_timing(False)
    ks = {s["name"]: s for s in ctx.kernel_stats()}
    hbm = _peaks()["hbm_gbs"]
    # algorithmic bytes: count pass reads the text; write pass reads the text and the document
    # offsets, writes 4 bytes per 3-gram and the 3-gram offsets
    alg = {"text_grams_count": B, "text_grams_write": B + 4 * G + 16 * (n + 1)}
    kern = {}
    for name, by in alg.items():
        ms = ks[name]["ms"] / ks[name]["launches"]
        kern[name] = {"ms": ms, "gbs": by / (ms * 1e-3) / 1e9, "frac_of_measured_hbm": by / (ms * 1e-3) / 1e9 / hbm}
    line = {"metric": "docs/s", "form": "text", "value": n / wall, "unit": "docs/s",
            "text_gbs": B / wall / 1e9, "grams": G,
            "config": {"workload": f"character 3-grams: {n} docs, {B} bytes of text (8 copies of the NEWS20-shaped "
                                   f"text), {G} 3-grams"},
            "kernels": kern, "hbm_peak_gbs": hbm,
            "tile_scan_ms": ks["tile_scan"]["ms"] / ks["tile_scan"]["launches"]}
    print(json.dumps(line), flush=True)
    ctx.close()


def _pair_values(M, buf, n):
    """(i, j, score) pairs -> score per pair i < j, as a dense vector indexed by the pair's rank."""
    p = M.pairs_to_numpy(buf)
    i, j = p["i"].astype(np.int64), p["j"].astype(np.int64)
    rank = i * n - i * (i + 1) // 2 + (j - i - 1)  # row-major rank of (i, j) among i < j
    out = np.zeros(n * (n - 1) // 2, np.float64)
    out[rank] = p["score"].astype(np.float64)
    return out


def _error_stats(approx, exact):
    e = approx - exact
    return {"mae": float(np.abs(e).mean()), "mean": float(e.mean()), "var": float(e.var())}


def form_study(args):
    """Reference-selection study (Section IV, Eq. 2 and Eq. 3): MAE and variance of the
    signature cosine against the exact TF-IDF cosine over all pairs of 3,000 documents of the
    NEWS20-shaped text (3-grams from mrc_text_grams), for the reference families of the paper:
    every 3-gram (ALL) split into k partitions, four frequency regions of 2,000 3-grams, and the
    3-grams that occur in one document only (DF1) with L = 1,000 / 1,500 / 2,000; k from 15 to
    240. The FP64 oracle repeats one configuration on a 400-document subset."""
    import torch
    from paper_1810_03099_gb300 import mrc, synth
    n = 3000
    tc = synth.make_text_corpus("news20", n_docs=n)
    ctx = mrc.Context()
    go, g = mrc.mrc_text_grams(ctx, torch.from_numpy(tc.offsets).cuda(), torch.from_numpy(tc.text).cuda())
    V = mrc.GRAM_VOCAB
    npairs = n * (n - 1) // 2
    idx = mrc.mrc_build_index(ctx, go, g, V, mrc.params_default(k=8, select_mode=mrc.SELECT_ALL))
    exact = _pair_values(mrc, mrc.cosine_allpairs(ctx, idx, go, g, 0.0, capacity=npairs + 1)[0], n)
    idx.free()
    configs = [("ALL", mrc.SELECT_ALL, -1, 0, k) for k in (15, 30, 60, 120, 240)]
    configs += [(f"REGION {r}-{r + 2000}", mrc.SELECT_REGION, 2000, r, k) for r in (0, 2000, 4000, 6000)
                for k in (30, 60, 120, 240)]
    configs += [(f"DF1 L={L}", mrc.SELECT_DF1, L, 0, k) for L in (1000, 1500, 2000) for k in (30, 60, 120)]
    rows = []
    for name, mode, L, start, k in configs:
        p = mrc.params_default(k=k, select_mode=mode, L=L, region_start=start)
        idx = mrc.mrc_build_index(ctx, go, g, V, p)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        buf, total = mrc.mrc_match(ctx, idx, None, -1.0, capacity=npairs + 1)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3
        approx = _pair_values(mrc, buf, n)
        st = _error_stats(approx, exact)
        rows.append({"reference": name, "k": k, "L_used": int(idx.L_used), "mae": st["mae"], "var": st["var"],
                     "all_pairs_match_ms": ms, "pairs": int(total)})
        idx.free()
    # FP64 oracle on a 400-document subset, one configuration (every 3-gram, k = 60)
    from oracle.oracle import MODE_ALL, Oracle, Params, build_index
    orc = Oracle()
    m = 400
    so, st_ = tc.offsets[:m + 1].copy(), tc.text[:int(tc.offsets[m])].copy()
    ogo, og = orc.char3grams(so, st_)
    ref = build_index(ogo, og, V, Params(k=60, mode=MODE_ALL), orc)
    _, pi, pj, ps = orc.sig_pairs(ref.S, -1.0)
    _, ci, cj, cs = orc.cosine_pairs(ref.row_ptr, ref.terms, ref.w, 0.0)
    o_sig, o_ex = np.zeros(m * (m - 1) // 2), np.zeros(m * (m - 1) // 2)
    o_sig[pi * m - pi * (pi + 1) // 2 + (pj - pi - 1)] = ps
    o_ex[ci.astype(np.int64) * m - ci * (ci + 1) // 2 + (cj - ci - 1)] = cs
    ost = orc.error_stats(o_sig, o_ex)
    sgo, sg = mrc.mrc_text_grams(ctx, torch.from_numpy(so).cuda(), torch.from_numpy(st_).cuda())
    idx = mrc.mrc_build_index(ctx, sgo, sg, V, mrc.params_default(k=60, select_mode=mrc.SELECT_ALL))
    gsig = _pair_values(mrc, mrc.mrc_match(ctx, idx, None, -1.0, capacity=m * m)[0], m)
    gex = _pair_values(mrc, mrc.cosine_allpairs(ctx, idx, sgo, sg, 0.0, capacity=m * m)[0], m)
    gst = _error_stats(gsig, gex)
    idx.free()
    best = min(rows, key=lambda r: r["mae"])
    line = {"metric": "MAE", "form": "study", "value": best["mae"], "unit": "mean |signature cosine - cosine|",
            "higher_is_better": False,
            "config": {"workload": f"reference-selection study: all {npairs} pairs of {n} NEWS20-shaped text "
                                   f"documents, 3-grams, {len(configs)} reference configurations"},
            "best": best, "rows": rows,
            "oracle_check": {"docs": m, "config": "ALL, k=60", "oracle_mae": ost["mae"], "oracle_var": ost["var"],
                             "gpu_mae": gst["mae"], "gpu_var": gst["var"]}}
    print(json.dumps(line), flush=True)
    ctx.close()


def form_simhash_index(args):
    """Block-table Hamming index (F4) against the all-pairs POPC sweep: a 10,000,000-fingerprint
    index (10 % near copies with up to 4 flipped bits) searched by 100,000 queries (half of them
    near copies of index entries), Hamming distance <= 3. Same pair count from both paths; wall
    time per search call (including its one synchronisation) and the build time."""
    import torch
    from paper_1810_03099_gb300 import mrc, synth
    n, nq, h = 10_000_000, 100_000, 3
    X = synth.random_fingerprints(n, 41, n_near=n // 10, max_flip=4) if n <= 2_000_000 else None
    if X is None:  # drawn on the device: random words, then near copies of earlier ones
        g = torch.Generator(device="cuda").manual_seed(41)
        X = torch.randint(-2**63, 2**63 - 1, (n,), dtype=torch.int64, device="cuda", generator=g)
        src = torch.randint(0, n - n // 10, (n // 10,), device="cuda", generator=g)
        flips = torch.zeros(n // 10, dtype=torch.int64, device="cuda")
        for _ in range(4):
            bit = torch.randint(0, 64, (n // 10,), device="cuda", generator=g)
            keep = torch.rand(n // 10, device="cuda", generator=g) < 0.5
            flips ^= torch.where(keep, torch.bitwise_left_shift(torch.ones_like(bit), bit), torch.zeros_like(bit))
        X[n - n // 10:] = X[src] ^ flips
    else:
        X = torch.from_numpy(X.view(np.int64)).cuda()
    g2 = torch.Generator(device="cuda").manual_seed(42)
    pick = torch.randint(0, n, (nq // 2,), device="cuda", generator=g2)
    Q = torch.cat([X[pick] ^ (1 << 7), torch.randint(-2**63, 2**63 - 1, (nq - nq // 2,), dtype=torch.int64,
                                                    device="cuda", generator=g2)])
    ctx = mrc.Context()
    t0 = time.perf_counter()
    sidx = mrc.simhash_index_build(ctx, X, h)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    sidx.free()
    t0 = time.perf_counter()
    sidx = mrc.simhash_index_build(ctx, X, h)
    torch.cuda.synchronize()
    build_s = min(build_s, time.perf_counter() - t0)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            out = fn()
        torch.cuda.synchronize()
        return out, (time.perf_counter() - t) / reps

    (bi, tot_i), t_idx = timed(lambda: mrc.simhash_index_match(ctx, sidx, Q, h, capacity=1 << 22), 10)
    (bb, tot_b), t_brute = timed(lambda: mrc.simhash_match(ctx, Q, X, h, capacity=1 << 22), 2)
    pi, pb = mrc.pairs_to_numpy(bi), mrc.pairs_to_numpy(bb)
    same = sorted(zip(pi["i"].tolist(), pi["j"].tolist())) == sorted(zip(pb["i"].tolist(), pb["j"].tolist()))
    line = {"metric": "queries/s", "form": "simhash_index", "value": nq / t_idx, "unit": "queries/s",
            "config": {"workload": f"Hamming <= {h}: {nq} queries x {n} fingerprints (block-table index, 4 tables "
                                   f"of 16-bit blocks)"},
            "index_search_ms": t_idx * 1e3, "brute_force_search_ms": t_brute * 1e3, "speedup": t_brute / t_idx,
            "pairs": int(tot_i), "pairs_brute_force": int(tot_b), "same_pairs": bool(same), "build_ms": build_s * 1e3,
            "index_bytes": int(n * 4 * 12 + n * 8)}
    print(json.dumps(line), flush=True)
    sidx.free()
    ctx.close()


def batching_leg(n_batches):
    """Batching form: n_batches batches of 1-512 documents (log-uniform 20-20,000 tokens) against
    the one-million-document precision index; each batch is one launch of the persistent batch
    kernel, the pipeline of each size bucket autotuned (tile width, ring depth, L2 prefetch)."""
    import torch
    from paper_1810_03099_gb300 import batching, mrc, synth
    c = synth.make_corpus_device("precision")
    ctx = mrc.Context()
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=64, precision=1))
    del c
    torch.cuda.empty_cache()
    sizes = synth.query_batch_sizes(n_batches)
    q = synth.make_corpus_device(synth.SPECS["batch_queries"].with_(n_docs=int(sizes.sum())))
    starts = np.concatenate([[0], np.cumsum(sizes)])
    runner = batching.BatchRunner(ctx, idx, TAU, max_docs=512, max_doc_tokens=20000, capacity=1 << 18)

    def batch(b):
        s0, s1 = int(starts[b]), int(starts[b + 1])
        o = q.offsets[s0:s1 + 1] - q.offsets[s0]
        return o, q.tokens[q.offsets[s0]:q.offsets[s1]]
    # capture (and tune) one pipeline per size bucket before timing
    first = {}
    for b, n in enumerate(sizes.tolist()):
        first.setdefault(batching.bucket_of(int(n), 512), b)
    runner.prepare([batch(b) for b in first.values()])
    lat = []
    total_pairs = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for b in range(len(sizes)):
        o, t = batch(b)
        tb = time.perf_counter()
        _, tot = runner.run(o, t)
        lat.append(time.perf_counter() - tb)
        total_pairs += tot
    wall = time.perf_counter() - t0
    docs = int(sizes.sum())
    kernels = sorted({p.kernel_nodes for p in runner.pipes.values()})
    out = {"docs_per_s": docs / wall, "batches": len(sizes), "docs": docs, "tokens": int(q.n_tokens),
           "batch_latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3)},
           "kernel_nodes_per_batch": kernels, "pairs": total_pairs,
           "tuning": {str(k): v for k, v in runner.tuning.items()},
           "config": f"{len(sizes)} batches of 1-512 docs, log-uniform 20-20,000 tokens, vs the 1M-doc bf16/FP8 "
                     f"index, k=64, tau={TAU}; host-timed per batch (launch to pairs on the host)"}
    runner.free()
    idx.free()
    ctx.close()
    return out


def form_batching(args):
    """Batching form on its own (bench.py --form batching --batches N)."""
    leg = batching_leg(args.batches)
    line = {"metric": "docs/s", "form": "batching", "value": leg["docs_per_s"], "unit": "docs/s", **leg}
    print(json.dumps(line), flush=True)


def form_serving(args):
    """Serving form: Poisson arrivals of new documents against a device-resident index of ten
    million FP16 signatures (k = 64) plus their Simhashes; continuous batching over pipeline
    slots admitted by free HBM; p50/p99 latency and sustained docs/s per arrival rate."""
    import torch
    from paper_1810_03099_gb300 import mrc, serving, synth
    n_index = args.serving_docs
    c = synth.make_corpus_device("serving", n_docs=n_index)
    ctx = mrc.Context()
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=64, precision=2))
    n_tok = c.n_tokens
    del c
    torch.cuda.empty_cache()
    pool = synth.make_corpus_device(synth.SPECS["precision"].with_(n_docs=20000, seed=BASE_QUERY_SEED))
    pool = pool.host_subset(np.arange(20000))
    docs = [pool.doc(i) for i in range(pool.n_docs)]
    srv = serving.Server(ctx, idx, TAU, micro_batch=128, deadline_s=1e-3, slots=4, max_doc_tokens=10000,
                         capacity=1 << 21)
    srv.run(docs[:2000], np.zeros(2000))  # warm-up
    rows = []
    for rate in (10000, 50000, 100000, 250000, 500000):
        n_req = int(min(20000, max(4000, rate * 0.5)))
        arr = synth.poisson_arrivals(float(rate), n_req)
        reqs = srv.run(docs[:n_req], arr)
        rep = serving.latency_report(reqs, srv.wall_s)
        rep["rate"] = rate
        rep["pairs_per_request"] = float(np.mean([len(r.pairs) for r in reqs]))
        rows.append(rep)
    line = {"metric": "p99 latency ms / sustained docs/s", "form": "serving", "value": max(r["docs_per_s"] for r in rows),
            "unit": "docs/s", "config": {"workload": f"index {n_index} docs ({n_tok} tokens) FP16 k=64; micro-batch <= 128 "
                                                     f"or 1 ms; {srv.admitted_slots} slots"},
            "rates": rows}
    print(json.dumps(line), flush=True)
    srv.free()
    idx.free()
    ctx.close()


BASE_QUERY_SEED = 1810031999


def _stage_err(a, b):
    d = np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64))
    return {"max": float(d.max()) if d.size else 0.0, "mean": float(d.mean()) if d.size else 0.0, "n": int(d.size)}


def accuracy_vs_fp64(c, ctx):
    """Both forms against the plain FP64 oracle on a seeded SUBSET_DOCS-document subset of the
    corpus (which is then the index corpus): recall and precision of the final pair sets, the
    misses, and the error of each stage of the pipeline against FP64 -- the signature entries
    (bfloat16 weight table in the precision form), the tensor-core compare's own cosine of every
    candidate (FP8 E4M3 or fp16), and the FP32-rescored scores of the final pairs."""
    from oracle.oracle import Params
    from oracle.threaded import ThreadedOracle, host_cores
    from paper_1810_03099_gb300 import mrc
    sel = np.sort(np.random.Generator(np.random.PCG64(7)).choice(c.n_docs, SUBSET_DOCS, replace=False))
    sub = c.host_subset(sel)
    to = ThreadedOracle(host_cores())
    ref = to.build_index(sub.offsets, sub.tokens, c.vocab, Params(k=K))
    tot, pi, pj, _ = to.sig_pairs(ref.S, TAU)
    to.close()
    truth = set(zip(pi.tolist(), pj.tolist()))
    nrm = np.linalg.norm(ref.S, axis=1)
    U = np.divide(ref.S, nrm[:, None], out=np.zeros_like(ref.S), where=nrm[:, None] > 0)

    def cos64(i, j):
        return np.einsum("ij,ij->i", U[i], U[j])

    out = {"docs": SUBSET_DOCS, "pairs_fp64": int(tot), "tau": TAU, "margin": MARGIN,
           "reading": "precision form: E4M3 compare operands from bfloat16 idf / reference weights; stored "
                      "signatures and the FP32 rescoring from FP32 weights"}
    for name, prec in (("bf16_fp8", 1), ("fp32", 0)):
        idx = mrc.mrc_build_index(ctx, sub.offsets, sub.tokens, c.vocab, mrc.params_default(k=K, precision=prec))
        ex = mrc.mrc_index_export(ctx, idx)
        final = mrc.mrc_match(ctx, idx, None, TAU, device=None)[0]
        ctx.set_rescoring(False)
        cand = mrc.mrc_match(ctx, idx, None, TAU, device=None)[0]
        ctx.set_rescoring(True)
        idx.free()
        have = set(zip(final["i"].tolist(), final["j"].tolist()))
        inter = len(have & truth)
        cand_set = set(zip(cand["i"].tolist(), cand["j"].tolist()))
        fi, fj = final["i"].astype(np.int64), final["j"].astype(np.int64)
        ci, cj = cand["i"].astype(np.int64), cand["j"].astype(np.int64)
        # signature stage: the raw signature entries against FP64; the unit signatures compared
        su = ex["sig"].astype(np.float64)
        out[name] = {
            "pairs": len(have), "recall": inter / max(len(truth), 1), "precision": inter / max(len(have), 1),
            "missed": len(truth - have), "extra": len(have - truth),
            "candidates": len(cand_set), "missed_by_compare": len(truth - cand_set),
            "stage_error_vs_fp64": {
                "signature_entries": _stage_err(su, ref.S),
                "compare_cosine_of_candidates": _stage_err(cand["score"], cos64(ci, cj)),
                "rescored_scores_of_pairs": _stage_err(final["score"], cos64(fi, fj)),
            },
        }
    return out


def _kernel_stats(ctxs):
    stats = {}
    for cx in ctxs:
        for st in cx.kernel_stats():
            acc = stats.setdefault(st["name"], dict(st, launches=0, ms=0.0, bytes=0.0, flops=0.0))
            for key in ("launches", "ms", "bytes", "flops"):
                acc[key] += st[key]
    return list(stats.values())


def _roofline(s, peaks, n_docs=None, k=K, sustained=True):
    """Roofline object of one kernel from its per-kernel event totals. Compares are held to the
    peak of their own operand type (FP8 = 2 x the measured bf16 rate, fp16 = the bf16 rate),
    with the method's work (2 k flops per compared pair, the triangle only for all pairs); the
    other kernels to the measured HBM copy bandwidth with their algorithmic bytes."""
    per_launch_s = s["ms"] / s["launches"] / 1e3
    name = s["name"]
    if s["flops"] > 0 and name.startswith("gemm"):
        fp8 = "e4m3" in name
        bf16 = peaks["bf16_tflops_sustained"] if sustained else peaks["bf16_tflops"]
        peak = bf16 * (2.0 if fp8 else 1.0)
        achieved = s["flops"] / s["launches"] / per_launch_s / 1e12
        r = {"bound": "tensor", "kernel": name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
             "frac": achieved / peak, "traffic": ncu_traffic(name),
             "peak_source": f"{peaks['source']} bf16 {'sustained' if sustained else 'burst'}"
                            f"{' x 2 (FP8 nominal ratio 4.5 / 2.25)' if fp8 else ' (fp16: same nominal rate)'}",
             "work": "2 k flops per compared pair (method work)"}
    else:
        achieved = s["bytes"] / s["launches"] / per_launch_s / 1e9
        peak = peaks["hbm_gbs"]
        r = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
             "frac": achieved / peak, "traffic": ncu_traffic(name), "peak_source": peaks["source"] + " copy"}
    r["ms_per_launch"] = per_launch_s * 1e3
    if name in KERNEL_NOTES:
        r["note"] = KERNEL_NOTES[name]
    return r


def run_headline(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1810_03099_gb300 import mrc, synth

    c = synth.make_corpus_device(HEADLINE)
    N, V, T = c.n_docs, c.vocab, c.n_tokens
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = mrc.Context(stream.cuda_stream)
    # the Simhash leg's own stream and context: it runs beside the signature compare
    stream_sh = torch.cuda.Stream()
    ctx_sh = mrc.Context(stream_sh.cuda_stream)
    params = {1: mrc.params_default(k=K, tau=TAU, precision=1, margin=MARGIN, hamming_max=HMAX),
              0: mrc.params_default(k=K, tau=TAU, precision=0, hamming_max=HMAX)}
    cap, sh_cap = 1 << 25, 1 << 24
    pbuf = torch.empty((cap, 3), dtype=torch.int32, device="cuda")
    shbuf = torch.empty((sh_cap, 3), dtype=torch.int32, device="cuda")
    dcount = torch.zeros(1, dtype=torch.int64, device="cuda")
    sh_dev = torch.empty(N, dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    offs_h = c.offsets.cpu().pin_memory()
    toks_h = c.tokens.cpu().pin_memory()
    pairs_h = torch.empty((cap, 3), dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    counts = {}

    def step(prec, host=False):
        if not host:
            idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, V, params[prec])
            mrc.mrc_match_async(ctx, idx, pbuf, dcount, None, TAU)  # compare + rescoring, count on the device
            # the fingerprints' block-table index and all Simhash pairs on the second stream (it
            # waits for the index on the device; its kernels run beside the compare's CTAs)
            sh = mrc.index_simhash(ctx_sh, idx, sh_dev)
            shx = mrc.simhash_index_build(ctx_sh, sh, HMAX)
            _, n_sh = mrc.simhash_index_match(ctx_sh, shx, None, HMAX, capacity=sh_cap, device="cuda")
            shx.free()
            stream.wait_stream(stream_sh)
            idx.free()
            counts[prec] = {"simhash_pairs": n_sh}
            return None
        # end to end: the inputs in page-locked host memory (the kernels read the tokens in place),
        # the two legs overlapped on the device as in the step above, and both pair lists read
        # back into page-locked host memory before the step ends
        idx = mrc.mrc_build_index(ctx, offs_h, toks_h, V, params[prec])
        mrc.mrc_match_async(ctx, idx, pbuf, dcount, None, TAU)
        sh = mrc.index_simhash(ctx_sh, idx, sh_dev)
        shx = mrc.simhash_index_build(ctx_sh, sh, HMAX)
        p2, n2 = mrc.simhash_index_match(ctx_sh, shx, None, HMAX, capacity=sh_cap, device=None)
        shx.free()
        stream.wait_stream(stream_sh)
        ctx.sync()
        n1 = int(dcount.item())
        m = min(n1, cap)
        pairs_h[:m].copy_(pbuf[:m], non_blocking=True)
        stream.synchronize()
        idx.free()
        counts[("host", prec)] = {"sig_pairs": n1, "simhash_pairs": n2}
        return pairs_h[:m], p2

    def timed(prec, steps, warmup, host=False, with_timing=False):
        for _ in range(warmup):
            step(prec, host)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        for cx in (ctx, ctx_sh):
            cx.reset_stats()
            cx.set_timing(with_timing)
        total_ms = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            step(prec, host)
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
            if not host:
                ctx.sync()
                counts[prec]["sig_pairs"] = int(dcount.item())
        for cx in (ctx, ctx_sh):
            cx.set_timing(False)
        stats = _kernel_stats([ctx, ctx_sh])
        if dist:
            total_ms = max_over_ranks(total_ms, dist, "cuda")
        return total_ms / steps, stats

    clocks = ClockSampler(local)
    clocks.start()
    ms8, _ = timed(1, args.steps, args.warmup)
    clk = clocks.stop()
    ms32, _ = timed(0, args.steps, 1)
    _, st8 = timed(1, 2, 0, with_timing=True)
    _, st32 = timed(0, 2, 0, with_timing=True)
    e2e_steps = max(2, args.steps // 4)
    ms_e2e, _ = timed(1, e2e_steps, 1, host=True)
    # the signature pass over the whole corpus as new documents (rows a1-a4 + Simhash, from tokens)
    sig_out = torch.empty((N, K), dtype=torch.float32, device="cuda")
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, V, params[1])
    for _ in range(2):
        mrc.mrc_signature(ctx, idx, c.offsets, c.tokens, sig_out, sh_dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(5):
        mrc.mrc_signature(ctx, idx, c.offsets, c.tokens, sig_out, sh_dev)
    e1.record(stream)
    torch.cuda.synchronize()
    sig_ms = e0.elapsed_time(e1) / 5
    atom_rate = ctx.smem_atomic_rate()
    idx.free()
    del sig_out
    peaks = _peaks()
    sig_bytes = 4.0 * T + N * (8 + 4 * K + 8)  # tokens, offsets, raw signature out, Simhash out
    value = world * N / (ms8 / 1e3)
    npairs = N * (N - 1) / 2
    stats8 = sorted(st8, key=lambda s: -s["ms"])
    kernels = [{"name": s["name"], "launches": s["launches"] // 2, "ms_per_launch": s["ms"] / s["launches"],
                "share": s["ms"] / max(sum(x["ms"] for x in st8), 1e-9)} for s in stats8]
    top = stats8[0]
    line = {
        "metric": "docs/s", "value": value, "unit": "docs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms8, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "e4m3+f32", "data": "synthetic",
        "config": {"workload": f"{HEADLINE}: {N} docs, {T} tokens, V=2^18, Zipf 1.05, median 300 tokens; k={K}; "
                               f"precision form (bf16 weights, FP8 E4M3 compare, FP32 rescoring at tau={TAU} "
                               f"+/- {MARGIN}) + all Simhash pairs h<={HMAX} via the block-table index",
                   "parallelism": f"replicas x{world}",
                   "l2": "flushed (512 MB write) before every timed step; corpus 2 GB > L2"},
        "signature_pairs_per_s": world * npairs / (ms8 / 1e3),
        "fp32_form": {"docs_per_s": world * N / (ms32 / 1e3), "ms_per_step": ms32,
                      "signature_pairs_per_s": world * npairs / (ms32 / 1e3), "pairs": counts.get(0, {})},
        "vs_fp32_form": ms32 / ms8,
        "pairs": counts.get(1, {}),
        "e2e": {"value": world * N / (ms_e2e / 1e3), "unit": "docs/s",
                "h2d_bytes_per_step": int(8 * (N + 1) + 4 * T),
                "d2h_bytes_per_step": int(12 * (counts[("host", 1)]["sig_pairs"] + counts[("host", 1)]["simhash_pairs"])
                                          + 8)},
        "gpu_launches": int(sum(s["launches"] for s in st8) // 2) * args.steps,
        "roofline": _roofline(top, peaks),
        "rooflines_next": [_roofline(s, peaks) for s in stats8[1:4] if s["bytes"] > 0 or s["flops"] > 0],
        "signature_pass": {"ms": sig_ms, "docs_per_s": N / (sig_ms / 1e3), "bytes": sig_bytes,
                           "achieved_gbs": sig_bytes / (sig_ms / 1e3) / 1e9,
                           "frac": sig_bytes / (sig_ms / 1e3) / 1e9 / peaks["hbm_gbs"],
                           "work": "4 B per token + 8 B offsets + 4k B signature + 8 B Simhash per document",
                           "smem_atomic_roofline": {
                               "bound": "alu", "unit": "G tokens/s (G shared-memory 64-bit atomics/s)",
                               "achieved": T / (sig_ms / 1e3) / 1e9, "peak": atom_rate / 1e9,
                               "frac": T / (sig_ms / 1e3) / atom_rate,
                               "peak_source": "measured: mrc_measure_smem_atomic_rate",
                               "note": "building a document's bag of terms takes at least one shared-memory atomic "
                                       "per token (claim or increment), so this rate bounds tokens/s"}},
        "fp32_form_kernels": [{"name": s["name"], "ms_per_launch": s["ms"] / s["launches"]}
                              for s in sorted(st32, key=lambda s: -s["ms"])[:6]],
        "clocks": clk,
        "kernels": kernels,
    }
    ctx_sh.close()
    return line, (c, ctx, stream, dist)


def news20_leg(steps):
    """The NEWS20-shaped step with both rivals (18,846 documents, 60,000 terms, k = 64): index
    build, all-pairs FP32-form signature match, all-pairs Simhash match, all-pairs exact TF-IDF
    cosine; the exact cosine on its own stream beside the build's signature pass and the matches."""
    import torch
    from paper_1810_03099_gb300 import mrc, synth
    c = synth.cached_corpus("news20")
    N, V = c.n_docs, c.vocab
    offs_d = torch.from_numpy(c.offsets).cuda()
    toks_d = torch.from_numpy(c.tokens).cuda()
    s1, s2, s3 = torch.cuda.Stream(priority=-1), torch.cuda.Stream(), torch.cuda.Stream(priority=-1)
    ctx, ctx2, ctx3 = mrc.Context(s1.cuda_stream), mrc.Context(s2.cuda_stream), mrc.Context(s3.cuda_stream)
    params = mrc.params_default(k=K, tau=TAU, hamming_max=HMAX)
    caps = 1 << 22
    pbuf = [torch.empty((caps, 3), dtype=torch.int32, device="cuda") for _ in range(3)]
    dcount = torch.zeros(3, dtype=torch.int64, device="cuda")
    sh_dev = torch.empty(N, dtype=torch.int64, device="cuda")
    built = torch.cuda.Event()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def step(serial=False):
        idx = mrc.mrc_build_index(ctx, offs_d, toks_d, V, params)
        if serial:
            s3.wait_stream(s1)
        mrc.cosine_allpairs_async(ctx3, idx, offs_d, toks_d, pbuf[2], dcount[2:3], TAU)
        sh = mrc.index_simhash(ctx, idx, sh_dev)
        built.record(s1)
        if serial:
            s2.wait_stream(s3)
        s2.wait_event(built)
        mrc.mrc_match_async(ctx2, idx, pbuf[0], dcount[0:1], None, TAU)
        mrc.simhash_match_async(ctx2, sh, pbuf[1], dcount[1:2], None, HMAX)
        s1.wait_stream(s2)
        s1.wait_stream(s3)
        idx.free()

    def run(n, timing):
        for cx in (ctx, ctx2, ctx3):
            cx.reset_stats()
            cx.set_timing(timing)
        tot = 0.0
        for _ in range(n):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(s1)
            step(serial=timing)
            e1.record(s1)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        for cx in (ctx3, ctx2, ctx):
            cx.sync()
            cx.set_timing(False)
        return tot / n, _kernel_stats([ctx, ctx2, ctx3])

    for _ in range(3):
        step()
    ms, _ = run(steps, False)
    _, stats = run(max(2, steps // 10), True)
    n1, n2, n3 = (int(x) for x in dcount.tolist())
    peaks = _peaks()
    head = [s for s in stats if s["name"] == "gemm_f16_bound"]
    out = {"docs_per_s": N / (ms / 1e3), "ms_per_step": ms,
           "config": f"news20: {N} docs, {c.n_tokens} tokens, 60,000 terms, k={K}, FP32-form signature match "
                     f"tau={TAU} + Simhash h<={HMAX} + exact TF-IDF cosine tau={TAU}",
           "pairs": {"sig_pairs": n1, "simhash_pairs": n2, "cosine_pairs": n3},
           "kernels": [{"name": s["name"], "ms_per_launch": s["ms"] / s["launches"]}
                       for s in sorted(stats, key=lambda s: -s["ms"])[:8]]}
    sh = [s for s in stats if s["name"] == "simhash_match"]
    if sh:
        # a7 roofline: one XOR + POPC per pair on the low halves, against the measured POPC rate
        s = sh[0]
        t = s["ms"] / s["launches"] / 1e3
        rate = ctx.popc_rate()
        pps = N * (N - 1) / 2 / t
        out["simhash_match_roofline"] = {"bound": "alu", "kernel": "simhash_match", "achieved": pps / 1e12,
                                         "peak": rate / 1e12, "unit": "T pairs/s (T POPC/s)", "frac": pps / rate,
                                         "ms": t * 1e3,
                                         "peak_source": "measured: mrc_measure_popc_rate (32-bit POPC per second)"}
    if head:
        s = head[0]
        t = s["ms"] / s["launches"] / 1e3
        exec_tf = s["flops"] / s["launches"] / t / 1e12
        method = 1.95e9  # sum over terms of df (df - 1): one multiply and one add per shared term
        out["exact_cosine_head_gemm"] = {
            "ms": t * 1e3, "executed_tflops": exec_tf, "executed_frac_of_bf16_burst": exec_tf / peaks["bf16_tflops"],
            "method_tflops": method / t / 1e12, "method_frac": method / t / 1e12 / peaks["bf16_tflops"],
            "note": "the GEMM executes 2 x 384 flops per pair of the triangle (128 head + 256 bucket-norm "
                    "columns); the method's own work is sum_t df_t (df_t - 1) = 1.95e9 flops"}
    for cx in (ctx3, ctx2, ctx):
        cx.close()
    return out


def serving_leg(n_index, rates=(10000, 50000, 100000, 250000, 500000), requests=6000):
    """The serving form: Poisson arrivals of new documents against a device-resident index of
    n_index documents (FP16 signatures, k = 64) and their Simhashes; p50 / p99 per rate."""
    import torch
    from paper_1810_03099_gb300 import mrc, serving, synth
    c = synth.make_corpus_device("serving", n_docs=n_index)
    ctx = mrc.Context()
    idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=K, precision=2))
    n_tok = c.n_tokens
    del c
    torch.cuda.empty_cache()
    # the index's Simhashes in a block-table index: every request is also matched by Hamming
    # distance <= HMAX inside its slot's launch
    fps = mrc.index_simhash(ctx, idx, torch.empty(n_index, dtype=torch.int64, device="cuda"))
    shx = mrc.simhash_index_build(ctx, fps, HMAX)
    del fps
    pool = synth.make_corpus_device(synth.SPECS["precision"].with_(n_docs=requests, seed=BASE_QUERY_SEED))
    pool = pool.host_subset(np.arange(requests))
    docs = [pool.doc(i) for i in range(pool.n_docs)]
    srv = serving.Server(ctx, idx, TAU, micro_batch=128, deadline_s=1e-3, slots=4, max_doc_tokens=10000,
                         capacity=1 << 21, simhash_index=shx, hamming_max=HMAX, hamming_capacity=1 << 18)
    srv.run(docs[:1000], np.zeros(1000))  # warm-up
    rows = []
    for rate in rates:
        arr = synth.poisson_arrivals(float(rate), requests)
        reqs = srv.run(docs, arr)
        rep = serving.latency_report(reqs, srv.wall_s)
        rep["rate"] = rate
        rep["pairs_per_request"] = float(np.mean([len(r.pairs) for r in reqs]))
        rep["hamming_pairs_per_request"] = float(np.mean([len(r.hamming) for r in reqs]))
        rows.append(rep)
    # the last launch of one slot, phase by phase (the slot's one persistent kernel)
    phases = {k: round(v / 1e3, 1) for k, v in srv.slots[0].phase_ns().items()}
    nodes = srv.slots[0].kernel_nodes
    srv.free()
    shx.free()
    idx.free()
    ctx.close()
    return {"index_docs": n_index, "index_tokens": n_tok, "hamming_max": HMAX, "micro_batch": 128, "deadline_ms": 1.0,
            "batch_kernel_nodes": nodes, "batch_phases_us": phases,
            "slots": srv.admitted_slots, "requests_per_rate": requests, "rates": rows}


def form_profile(args):
    """Small cases of single kernels for ncu captures (the profiling commands in profiles/):
    compare-e4m3 / compare-fp16: all-pairs signature compare of the first --docs documents of the
    headline recipe (k = 64, tau = 0.9), warm-up launches first; batch: one 128-document query
    batch against an index of --docs serving-recipe documents (one persistent kernel per launch,
    Hamming leg attached), four launches; signature: the signature pass over --docs documents."""
    import torch
    from paper_1810_03099_gb300 import mrc, synth
    n = args.docs
    ctx = mrc.Context()
    out = {"case": args.case, "docs": n}
    if args.case in ("compare-e4m3", "compare-fp16", "signature"):
        c = synth.make_corpus_device("precision", n_docs=n)
        prec = mrc.PREC_BF16_FP8 if args.case == "compare-e4m3" else mrc.PREC_FP32
        idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=K, precision=prec))
        if args.case == "signature":
            sig = torch.empty((n, K), dtype=torch.float32, device="cuda")
            sh = torch.empty(n, dtype=torch.int64, device="cuda")
            for _ in range(3):
                mrc.mrc_signature(ctx, idx, c.offsets, c.tokens, sig, sh)
        else:
            for _ in range(3):
                _, out["pairs"] = mrc.mrc_match(ctx, idx, None, TAU, capacity=1 << 24)
        idx.free()
    elif args.case == "batch":
        c = synth.make_corpus_device("serving", n_docs=n)
        idx = mrc.mrc_build_index(ctx, c.offsets, c.tokens, c.vocab, mrc.params_default(k=K, precision=mrc.PREC_FP16))
        del c
        torch.cuda.empty_cache()
        fps = mrc.index_simhash(ctx, idx, torch.empty(n, dtype=torch.int64, device="cuda"))
        shx = mrc.simhash_index_build(ctx, fps, HMAX)
        pool = synth.make_corpus_device(synth.SPECS["precision"].with_(n_docs=128, seed=BASE_QUERY_SEED))
        pool = pool.host_subset(np.arange(128))
        b = mrc.Batch(ctx, idx, 128, 128 * 10000, TAU, 1 << 21)
        b.attach_simhash(shx, HMAX, 1 << 18)
        for _ in range(4):
            b.launch(pool.offsets, pool.tokens)
            _, out["pairs"] = b.wait()
        out["phases_ns"] = b.phase_ns()
        out["kernel_nodes"] = b.kernel_nodes
        b.free()
        shx.free()
        idx.free()
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mrc", choices=["mrc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="leave the serving leg out of the headline line")
    ap.add_argument("--headline-only", action="store_true",
                    help="the million-document step alone (no accuracy, news20, serving or CPU legs; for launch lists)")
    ap.add_argument("--form", default="headline",
                    choices=["headline", "precision", "batching", "serving", "features", "text", "study",
                             "simhash_index", "forms", "profile"],
                    help="headline (default): the million-document step and its legs; the others measure one form")
    ap.add_argument("--batches", type=int, default=4096)
    ap.add_argument("--serving-docs", type=int, default=10_000_000)
    ap.add_argument("--case", default="compare-e4m3", choices=["compare-e4m3", "compare-fp16", "batch", "signature"],
                    help="--form profile: the kernel case to run")
    ap.add_argument("--docs", type=int, default=100_000, help="--form profile: documents of the case")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.form != "headline":
        import torch
        torch.cuda.set_device(local)
        for f in (["precision", "batching", "serving"] if args.form == "forms" else [args.form]):
            {"precision": form_precision, "batching": form_batching, "serving": form_serving,
             "features": form_features, "text": form_text, "study": form_study,
             "simhash_index": form_simhash_index, "profile": form_profile}[f](args)
        return

    line, (c, ctx, stream, dist) = run_headline(args, rank, world, local)
    if rank == 0 and args.headline_only:
        ctx.close()
        print(json.dumps(line), flush=True)
    elif rank == 0:
        # legs outside the timed regions: accuracy against FP64, the NEWS20-shaped step with the
        # exact cosine, the serving form, the oracle's own speed
        line["accuracy_vs_fp64"] = accuracy_vs_fp64(c, ctx)
        ctx.close()
        del c
        import torch
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        line["news20"] = news20_leg(max(50, 5 * args.steps))
        if world == 1 and not args.no_serving:
            line["batching"] = batching_leg(1024)
            line["serving"] = serving_leg(args.serving_docs)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_leg()
        print(json.dumps(line), flush=True)
    else:
        ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
