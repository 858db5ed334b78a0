"""Benchmark of the Multi-reference Cosine hot path on one GB300 (replicas on N GPUs).

One step = the whole path over the NEWS20-shaped synthetic corpus (18,846
documents, 60,000 terms, k = 64): index build (term counts, TF-IDF, reference
selection, signatures, Simhash, packed operands), all-pairs signature match
(FP32 form, tau = 0.9), all-pairs Simhash match (Hamming <= 3), and all-pairs
exact TF-IDF cosine (tau = 0.9).

value = documents/s of the whole step with inputs resident in HBM; e2e = the
same through the C ABI with host buffers (host->device copies of the corpus
and device->host copies of every pair list inside the timed region).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mrc|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "news20"
K = 64
TAU = 0.9
HMAX = 3
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d["bf16_tflops_sustained"], "source": "measured"}
    except Exception:  # noqa: BLE001
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

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
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
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


def load_workload():
    from paper_1810_03099_gb300 import synth
    return synth.cached_corpus(WORKLOAD)


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, on a bounded sample of the same workload."""
    if rank != 0:
        return
    from oracle.oracle import Oracle, Params, build_index
    c = load_workload()
    N = c.n_docs
    n = 3000  # sample: the first 3,000 documents
    sub = c.subset(np.arange(n))
    orc = Oracle()
    p = Params(k=K, tau=TAU, hamming_max=HMAX)
    times = []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        ref = build_index(sub.offsets, sub.tokens, c.vocab, p, orc)
        t1 = time.perf_counter()
        orc.sig_pairs(ref.S, TAU)
        orc.hamming_pairs(ref.F, None, HMAX)
        orc.cosine_pairs(ref.row_ptr, ref.terms, ref.w, TAU)
        t2 = time.perf_counter()
        if it >= args.warmup:
            times.append((t1 - t0, t2 - t1))
    lin = float(np.mean([t[0] for t in times]))
    quad = float(np.mean([t[1] for t in times]))
    # per-document work scales with N, pair work with N^2: extrapolate the sample to the workload
    full_s = lin * (N / n) + quad * (N / n) ** 2
    value = N / full_s
    line = {"metric": "docs/s", "value": value, "unit": "docs/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": full_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"{WORKLOAD}: 18,846 docs, 60,000 terms, k={K}, all-pairs signature match "
                                   f"tau={TAU} + Simhash h<={HMAX} + exact cosine tau={TAU}"},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "docs/s", "cores": 1,
                             "sample": f"first {n} of {N} documents per step; per-document time scaled by N/n and "
                                       f"all-pairs time by (N/n)^2"},
            "e2e": {"value": value, "unit": "docs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_leg(c):
    """A short timing of the oracle (same as --impl reference, fewer steps)."""
    from oracle.oracle import Oracle, Params, build_index
    N = c.n_docs
    n = 3000
    sub = c.subset(np.arange(n))
    orc = Oracle()
    p = Params(k=K, tau=TAU, hamming_max=HMAX)
    t0 = time.perf_counter()
    ref = build_index(sub.offsets, sub.tokens, c.vocab, p, orc)
    t1 = time.perf_counter()
    orc.sig_pairs(ref.S, TAU)
    orc.hamming_pairs(ref.F, None, HMAX)
    orc.cosine_pairs(ref.row_ptr, ref.terms, ref.w, TAU)
    t2 = time.perf_counter()
    full_s = (t1 - t0) * (N / n) + (t2 - t1) * (N / n) ** 2
    return {"value": N / full_s, "unit": "docs/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} of {N} documents, one pass; per-document time x N/n, all-pairs time x (N/n)^2"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mrc", choices=["mrc", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1810_03099_gb300 import mrc

    c = load_workload()
    N, V = c.n_docs, c.vocab
    offs_d = torch.from_numpy(c.offsets).cuda()
    toks_d = torch.from_numpy(c.tokens).cuda()
    offs_h = torch.from_numpy(c.offsets).pin_memory()
    toks_h = torch.from_numpy(c.tokens).pin_memory()
    stream = torch.cuda.current_stream()
    ctx = mrc.Context(stream.cuda_stream)
    params = mrc.params_default(k=K, tau=TAU, hamming_max=HMAX)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    caps = {"sig": 1 << 22, "cos": 1 << 22, "sh": 1 << 22}
    counts = {}

    def step(host: bool):
        if host:
            idx = mrc.mrc_build_index(ctx, offs_h, toks_h, V, params)
            ex_sh = mrc.index_simhash(ctx, idx, np.empty(N, np.uint64))
            p1, n1 = mrc.mrc_match(ctx, idx, None, TAU, capacity=caps["sig"], device=None)
            p2, n2 = mrc.simhash_match(ctx, ex_sh, None, HMAX, capacity=caps["sh"], device=None)
            p3, n3 = mrc.cosine_allpairs(ctx, idx, offs_h, toks_h, TAU, capacity=caps["cos"], device=None)
        else:
            idx = mrc.mrc_build_index(ctx, offs_d, toks_d, V, params)
            sh = mrc.index_simhash(ctx, idx, torch.empty(N, dtype=torch.int64, device="cuda"))
            p1, n1 = mrc.mrc_match(ctx, idx, None, TAU, capacity=caps["sig"])
            p2, n2 = mrc.simhash_match(ctx, sh, None, HMAX, capacity=caps["sh"])
            p3, n3 = mrc.cosine_allpairs(ctx, idx, offs_d, toks_d, TAU, capacity=caps["cos"])
        idx.free()
        counts.update(sig_pairs=n1, simhash_pairs=n2, cosine_pairs=n3)
        return (p1, p2, p3)

    def timed(host: bool, steps: int, warmup: int, with_timing: bool):
        for _ in range(warmup):
            step(host)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        ctx.reset_stats()
        ctx.set_timing(with_timing)
        total_ms = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            step(host)
            e1.record(stream)
            torch.cuda.synchronize()
            total_ms += e0.elapsed_time(e1)
        ctx.set_timing(False)
        stats = ctx.kernel_stats()
        if dist:
            t = torch.tensor([total_ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total_ms = float(t.item())
        return total_ms, stats

    clocks = ClockSampler(local)
    clocks.start()
    dev_ms, stats = timed(False, args.steps, args.warmup, True)
    clk = clocks.stop()
    host_ms, _ = timed(True, max(2, args.steps // 2), 1, False)

    ms_step = dev_ms / args.steps
    value = world * N / (ms_step / 1e3)
    e2e_ms = host_ms / max(2, args.steps // 2)
    e2e = world * N / (e2e_ms / 1e3)
    pair_bytes = 12 * (counts["sig_pairs"] + counts["simhash_pairs"] + counts["cosine_pairs"])

    peaks = _peaks()
    top = max(stats, key=lambda s: s["ms"]) if stats else None
    roofline = None
    kernels = []
    for s in sorted(stats, key=lambda s: -s["ms"]):
        per = s["ms"] / max(s["launches"], 1)
        kernels.append({"name": s["name"], "launches": s["launches"], "ms_per_launch": per,
                        "share": s["ms"] / max(sum(x["ms"] for x in stats), 1e-9)})
    if top:
        per_launch_s = top["ms"] / top["launches"] / 1e3
        if top["flops"] > 0 and top["name"].startswith("gemm"):
            achieved = top["flops"] / top["launches"] / per_launch_s / 1e12
            peak = peaks["bf16_tflops"]
            roofline = {"bound": "tensor", "kernel": top["name"], "achieved": achieved, "peak": peak,
                        "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                        "peak_source": peaks["source"] + " bf16 burst (fp16 same rate)",
                        "note": "executed split-fp16 flops (3 products per term pair)"}
        else:
            achieved = top["bytes"] / top["launches"] / per_launch_s / 1e9
            peak = peaks["hbm_gbs"]
            roofline = {"bound": "hbm", "kernel": top["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None, "peak_source": peaks["source"]}
    gpu_launches = int(sum(s["launches"] for s in stats))

    line = {
        "metric": "docs/s", "value": value, "unit": "docs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: 18,846 docs, 60,000 terms, k={K}, all-pairs signature match "
                               f"tau={TAU} (FP32 form) + Simhash h<={HMAX} + exact TF-IDF cosine tau={TAU}",
                   "parallelism": f"replicas x{world}", "l2": "flushed (512 MB write) before every timed step"},
        "e2e": {"value": e2e, "unit": "docs/s", "h2d_bytes_per_step": int(8 * (N + 1) + 4 * c.n_tokens) * 2,
                "d2h_bytes_per_step": int(pair_bytes + 8 * N)},
        "gpu_launches": gpu_launches,
        "roofline": roofline,
        "clocks": clk,
        "pairs": counts,
        "signature_pairs_per_s": None,
        "kernels": kernels[:8],
    }
    sig_k = [s for s in stats if s["name"] == "gemm_split16_thresh"]
    if sig_k:
        per = sig_k[0]["ms"] / sig_k[0]["launches"] / 1e3
        line["signature_pairs_per_s"] = N * (N - 1) / 2 / per
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_leg(c)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
