"""Host-side logic of the batching and serving forms (no GPU): size buckets, a pipeline slot's
device footprint (what admission by free memory divides by), and the latency report."""
import numpy as np

from paper_1810_03099_gb300 import batching, serving


def test_bucket_of_rounds_up_to_a_power_of_two_capped_by_max_docs():
    assert [batching.bucket_of(n, 512) for n in (1, 2, 3, 4, 5, 127, 128, 129, 511, 512)] == [
        1, 2, 4, 4, 8, 128, 128, 256, 512, 512]
    assert batching.bucket_of(600, 512) == 512  # never above the pipeline's capacity
    assert batching.bucket_of(100, 96) == 96


class _Index:
    def __init__(self, k):
        self.k = k


def test_slot_footprint_counts_every_buffer_and_grows_with_each_size():
    base = serving.slot_footprint(_Index(64), 128, 128 * 10000, 1 << 16)
    # the token buffer alone is 4 bytes per token; the candidate list 12 bytes per candidate
    assert base > 4 * 128 * 10000 + 12 * 4 * (1 << 16)
    assert serving.slot_footprint(_Index(64), 256, 128 * 10000, 1 << 16) > base
    assert serving.slot_footprint(_Index(64), 128, 256 * 10000, 1 << 16) > base
    assert serving.slot_footprint(_Index(64), 128, 128 * 10000, 1 << 17) > base
    assert serving.slot_footprint(_Index(128), 128, 128 * 10000, 1 << 16) > base


def test_latency_report_percentiles():
    class R:
        def __init__(self, a, d):
            self.arrival, self.done = a, d

    lat = np.arange(1, 101) * 1e-3  # 1 .. 100 ms
    reqs = [R(0.0, x) for x in lat]
    rep = serving.latency_report(reqs, wall_s=2.0)
    assert rep["requests"] == 100
    assert abs(rep["p50_ms"] - np.percentile(lat, 50) * 1e3) < 1e-9
    assert abs(rep["p99_ms"] - np.percentile(lat, 99) * 1e3) < 1e-9
    assert abs(rep["max_ms"] - 100.0) < 1e-9
    assert rep["docs_per_s"] == 50.0
