"""The measurement probes behind two rooflines: the POPC issue rate (bound of the Simhash
match) and the shared-memory 64-bit atomic rate (bound of the signature pass). Each returns a
positive rate below what the SMs could issue at the highest clock (one operation per lane per
cycle), and repeated calls agree within a factor of two."""
import pytest

from tests.gpu_common import cuda_or_skip

pytestmark = pytest.mark.gpu


def test_probe_rates_are_plausible():
    torch = cuda_or_skip()
    from paper_1810_03099_gb300 import mrc
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * 2.2e9  # 128 lanes per SM and cycle at 2.2 GHz
    with mrc.Context() as ctx:
        for probe in (ctx.popc_rate, ctx.smem_atomic_rate):
            a, b = probe(), probe()
            assert 0 < a < ceiling and 0 < b < ceiling
            assert 0.5 < a / b < 2.0
