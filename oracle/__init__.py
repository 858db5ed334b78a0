"""FP64 CPU oracle of Multi-reference Cosine (arXiv 1810.03099).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``. The product package never imports it.

Parity status of each function (what pins it) is listed in ``tests/test_oracle_pins.py``.
"""
