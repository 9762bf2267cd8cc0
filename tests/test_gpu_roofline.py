"""The random-access measurement behind the bench's second ceiling: every
operation (read, read + CAS, CAS alone) runs over a buffer far larger than
L2 and reports a positive, finite rate; a read followed by a CAS on the same
sector is not faster than the read alone."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_random_access_operations_report_rates(mc):
    rates = {}
    for op in (0, 1, 2):
        r = mc.mc_measure_random_access(4 << 30, 20_000_000, op)
        assert r["sectors_per_s"] > 0 and math.isfinite(r["sectors_per_s"]) and r["ms"] > 0
        rates[op] = r["sectors_per_s"]
    assert rates[1] <= rates[0] * 1.10


def test_pool_retention_keeps_and_returns_a_destroyed_models_memory(mc):
    """With a high retention the buffers of a destroyed model stay in the
    library's pool (device memory stays taken); lowering the retention gives
    them back at the next synchronisation.  The default is restored after."""
    import torch
    from paper_2305_09130_gb300 import workloads as W
    mc.mc_release_cached()
    torch.cuda.synchronize()
    try:
        mc.mc_set_pool_retention(16 << 30)
        free0 = torch.cuda.mem_get_info()[0]
        m = mc.mc_model_create(W.c3(G=24, rule=W.FREE, key_bits=128), mc.mc_options_default(engine="level"),
                               allocator=None)
        mc.mc_reserve(m)
        size = mc.mc_model_layout(m)["device_bytes"]
        assert size > 1 << 30
        assert mc.mc_count_states(m) == 63_885_179
        mc.mc_model_destroy(m)
        torch.cuda.synchronize()
        kept = free0 - torch.cuda.mem_get_info()[0]
        assert kept >= size - (256 << 20), (kept, size)
        mc.mc_set_pool_retention(0)
        torch.cuda.synchronize()
        back = free0 - torch.cuda.mem_get_info()[0]
        assert back <= (256 << 20), back
    finally:
        mc.mc_set_pool_retention(1 << 30)
        mc.mc_release_cached()
