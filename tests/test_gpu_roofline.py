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
