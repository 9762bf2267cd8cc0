"""The model's statistics with mc_options.timing = 1: every exploration
launch's CUDA-event time is counted once.  The library reads a launch's pair
of events lazily (when the statistics are read, or when the pair comes round
again in its ring of 64), so this checks many launches without a read in
between, the ring wrapping, and a reset dropping pairs not yet read."""
import pytest

from paper_2305_09130_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_timed_launches_are_each_counted_once(mc):
    m = mc.mc_model_create(W.c2_star(), mc.mc_options_default(timing=1, load_factor_pct=10))
    mc.mc_min_time(m, trace=False)  # sizes the buffers
    per_launch = []
    for _ in range(5):  # read after every query
        mc.mc_reset_stats(m)
        mc.mc_min_time(m, trace=False)
        st = mc.mc_get_stats(m)
        assert st["explore_launches"] == 3  # the lowering's three checks
        per_launch.append(st["explore_ms"] / 3)
    eager = sorted(per_launch)[2]

    mc.mc_reset_stats(m)
    for _ in range(30):  # 90 launches, no read in between: the ring of 64 pairs wraps
        mc.mc_min_time(m, trace=False)
    st = mc.mc_get_stats(m)
    assert st["explore_launches"] == 90
    assert 0.8 * eager < st["explore_ms"] / 90 < 1.25 * eager
    assert mc.mc_get_stats(m)["explore_ms"] == st["explore_ms"]  # a second read adds nothing

    for _ in range(10):  # pending when the reset comes: dropped with it
        mc.mc_min_time(m, trace=False)
    mc.mc_reset_stats(m)
    mc.mc_min_time(m, trace=False)
    st = mc.mc_get_stats(m)
    assert st["explore_launches"] == 3
    assert 0.5 * eager < st["explore_ms"] / 3 < 2.0 * eager
    mc.mc_model_destroy(m)


def test_untimed_queries_report_no_time(mc):
    m = mc.mc_model_create(W.c1(), mc.mc_options_default(timing=0))
    for _ in range(3):
        assert mc.mc_min_time(m, trace=False)["t_min"] == 80
    st = mc.mc_get_stats(m)
    assert st["explore_launches"] > 0 and st["explore_ms"] == 0.0
    mc.mc_model_destroy(m)
