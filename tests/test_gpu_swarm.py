"""Swarm search (Section 5) on the GPU against the oracle's replay of the
same counter-based runs."""
import pytest

import replay as RP
from paper_2305_09130_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("spec", [W.tiny(W.FREE), W.tiny(W.GREEDY), W.c1(W.FREE), W.c1(W.GREEDY),
                                  W.random_small(81, 5, 3, 2, 6, rule=W.FREE),
                                  W.random_small(82, 8, 2, 2, 4, rule=W.GREEDY, key_bits=128)],
                         ids=lambda s: f"{s.name}_r{s.rule}_k{s.key_bits}")
def test_swarm_matches_oracle(mc, oracle, spec):
    for seed, walks in ((7, 256), (2305091300, 1000)):
        m = mc.mc_model_create(spec)
        got = mc.mc_swarm(m, seed, walks, max_rounds=40)
        exp = oracle.swarm(spec, seed, walks, 40)
        for k in ("best_time", "first_time", "rounds", "walks", "best_walk", "i", "j"):
            assert got[k] == exp[k], (k, got, exp)
        lay = mc.mc_model_layout(m)
        t, i, j, _n = RP.replay(spec, lay, got["trace"], lambda t: t == got["best_time"])
        assert (i, j) == (got["i"], got["j"])
        assert got["best_time"] >= oracle.min_time(spec)["t_min"]
