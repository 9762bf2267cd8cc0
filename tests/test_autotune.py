"""Autotuner: search, correctness guard and cache (host logic on CPU; the
GPU test tunes a real query)."""
import json

import pytest

from paper_2305_09130_gb300 import autotune as AT
from paper_2305_09130_gb300 import workloads as W


def test_picks_the_fastest_candidate_with_the_reference_answer():
    space = {"threads_per_block": [128, 256], "blocks_per_sm": [1, 2], "load_factor_pct": [25]}

    def measure(c):
        ms = 10.0 / c["blocks_per_sm"] + (1.0 if c["threads_per_block"] == 128 else 0.5)
        return ms, "answer"

    out = AT.tune(measure, space, reps=2)
    assert out["options"] == {"threads_per_block": 256, "blocks_per_sm": 2, "load_factor_pct": 25}
    assert len(out["timings"]) == 4


def test_rejects_candidates_that_change_the_answer():
    space = {"threads_per_block": [128, 256], "blocks_per_sm": [1], "load_factor_pct": [25]}

    def measure(c):
        # the faster candidate is wrong: it must not win
        return (1.0, "wrong") if c["threads_per_block"] == 256 else (5.0, "right")

    out = AT.tune(measure, space, reps=1)
    assert out["options"]["threads_per_block"] == 128
    assert len(out["timings"]) == 1


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "cache.json")
    AT.save_cache({"sig": {"options": {"blocks_per_sm": 2}, "ms": 1.0}}, p)
    assert AT.load_cache(p)["sig"]["options"] == {"blocks_per_sm": 2}
    assert AT.load_cache(str(tmp_path / "missing.json")) == {}


def test_signature_separates_shapes():
    lay = {"key_bits": 64, "max_level": 66, "state_bound": 8763}
    a = AT.signature(lay, W.c1(W.FREE), "min_time")
    b = AT.signature(lay, W.c1(W.GREEDY), "min_time")
    c = AT.signature(lay, W.c1(W.FREE), "count")
    assert len({a, b, c}) == 3


@pytest.mark.gpu
def test_tuned_options_reproduce_results(mc, tmp_path):
    path = str(tmp_path / "tune.json")
    spec = W.c1(W.FREE)
    space = {"threads_per_block": [128, 256], "blocks_per_sm": [0, 1], "load_factor_pct": [25, 50]}
    out = AT.tune_query(spec, "min_time", space=space, reps=1, path=path)
    assert len(out["timings"]) == 8
    opts = AT.options_for(spec, "min_time", path=path)
    m = mc.mc_model_create(spec, opts)
    assert mc.mc_min_time(m, trace=False)["t_min"] == 80
    assert json.load(open(path))[out["signature"]]["options"] == out["options"]


def test_candidates_cover_knobs_outside_the_default_space():
    c = AT.candidates({"lanes_per_state": [8, 16], "blocks_per_sm": [0, 1]})
    assert sorted((x["lanes_per_state"], x["blocks_per_sm"]) for x in c) == [(8, 0), (8, 1), (16, 0), (16, 1)]
