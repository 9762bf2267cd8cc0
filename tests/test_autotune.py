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


def test_candidates_of_several_spaces_are_their_union():
    c = AT.candidates([{"engine": [1], "blocks_per_sm": [0, 2]}, {"engine": [2], "unit_threads": [0, 256]},
                       {"engine": [1], "blocks_per_sm": [2]}])
    assert c == [{"engine": 1, "blocks_per_sm": 0}, {"engine": 1, "blocks_per_sm": 2},
                 {"engine": 2, "unit_threads": 0}, {"engine": 2, "unit_threads": 256}]
    # the named knobs of both engines
    level = AT.candidates(AT.LEVEL_SPACE)
    assert {"probe_scheme", "stage_chunk", "load_factor_pct", "blocks_per_sm"} <= set(level[0])
    config = AT.candidates(AT.CONFIG_SPACE)
    assert {"unit_threads", "lanes_per_state"} <= set(config[0])


def test_candidates_the_library_refuses_are_skipped():
    space = {"lanes_per_state": [0, 2, 4]}

    def measure(c):
        if c["lanes_per_state"] == 2:
            raise RuntimeError("lanes below P")
        return 1.0 + c["lanes_per_state"], "answer"

    out = AT.tune(measure, space, reps=1)
    assert out["options"] == {"lanes_per_state": 0} and len(out["timings"]) == 2


@pytest.mark.gpu
def test_tuning_covers_both_engines_and_their_knobs(mc, tmp_path):
    """The single-model tuner searches both engines (C1 fits the configuration
    engine) and the batch tuner both batch engines; every candidate it keeps
    gave the default's answer."""
    path = str(tmp_path / "tune.json")
    spec = W.c1(W.GREEDY)
    space = [dict(AT.LEVEL_SPACE, load_factor_pct=[25], blocks_per_sm=[0]),
             dict(AT.CONFIG_SPACE, unit_threads=[0, 256])]
    out = AT.tune_query(spec, "min_time", space=space, reps=1, path=path)
    keys = [json.loads(k) for k in out["timings"]]
    assert {k["engine"] for k in keys} == {1, 2}
    assert {k.get("stage_chunk") for k in keys if k["engine"] == 1} == {64, 128, 192}
    assert {k.get("probe_scheme") for k in keys if k["engine"] == 1} == {1, 2, 3, 4}
    assert {k.get("lanes_per_state") for k in keys if k["engine"] == 2} == {0, 16}
    assert len(keys) == 12 + 4  # probe scheme x chunk, threads x lanes
    m = mc.mc_model_create(spec, AT.options_for(spec, "min_time", path=path))
    assert mc.mc_min_time(m, trace=False)["t_min"] == 80
    specs = W.c4_instances(12)
    queries = [("min_time", None)] * 12
    b = AT.tune_batch(specs, queries, reps=1, cache={}, path=str(tmp_path / "b.json"))
    assert {json.loads(k)["engine"] for k in b["timings"]} == {1, 2}
