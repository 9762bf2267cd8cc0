"""Batched exploration (many models per run: the lockstep engine's one
persistent launch, or the configuration engine's four launches) against the
CPU oracle, the closed forms and the single-model entry points.

Integer results, tolerance zero: per instance the decision, counts, levels,
counterexample or minimum, configuration and witness state; traces replay.
"""
import pytest

import closed_forms as CF
import replay as RP
from paper_2305_09130_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NO_LIMIT = (1 << 64) - 1
ENGINES = ["level", "config"]


def engine_launches(mc, b, engine, runs):
    """The engine that ran: one exploration launch per run on the lockstep
    engine, two (first passes; certificate and final passes) on the
    configuration engine."""
    assert mc.mc_batch_get_stats(b)["explore_launches"] == runs * (2 if engine == "config" else 1)


def layout128(mc, spec):
    m = mc.mc_model_create(spec.with_key_bits(128), allocator=None)
    return mc.mc_model_layout(m)


def mixed_specs():
    specs = [W.tiny(W.FREE), W.tiny(W.GREEDY), W.c1(W.FREE), W.c1(W.GREEDY)]
    seed = 7000
    shapes = [(1, 2, 2, 9), (2, 3, 2, 8), (3, 2, 2, 6), (4, 2, 3, 5), (5, 2, 1, 5), (6, 1, 2, 4),
              (8, 2, 2, 3), (12, 1, 1, 3), (16, 1, 2, 2)]
    for P, a, b, n_max in shapes:
        for rule in (W.FREE, W.GREEDY):
            specs.append(W.random_small(seed, P, a, b, n_max, cost_max=7, speed_max=3, rule=rule))
            seed += 1
    return specs


def make_queries(specs, t_mins):
    rng = W.SplitMix64(2305091399)
    q = []
    for spec, t in zip(specs, t_mins):
        if rng.uniform(0, 1):
            q.append(("min_time", None))
        else:
            q.append(("check", max(0, round(t * rng.uniform(800, 1200) / 1000))))
    return q


def check_against_oracle(mc, oracle, spec, query, r):
    lay = layout128(mc, spec)
    assert r["status"] == 0
    if query[0] == "check":
        T = query[1]
        exp = oracle.check(spec, T)
        got = {"holds": r["holds"], "states": r["states"], "levels": r["levels"]}
        if not r["holds"]:
            i, j, n = RP.decode(lay, r["key"])
            got.update(cex_time=r["time"], cex_i=r["i"], cex_j=r["j"], cex_level=r["level"], cex_n=n)
            assert (i - 1, j - 1) == (r["i"], r["j"])
        assert got == exp
    else:
        exp = oracle.min_time(spec)
        i, j, n = RP.decode(lay, r["key"])
        got = {"t_min": r["time"], "t_ini": r["t_ini"], "states": r["states"], "checks": r["checks"],
               "i": r["i"], "j": r["j"], "level": r["level"], "n": n}
        assert got == exp


@pytest.mark.parametrize("engine", ENGINES)
def test_batch_matches_oracle(mc, oracle, engine):
    specs = mixed_specs()
    t_mins = [oracle.min_time(s)["t_min"] for s in specs]
    queries = make_queries(specs, t_mins)
    assert {k for k, _ in queries} == {"check", "min_time"}
    b = mc.mc_batch_create(specs, mc.mc_options_default(engine=engine))
    for _run in range(2):  # the pool is reused; results must not depend on its contents
        res = mc.mc_batch_run(b, queries)
        for k, (spec, q, r) in enumerate(zip(specs, queries, res)):
            check_against_oracle(mc, oracle, spec, q, r)
            if q[0] == "min_time" or not r["holds"]:
                keys = mc.mc_batch_trace(b, k)
                assert len(keys) == r["level"] + 1 and keys[-1] == r["key"]
                bound = r["time"]
                RP.replay(spec, layout128(mc, spec), keys,
                          (lambda t, b_=bound: t == b_) if q[0] == "min_time" else (lambda t, T=q[1]: t <= T))
    # the runs replay one captured CUDA graph; new queries reach it through
    # its pinned inputs
    flipped = [("min_time", None) if k == "check" else ("check", t - 1) for (k, _T), t in zip(queries, t_mins)]
    for spec, q, r in zip(specs, flipped, mc.mc_batch_run(b, flipped)):
        check_against_oracle(mc, oracle, spec, q, r)
    assert mc.mc_batch_get_stats(b)["graph_launches"] == 3
    engine_launches(mc, b, engine, 3)


@pytest.mark.parametrize("engine", ENGINES)
def test_batch_equals_single_model_queries(mc, engine):
    specs = W.c4_instances(96)
    t_mins = [CF.tmin(s)[0] for s in specs]
    queries = c4_queries(specs, t_mins)
    b = mc.mc_batch_create(specs, mc.mc_options_default(engine=engine))
    res = mc.mc_batch_run(b, queries)
    engine_launches(mc, b, engine, 1)
    for spec, q, r, t_min in zip(specs, queries, res, t_mins):
        check_against_single_model(mc, spec, q, r, t_min)


def c4_queries(specs, t_mins):
    return [("min_time", None) if s.meta["query"] else ("check", round(t * s.meta["t_frac_milli"] / 1000))
            for s, t in zip(specs, t_mins)]


def check_against_single_model(mc, spec, q, r, t_min):
    """One batch answer equals the single-model entry point's, and a minimum
    or a check's outcome agrees with the closed-form minimal time."""
    assert r["status"] == 0
    m = mc.mc_model_create(spec.with_key_bits(128))
    if q[0] == "min_time":
        s = mc.mc_min_time(m, trace=False)
        assert (r["time"], r["t_ini"], r["i"], r["j"], r["states"], r["checks"], r["level"], r["key"]) == \
               (s["t_min"], s["t_ini"], s["i"], s["j"], s["states"], s["checks"], s["level"], s["witness_key"])
        assert r["time"] == t_min
    else:
        s = mc.mc_check(m, q[1], trace=False)
        assert r["holds"] == s["holds"] == (q[1] < t_min)
        assert (r["states"], r["levels"]) == (s["states"], s["levels"])
        if not s["holds"]:
            assert (r["time"], r["i"], r["j"], r["level"], r["key"]) == \
                   (s["cex_time"], s["cex_i"], s["cex_j"], s["cex_level"], s["cex_key"])
    mc.mc_model_destroy(m)


@pytest.mark.parametrize("kind", ["warp", "block"])
def test_configuration_batch_of_one_unit_kind(mc, kind):
    """A configuration-engine batch whose models all run a warp per
    configuration (no block units in its launches), or all a block per
    configuration (no warp blocks), answers as the single-model entry points,
    over two replays of its graph with the queries swapped between them."""
    specs = []
    for s in W.c4_instances(96):
        m = mc.mc_model_create(s.with_key_bits(128), mc.mc_options_default(engine="config"))
        mc.mc_reserve(m)
        if (mc.mc_model_layout(m)["unit_threads"] == 32) == (kind == "warp"):
            specs.append(s)
        mc.mc_model_destroy(m)
    assert len(specs) >= 16
    t_mins = [CF.tmin(s)[0] for s in specs]
    queries = c4_queries(specs, t_mins)
    swapped = [("min_time", None) if k == "check" else ("check", t - 1) for (k, _T), t in zip(queries, t_mins)]
    b = mc.mc_batch_create(specs, mc.mc_options_default(engine="config"))
    for qs in (queries, swapped, queries):
        for spec, q, r, t_min in zip(specs, qs, mc.mc_batch_run(b, qs), t_mins):
            check_against_single_model(mc, spec, q, r, t_min)
    assert mc.mc_batch_get_stats(b)["graph_launches"] == 3
    engine_launches(mc, b, "config", 3)


@pytest.mark.parametrize("engine", ENGINES)
def test_batch_full_c4_in_the_bench_configuration(mc, engine):
    """All 256 C4 instances in one batch with options the benchmark's tuner
    may pick (one block per SM, load factor 25%), run twice through the
    captured graph: every answer equals the single-model entry point's and the
    closed-form minimal time."""
    specs = W.c4_instances(256)
    t_mins = [CF.tmin(s)[0] for s in specs]
    queries = [("min_time", None) if s.meta["query"] else ("check", round(t * s.meta["t_frac_milli"] / 1000))
               for s, t in zip(specs, t_mins)]
    b = mc.mc_batch_create(specs, mc.mc_options_default(blocks_per_sm=1, load_factor_pct=25, engine=engine))
    first = mc.mc_batch_run(b, queries)
    again = mc.mc_batch_run(b, queries)
    assert [(r["status"], r["time"], r["states"], r["key"]) for r in first] == \
           [(r["status"], r["time"], r["states"], r["key"]) for r in again]
    for spec, q, r, t_min in zip(specs, queries, first, t_mins):
        assert r["status"] == 0
        m = mc.mc_model_create(spec.with_key_bits(128))
        if q[0] == "min_time":
            s = mc.mc_min_time(m, trace=False)
            assert r["time"] == s["t_min"] == t_min
            assert (r["i"], r["j"], r["states"], r["checks"], r["key"]) == \
                   (s["i"], s["j"], s["states"], s["checks"], s["witness_key"])
        else:
            s = mc.mc_check(m, q[1], trace=False)
            assert r["holds"] == s["holds"] == (q[1] < t_min)
            assert (r["states"], r["levels"]) == (s["states"], s["levels"])
        mc.mc_model_destroy(m)
    assert mc.mc_batch_get_stats(b)["graph_launches"] == 2
    engine_launches(mc, b, engine, 2)


def test_batch_with_a_model_the_configuration_engine_cannot_take(mc, oracle):
    """AUTO takes the lockstep engine for the whole batch when one instance's
    configuration levels are too wide (C2 at G=80 under FREE); forcing the
    configuration engine is refused."""
    specs = [W.c1(W.GREEDY), W.c2_star()]
    b = mc.mc_batch_create(specs)
    res = mc.mc_batch_run(b, [("check", 80), ("check", 95)])
    engine_launches(mc, b, "level", 1)
    for spec, T, r in zip(specs, (80, 95), res):
        e = oracle.check(spec, T)
        assert (r["holds"], r["states"], r["levels"], r["time"]) == (e["holds"], e["states"], e["levels"],
                                                                     e.get("cex_time", 0))
    assert not res[0]["holds"] and res[1]["holds"]
    with pytest.raises(mc.MCError) as err:
        mc.mc_batch_create(specs, mc.mc_options_default(engine="config"))
    assert err.value.code == mc.MC_ERR_INVAL


def test_batch_errors_are_per_instance(mc):
    specs = [W.c1(W.FREE), W.tiny(W.GREEDY)]
    b = mc.mc_batch_create(specs, mc.mc_options_default(table_log2=3, max_probes=1, engine="level"))
    res = mc.mc_batch_run(b, [("check", NO_LIMIT), ("min_time", None)])
    assert [r["status"] for r in res] == [mc.MC_ERR_TABLE_FULL, mc.MC_ERR_TABLE_FULL]


def test_batch_barrier_timeout(mc):
    b = mc.mc_batch_create([W.c1(W.FREE)], mc.mc_options_default(debug_barrier_extra=1,
                                                                    barrier_timeout_ns=200_000_000,
                                                                    engine="level"))
    with pytest.raises(mc.MCError) as e:
        mc.mc_batch_run(b, [("min_time", None)])
    assert e.value.code == mc.MC_ERR_TIMEOUT
    ok = mc.mc_batch_create([W.c1(W.FREE)])
    assert mc.mc_batch_run(ok, [("min_time", None)])[0]["time"] == 80
