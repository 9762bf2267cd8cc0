"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Integer work: every count, level width, threshold decision, minimal time,
configuration and witness state must be bit-exact.  The parent chain of a
trace is chosen by racing inserts, so traces are checked by replay
(tests/replay.py) rather than compared.
"""
import json
import os

import pytest

import closed_forms as CF
import replay as RP
from paper_2305_09130_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FREE, GREEDY = W.FREE, W.GREEDY
NO_LIMIT = (1 << 64) - 1
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_expected.json")


def make(mc, spec, **opts):
    m = mc.mc_model_create(spec, mc.mc_options_default(**opts))
    return m


def gpu_check(mc, model, T, prune=True, early_exit=True, trace=True):
    mc.mc_set_options(model, mc.mc_options_default(prune=prune, early_exit=early_exit))
    r = mc.mc_check(model, T, trace=trace)
    lay = mc.mc_model_layout(model)
    out = {"holds": r["holds"], "states": r["states"], "levels": r["levels"]}
    if not r["holds"]:
        i, j, n = RP.decode(lay, r["cex_key"])
        assert (i - 1, j - 1) == (r["cex_i"], r["cex_j"])
        out.update(cex_time=r["cex_time"], cex_i=r["cex_i"], cex_j=r["cex_j"],
                   cex_level=r["cex_level"], cex_n=n)
        if trace:
            keys = r["trace"]
            assert len(keys) == r["cex_level"] + 1
            assert keys[-1] == r["cex_key"]
            t, ti, tj, tn = RP.replay(model.spec, lay, keys, lambda t: t <= T)
            assert (t, ti, tj, tn) == (r["cex_time"], r["cex_i"], r["cex_j"], n)
    return out


def gpu_min(mc, model, search, prune, seed=2305091300, walks=1, refine=True, **opts):
    mc.mc_set_options(model, mc.mc_options_default(prune=prune, search=search, sim_seed=seed,
                                                   sim_walks=walks, refine=refine, **opts))
    r = mc.mc_min_time(model)
    lay = mc.mc_model_layout(model)
    i, j, n = RP.decode(lay, r["witness_key"])
    assert (i - 1, j - 1) == (r["i"], r["j"])
    keys = r["trace"]
    assert keys[-1] == r["witness_key"] and len(keys) == r["level"] + 1
    RP.replay(model.spec, lay, keys, lambda t: t == r["t_min"])
    return {"t_min": r["t_min"], "t_ini": r["t_ini"], "states": r["states"], "checks": r["checks"],
            "i": r["i"], "j": r["j"], "level": r["level"], "n": n}


ENGINES = ["level", "config"]


def thresholds(oracle, spec):
    t_min = oracle.min_time(spec)["t_min"]
    return sorted({0, 1, t_min - 1, t_min, t_min + 1, 2 * t_min, 5 * t_min, NO_LIMIT})


# ---------------------------------------------------------------- small exact parity

@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("name,rule", [("tiny", FREE), ("tiny", GREEDY), ("c1", FREE), ("c1", GREEDY)])
def test_checks_match_oracle(mc, oracle, name, rule, engine):
    spec = W.NAMED[name](rule)
    model = make(mc, spec, engine=engine)
    assert mc.mc_count_states(model) == oracle.count(spec) == CF.count(spec)
    assert mc.mc_last_widths(model) == CF.widths(spec)
    for T in thresholds(oracle, spec):
        for prune in (False, True):
            for ee in (False, True):
                got = gpu_check(mc, model, T, prune, ee)
                exp = oracle.check(spec, T, prune=prune, early_exit=ee)
                assert got == exp, (T, prune, ee)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("name,rule", [("tiny", FREE), ("tiny", GREEDY), ("c1", FREE), ("c1", GREEDY)])
def test_min_time_matches_oracle(mc, oracle, name, rule, engine):
    spec = W.NAMED[name](rule)
    model = make(mc, spec, engine=engine)
    for search in ("single", "lower", "bisect"):
        for prune in (False, True):
            got = gpu_min(mc, model, search, prune)
            exp = oracle.min_time(spec, search=search, prune=prune)
            assert got == exp, (search, prune)


def sweep_models():
    out = []
    seed = 9000
    shapes = [(1, 3, 2, 12), (2, 2, 3, 9), (3, 3, 2, 7), (4, 2, 2, 6), (5, 2, 2, 5), (6, 2, 1, 4),
              (7, 1, 2, 4), (8, 2, 2, 3), (9, 1, 1, 3), (12, 1, 2, 2), (16, 2, 1, 2), (16, 1, 1, 3)]
    for P, a, b, n_max in shapes:
        for rule in (FREE, GREEDY):
            for key_bits in (0, 128):
                out.append(W.random_small(seed, P, a, b, n_max, cost_max=7, speed_max=3, rule=rule,
                                          key_bits=key_bits))
                seed += 1
    return out


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("spec", sweep_models(), ids=lambda s: f"P{s.P}_r{s.rule}_k{s.key_bits}_{s.meta['seed']}")
def test_random_models_match_oracle(mc, oracle, spec, engine):
    model = make(mc, spec, engine=engine)
    assert mc.mc_model_layout(model)["engine"] == mc.ENGINE[engine]
    assert mc.mc_model_layout(model)["key_bits"] == (spec.key_bits or 64)
    assert mc.mc_count_states(model) == oracle.count(spec) == CF.count(spec)
    assert mc.mc_last_widths(model) == CF.widths(spec)
    t_min = oracle.min_time(spec)["t_min"]
    for T in (t_min - 1, t_min, t_min + 3, 3 * t_min):
        for prune, ee in ((True, True), (False, False), (True, False)):
            assert gpu_check(mc, model, T, prune, ee) == oracle.check(spec, T, prune=prune, early_exit=ee)
    for search in ("single", "lower", "bisect"):
        assert gpu_min(mc, model, search, True) == oracle.min_time(spec, search=search, prune=True)


def test_simulation_matches_oracle(mc, oracle):
    for spec in (W.c1(FREE), W.c1(GREEDY), W.c2(rule=GREEDY), W.c3(rule=GREEDY), W.tiny(GREEDY)):
        model = make(mc, spec)
        for seed in (0, 1, 2305091300, 123456789):
            for walks in (1, 7, 1000):
                assert mc.mc_simulate(model, seed, walks) == oracle.simulate(spec, seed, walks)


def test_library_allocator_create_query_destroy_cycles(mc, oracle):
    """The library's own device pool and pooled pinned staging: many models
    made, queried and destroyed in a row (buffers reused across them), with
    models on the PyTorch allocator in between, all give the oracle's answers."""
    exp = oracle.min_time(W.c1(FREE))
    exp_g = oracle.min_time(W.c1(GREEDY))
    for k in range(24):
        spec = W.c1(FREE) if k % 2 == 0 else W.c1(GREEDY)
        want = exp if k % 2 == 0 else exp_g
        m = mc.mc_model_create(spec, allocator=None if k % 3 else "torch")
        r = mc.mc_min_time(m, trace=(k % 4 == 0))
        assert (r["t_min"], r["i"], r["j"], r["states"]) == (want["t_min"], want["i"], want["j"], want["states"])
        mc.mc_model_destroy(m)
        if k == 12:
            mc.mc_release_cached()  # the next models allocate afresh


def test_key_width_does_not_change_results(mc):
    spec = W.c1(FREE)
    a = make(mc, spec)
    b = make(mc, spec.with_key_bits(128))
    assert mc.mc_model_layout(b)["key_words"] == 2
    for T in (60, 79, 80, 200):
        ra, rb = mc.mc_check(a, T, trace=False), mc.mc_check(b, T, trace=False)
        ra.pop("cex_key", None)
        rb.pop("cex_key", None)
        assert ra == rb
    assert mc.mc_min_time(a, trace=False)["t_min"] == mc.mc_min_time(b, trace=False)["t_min"]


# ---------------------------------------------------------------- named workloads at full size

def golden():
    with open(GOLDEN) as f:
        return json.load(f)


@pytest.mark.parametrize("engine", ENGINES)
def test_c2_literal_greedy(mc, oracle, engine):
    spec = W.c2(rule=GREEDY)
    g = golden()["c2_greedy"]
    model = make(mc, spec, engine=engine)
    assert mc.mc_count_states(model) == g["count"] == CF.count(spec)
    assert mc.mc_last_widths(model) == CF.widths(spec)
    for key, exp in g["min_time"].items():
        search, prune = key.split("/prune")
        got = gpu_min(mc, model, search, bool(int(prune)))
        assert got == {k: exp[k] for k in got}, key
    t_min = g["min_time"]["single/prune1"]["t_min"]
    for T in (t_min - 1, t_min):
        assert gpu_check(mc, model, T) == oracle.check(spec, T)


@pytest.mark.parametrize("engine", ENGINES)
def test_c3_literal_greedy_u128(mc, oracle, engine):
    spec = W.c3(rule=GREEDY)
    g = golden()["c3_greedy"]
    model = make(mc, spec, engine=engine)
    assert mc.mc_model_layout(model)["key_words"] == 2
    assert mc.mc_count_states(model) == g["count"] == CF.count(spec)
    got = gpu_min(mc, model, "single", True)
    exp = g["min_time"]["single/prune1"]
    assert got == {k: exp[k] for k in got}
    assert got["t_min"] == CF.tmin(spec)[0]


@pytest.mark.parametrize("load_factor_pct", [25, 15, 10])
def test_c2_star_full(mc, load_factor_pct):
    """C2 at G=80 at full size; load factors of 10% and 15% are the visited-set
    sizes the benchmark's inline tuner picks (the bench's launch configuration)."""
    spec = W.c2_star()
    g = golden()["c2_star"]
    model = make(mc, spec, load_factor_pct=load_factor_pct)
    assert mc.mc_count_states(model) == 10_385_335 == g["count"]
    assert mc.mc_last_widths(model) == CF.widths(spec)
    t_min, argmins = CF.tmin(spec)
    for key, exp in g["min_time"].items():
        search, prune = key.split("/prune")
        got = gpu_min(mc, model, search, bool(int(prune)))
        assert got == {k: exp[k] for k in got}, key
        assert got["t_min"] == t_min and (got["i"], got["j"]) in argmins


@pytest.mark.parametrize("opts", [{}, {"load_factor_pct": 15, "stage_chunk": 192, "probe_scheme": 3}],
                         ids=["defaults", "bench_tuned"])
def test_c3_star_full(mc, opts):
    """1,072,924,481 states with 128-bit keys, with the library's defaults and
    in the configuration the bench's tuner picks (CAS-first insert, chunk 192,
    load factor 15%), then the bench's own query: lowering without pruning."""
    spec = W.c3_star()
    model = make(mc, spec, **opts)
    lay = mc.mc_model_layout(model)
    assert lay["key_words"] == 2 and lay["max_width"] == 193_344_684
    assert mc.mc_count_states(model) == 1_072_924_481 == CF.count(spec)
    assert mc.mc_last_widths(model) == CF.widths(spec)
    t_min, argmins = CF.tmin(spec)
    got = gpu_min(mc, model, "single", True, **opts)
    assert got["t_min"] == t_min
    # the witness comes from the first BFS level holding a T_min terminal:
    # the optimal configurations with the fewest work-groups
    n_of = lambda ij: spec.n_workgroups[ij[0] * spec.b + ij[1]]
    first = min(n_of(ij) for ij in argmins)
    assert (got["i"], got["j"]) == min(ij for ij in argmins if n_of(ij) == first)
    assert got["level"] == first + 2
    # the check at T_ini stops at its first violating level (551 states), the
    # check at T_min - 1 = 0 holds and explores every state
    low = gpu_min(mc, model, "lower", False, **opts)
    assert (low["t_min"], low["i"], low["j"], low["level"]) == (t_min, got["i"], got["j"], got["level"])
    assert low["checks"] == 2 and low["states"] == 1_072_925_032


def warp_eligible_models():
    out = [W.tiny(GREEDY), W.c1(GREEDY), W.c2(G=256, rule=GREEDY)]
    out += [s for s in sweep_models() if s.rule == GREEDY and s.P <= 4]
    # at the boundary: FREE models with P=2 whose widest configuration level
    # holds exactly 16 states (16 x 2 lanes fill the warp), one unit, three
    # units under GREEDY, four FREE units with 4 states
    out += [W.random_small(9505, 2, 2, 3, 16), W.random_small(9506, 2, 2, 3, 16, key_bits=128),
            W.random_small(9500, 1, 2, 3, 30), W.random_small(9500, 3, 2, 3, 5, rule=GREEDY),
            W.random_small(9528, 4, 2, 3, 2)]
    return out


def test_a_level_one_state_wider_than_a_warp_takes_a_block(mc, oracle):
    """17 states of 2 lanes: block units; the same answers as the oracle."""
    spec = W.random_small(9502, 2, 2, 3, 16)
    model = make(mc, spec, engine="config")
    mc.mc_reserve(model)
    lay = mc.mc_model_layout(model)
    assert lay["unit_width"] == 17 and lay["unit_threads"] == 64
    assert mc.mc_count_states(model) == oracle.count(spec)
    assert gpu_min(mc, model, "single", True) == oracle.min_time(spec, search="single", prune=True)


@pytest.mark.parametrize("spec", warp_eligible_models(), ids=lambda s: f"{s.name}_P{s.P}_k{s.key_bits}")
def test_warp_and_block_units_match_oracle(mc, oracle, spec):
    """Models whose widest configuration level fits a warp run one warp per
    configuration by default and one block per configuration when the
    block's threads are given; both give the oracle's counts, widths,
    checks (witness and trace included) and minima."""
    exp_count, exp_widths = oracle.count(spec), CF.widths(spec)
    t_min = oracle.min_time(spec)["t_min"]
    for threads in (0, 64):
        model = make(mc, spec, engine="config", unit_threads=threads)
        mc.mc_reserve(model)
        lay = mc.mc_model_layout(model)
        assert lay["engine"] == mc.ENGINE["config"]
        assert lay["unit_threads"] == (32 if threads == 0 else 64), spec.name
        assert mc.mc_count_states(model) == exp_count
        assert mc.mc_last_widths(model) == exp_widths
        for T in (t_min - 1, t_min, 2 * t_min):
            for prune, ee in ((True, True), (False, False), (True, False)):
                assert gpu_check(mc, model, T, prune, ee) == oracle.check(spec, T, prune=prune, early_exit=ee)
        for search in ("single", "lower"):
            assert gpu_min(mc, model, search, True) == oracle.min_time(spec, search=search, prune=True)


# ---------------------------------------------------------------- edge cases and errors

@pytest.mark.parametrize("engine", ENGINES)
def test_degenerate_models(mc, oracle, engine):
    cases = [
        W.ModelSpec("one", 1, [1], [1], [1], [1], [1]),
        W.ModelSpec("one_g", 1, [1], [1], [1], [1], [1], GREEDY),
        W.ModelSpec("p16", 16, [1, 2], [1], [3, 1], [2, 5], list(range(1, 17))),
        W.ModelSpec("p16g", 16, [1, 2], [1], [20, 1], [2, 5], [1] * 16, GREEDY),
        W.ModelSpec("wide_ab", 2, list(range(1, 41)), list(range(1, 31)),
                    [1 + (k % 3) for k in range(1200)], [1 + (k % 5) for k in range(1200)], [1, 2]),
    ]
    for spec in cases:
        if engine == "config" and mc.mc_model_layout(make(mc, spec))["engine"] != mc.ENGINE["config"]:
            # p16g: one configuration's GREEDY level can hold C(16, 8) states,
            # beyond a block's shared memory; forcing the engine is refused
            with pytest.raises(mc.MCError) as e:
                mc.mc_reserve(make(mc, spec, engine=engine))
            assert e.value.code == mc.MC_ERR_INVAL and spec.name == "p16g"
            continue
        model = make(mc, spec, engine=engine)
        assert mc.mc_count_states(model) == oracle.count(spec) == CF.count(spec), spec.name
        for T in (0, 1, 3, NO_LIMIT):
            assert gpu_check(mc, model, T) == oracle.check(spec, T), (spec.name, T)
        assert gpu_min(mc, model, "single", True) == oracle.min_time(spec), spec.name


@pytest.mark.parametrize("engine", ENGINES)
def test_threshold_zero_keeps_only_selects(mc, engine):
    spec = W.c1(FREE)
    model = make(mc, spec, engine=engine)
    r = gpu_check(mc, model, 0, prune=True, early_exit=True)
    assert r == {"holds": True, "states": 1 + spec.a + spec.a * spec.b, "levels": 3}


@pytest.mark.parametrize("key_bits", [0, 128])
@pytest.mark.parametrize("scheme", ["split", "one_call", "cas_first", "cas_clear"])
def test_table_full_is_reported(mc, scheme, key_bits):
    """A visited set of 8 slots with a 2-bucket probe limit fills at once with
    every insert; the next query on the same model reports it again."""
    model = make(mc, W.c1(FREE).with_key_bits(key_bits) if key_bits else W.c1(FREE), table_log2=3,
                 max_probes=2, engine="level", probe_scheme=scheme)
    for _ in range(2):
        with pytest.raises(mc.MCError) as e:
            mc.mc_count_states(model)
        assert e.value.code == mc.MC_ERR_TABLE_FULL


@pytest.mark.parametrize("scheme", ["split", "cas_first"])
def test_frontier_overflow_is_reported(mc, scheme):
    model = make(mc, W.c1(FREE), log_capacity=100, engine="level", probe_scheme=scheme)
    with pytest.raises(mc.MCError) as e:
        mc.mc_count_states(model)
    assert e.value.code == mc.MC_ERR_FRONTIER


def test_barrier_timeout_is_reported_and_context_survives(mc):
    # every device-wide wait expects one arrival that never comes: each block
    # gives up after 0.2 s of %globaltimer and the pass returns MC_ERR_TIMEOUT
    model = make(mc, W.c1(FREE), debug_barrier_extra=1, barrier_timeout_ns=200_000_000, engine="level")
    with pytest.raises(mc.MCError) as e:
        mc.mc_count_states(model)
    assert e.value.code == mc.MC_ERR_TIMEOUT
    fresh = make(mc, W.c1(FREE))
    assert mc.mc_count_states(fresh) == 8763


def test_invalid_descriptions_are_rejected(mc):
    bad = W.ModelSpec("bad", 2, [1], [1], [0], [1], [1, 1])
    with pytest.raises(mc.MCError) as e:
        mc.mc_model_create(bad)
    assert e.value.code == mc.MC_ERR_INVAL


def staircase(P, b, rule):
    """Configuration j has N = j+1 work-groups and a cost chosen so that the
    model time falls as N grows: each lowering check stops at a shallower
    level than the minimum, and the search takes many checks."""
    n = [j + 1 for j in range(b)]
    cost = [max(1, 600 // (j + 1) - 7 * j) for j in range(b)]
    return W.ModelSpec(f"staircase_P{P}", P, [1], W.pow2_range(0, b - 1), n, cost, [1] * P, rule)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("P,b", [(1, 12), (2, 10), (3, 9)])
@pytest.mark.parametrize("rule", [FREE, GREEDY])
def test_lowering_chained_over_several_groups(mc, oracle, P, b, rule, engine):
    # the device chains the lowering checks in groups of three over four
    # result slots; up to eight checks here cross two group boundaries, and a
    # group's remaining checks are skipped once one holds
    spec = staircase(P, b, rule)
    model = make(mc, spec, engine=engine)
    for prune in (True, False):
        exp = oracle.min_time(spec, search="lower", prune=prune)
        assert gpu_min(mc, model, "lower", prune) == exp
        st = mc.mc_get_stats(model)
        assert st["explore_launches"] >= exp["checks"]
        mc.mc_reset_stats(model)


# ---------------------------------------------------------------- probe schemes

@pytest.mark.parametrize("load_factor", [25, 90])
@pytest.mark.parametrize("scheme", ["split", "one_call", "cas_first", "cas_clear"])
def test_probe_schemes_match_oracle(mc, oracle, scheme, load_factor):
    """Every insert (mc_options.probe_scheme), forced on 64- and 128-bit keys,
    gives the oracle's counts, widths, checks and minima; at a 90% load
    factor most first slots are taken, so the CAS-first insert's fallback
    (another key, or a key of an earlier level, in the first slot) runs
    often."""
    for spec in sweep_models()[::3]:
        model = make(mc, spec, probe_scheme=scheme, engine="level", load_factor_pct=load_factor)
        mc.mc_reserve(model)  # the scheme is fixed once the buffers exist
        assert mc.mc_model_layout(model)["probe_scheme"] == mc.PROBE[scheme]
        assert mc.mc_count_states(model) == oracle.count(spec)
        assert mc.mc_last_widths(model) == CF.widths(spec)
        t_min = oracle.min_time(spec)["t_min"]
        for T in (t_min - 1, t_min, 3 * t_min):
            for prune, ee in ((True, True), (False, False)):
                assert gpu_check(mc, model, T, prune, ee) == oracle.check(spec, T, prune=prune, early_exit=ee)
        assert mc.mc_model_layout(model)["probe_scheme"] == mc.PROBE[scheme]
        assert gpu_min(mc, model, "single", True) == oracle.min_time(spec, search="single", prune=True)


@pytest.mark.parametrize("scheme", ["split", "one_call", "cas_first", "cas_clear"])
def test_probe_schemes_at_full_size(mc, scheme):
    """C2 at G=80 (64-bit keys) and C3 literal under GREEDY (128-bit keys) with
    each insert forced: the full counts, every level's width and the minimum."""
    g = golden()
    for spec, exp in ((W.c2_star(), g["c2_star"]), (W.c3(rule=GREEDY), g["c3_greedy"])):
        model = make(mc, spec, probe_scheme=scheme, load_factor_pct=10, engine="level")
        mc.mc_reserve(model)
        assert mc.mc_count_states(model) == exp["count"] == CF.count(spec)
        assert mc.mc_last_widths(model) == CF.widths(spec)
        got = gpu_min(mc, model, "single", True)
        want = exp["min_time"]["single/prune1"]
        assert got == {k: want[k] for k in got}


# ---------------------------------------------------------------- tagged frontier log

@pytest.mark.parametrize("spec", [W.ModelSpec("wrap8", 6, [1], [1], [256], [3], [1] * 6, GREEDY),
                                  W.ModelSpec("wrap8w", 10, [1], [1], [1024], [3], [1] * 10, GREEDY)],
                         ids=["u64", "u128"])
def test_tagged_log_survives_tag_wrap(mc, oracle, spec):
    """8 tag bits (56 of 64 key bits used; 112 of 128, two 56-bit words):
    the log's tag counter wraps every 255 passes (the host clears the log
    then); 600 checks on one model all agree with the oracle, and so does a
    min-time query after them."""
    model = make(mc, spec, engine="level")
    assert mc.mc_model_layout(model)["log_tag_bits"] == 8
    exp_min = oracle.min_time(spec)
    t_min = exp_min["t_min"]
    exp = {T: oracle.check(spec, T) for T in (t_min - 1, t_min)}
    for k in range(600):
        T = t_min - 1 + (k & 1)
        assert gpu_check(mc, model, T, trace=(k % 50 == 0)) == exp[T], k
    assert gpu_min(mc, model, "single", True) == exp_min


def test_tagged_and_untagged_logs_agree(mc, oracle):
    """The same models with a tagged log and with mc_options.no_log_tags:
    identical counts, widths, checks and minima."""
    for spec in (W.c1(FREE), W.c1(GREEDY), W.c2(rule=GREEDY), W.c1(FREE).with_key_bits(128),
                 W.c1(GREEDY).with_key_bits(128)):
        a, b = make(mc, spec, engine="level"), make(mc, spec, no_log_tags=1, engine="level")
        mc.mc_reserve(b)  # fixed once the buffers exist
        assert mc.mc_model_layout(a)["log_tag_bits"] > 0 and mc.mc_model_layout(b)["log_tag_bits"] == 0
        assert mc.mc_count_states(a) == mc.mc_count_states(b) == oracle.count(spec)
        assert mc.mc_last_widths(a) == mc.mc_last_widths(b)
        for T in thresholds(oracle, spec):
            assert gpu_check(mc, a, T) == gpu_check(mc, b, T) == oracle.check(spec, T), T
        assert mc.mc_model_layout(b)["log_tag_bits"] == 0
        assert gpu_min(mc, a, "lower", True) == gpu_min(mc, b, "lower", True) == \
            oracle.min_time(spec, search="lower", prune=True)


def test_tagged_log_on_c3_literal(mc, oracle):
    """C3 literal (GREEDY, 111 of 128 key bits, 8 tag bits per word, 4,099
    levels): tagged and untagged logs give the golden count, every level's
    width and the minimum."""
    spec = W.c3(rule=GREEDY)
    g = golden()["c3_greedy"]
    exp = g["min_time"]["single/prune1"]
    for opts in ({}, {"no_log_tags": 1}):
        model = make(mc, spec, engine="level", **opts)
        mc.mc_reserve(model)
        assert mc.mc_model_layout(model)["log_tag_bits"] == (0 if opts else 8)
        assert mc.mc_count_states(model) == g["count"] == CF.count(spec)
        assert mc.mc_last_widths(model) == CF.widths(spec)
        got = gpu_min(mc, model, "single", True)
        assert got == {k: exp[k] for k in got}


def test_models_with_different_shared_memory_interleave(mc, oracle):
    """The configuration kernel's shared-memory limit is a property of the
    function, not of a model: a model whose configuration levels need more
    than 48 KB of shared memory still runs after a smaller model was reserved
    (FREE, P=2, 1000 work-groups: 1001 states per level, 64-bit keys)."""
    big = W.ModelSpec("big_smem", 2, [1, 2], [1], [1000, 500], [1, 2], [1, 2])
    small = W.c1(FREE)
    a = make(mc, big, engine="config")
    mc.mc_reserve(a)
    b = make(mc, small, engine="config")
    mc.mc_reserve(b)
    assert mc.mc_model_layout(a)["unit_width"] == 1001
    assert mc.mc_count_states(a) == oracle.count(big) == CF.count(big)
    assert mc.mc_count_states(b) == 8763
    assert gpu_min(mc, a, "single", True) == oracle.min_time(big)


@pytest.mark.parametrize("engine", ENGINES)
def test_lanes_per_state_and_stage_chunk_match_oracle(mc, oracle, engine):
    """The tuner's knobs change the speed, never the answer: every tile width
    from P (rounded up) to 16 lanes per state on both engines, and the
    staging chunk of the level-synchronous kernel."""
    for spec in sweep_models()[::4]:
        t = 1 << (spec.P - 1).bit_length()
        for lanes in sorted({t, min(16, 2 * t), 16}):
            if lanes < spec.P:
                continue
            for chunk in ((64, 96, 128, 192) if engine == "level" else (0,)):
                model = make(mc, spec, engine=engine, lanes_per_state=lanes, stage_chunk=chunk)
                assert mc.mc_count_states(model) == oracle.count(spec), (spec.name, lanes, chunk)
                assert mc.mc_last_widths(model) == CF.widths(spec)
                assert gpu_min(mc, model, "single", True) == oracle.min_time(spec), (spec.name, lanes, chunk)
