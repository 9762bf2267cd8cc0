"""Pins of the CPU oracle against brute force, closed forms and invariants.

Each check here fixes the oracle to something other than itself: the tree of
every schedule (tests/bruteforce.py), counting formulas (tests/closed_forms.py),
hand-derived worked values, and the logical properties of the method
(Section 2: C_ex(T_min) is true and C_ex(T_min - 1) is false; the check is
monotone in T; the reachable count does not depend on search order).
"""
import itertools

import pytest

import bruteforce as BF
import closed_forms as CF
from paper_2305_09130_gb300 import workloads as W

FREE, GREEDY = W.FREE, W.GREEDY


def tiny_models():
    out = []
    seed = 1000
    for P in (1, 2, 3):
        for rule in (FREE, GREEDY):
            for a, b in ((1, 1), (2, 1), (1, 2), (2, 2)):
                n_max = {1: 6, 2: 5, 3: 4}[P]
                out.append(W.random_small(seed, P, a, b, n_max, cost_max=5, speed_max=3, rule=rule))
                seed += 1
    return out


# ---------------------------------------------------------------- worked values

def test_c1_worked_values(oracle):
    # G=64, P=2, WG in {1,2,4,8,16} -> N = 64, 32, 16, 8, 4; TS in {1,2,4}.
    # FREE: 1 + 5 + 3 * (C(66,2) + C(34,2) + C(18,2) + C(10,2) + C(6,2))
    #     = 6 + 3 * (2145 + 561 + 153 + 45 + 15) = 8763.
    assert oracle.count(W.c1(FREE)) == 8763
    # GREEDY, equal speeds: each level k holds C(2, k mod 2) states, so a
    # configuration with even N has 3N/2 + 1 states: 97+49+25+13+7 = 191;
    # 1 + 5 + 3 * 191 = 579.
    assert oracle.count(W.c1(GREEDY)) == 579
    # WG=16, TS=4: cost = ceil(16/4)*4 + 16 + 2*4 = 40, N = 4, two units take
    # two each: 80.  WG=8, TS=4: cost = 24, N = 8 -> 96 (the next best).
    for rule in (FREE, GREEDY):
        r = oracle.min_time(W.c1(rule))
        assert (r["t_min"], r["i"], r["j"], r["n"]) == (80, 4, 2, [2, 2])
        assert oracle.check(W.c1(rule), 79)["holds"]
        c = oracle.check(W.c1(rule), 80)
        assert not c["holds"] and (c["cex_time"], c["cex_i"], c["cex_j"]) == (80, 4, 2)
    per = {cfg: CF.free_tmin_cfg(W.c1(), cfg) for cfg in range(15)}
    assert sorted(per.values())[:2] == [80, 96]
    assert [k for k, v in per.items() if v == 96] == [3 * 3 + 2]


def test_tiny_worked_values(oracle):
    # G=8, P=2, WG {1,2}, TS {1,2}, speeds (1,3): N = 8, 4; FREE count
    # 1 + 2 + 2 * (C(10,2) + C(6,2)) = 123.  WG=2, TS=2: cost 10, unit times
    # (10, 30); the 4th smallest of {10,20,30,40,..} U {30,60,..} is 30.
    spec = W.tiny(FREE)
    assert oracle.count(spec) == 123
    assert oracle.count(W.tiny(GREEDY)) == 37
    for rule in (FREE, GREEDY):
        r = oracle.min_time(W.tiny(rule))
        assert (r["t_min"], r["i"], r["j"]) == (30, 1, 1)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("spec", tiny_models(), ids=lambda s: f"{s.name}_P{s.P}_r{s.rule}_{s.a}x{s.b}")
def test_oracle_matches_bruteforce(oracle, spec):
    levels, terminals = BF.enumerate_model(spec)
    assert oracle.count(spec) == len(levels)
    times = sorted(set(terminals.values()))
    probe_T = sorted({0, times[0] - 1, times[0], times[-1], times[-1] + 1}
                     | set(times[:: max(1, len(times) // 4)]))
    for T, prune, ee in itertools.product(probe_T, (False, True), (False, True)):
        if T < 0:
            continue
        got = oracle.check(spec, T, prune=prune, early_exit=ee)
        exp = BF.brute_check(spec, T, prune=prune, early_exit=ee)
        assert got == exp, (T, prune, ee)


@pytest.mark.parametrize("spec", tiny_models()[:12], ids=lambda s: f"{s.name}_P{s.P}_r{s.rule}")
def test_oracle_tmin_matches_all_schedules(oracle, spec):
    sched = BF.schedules(spec)
    best = min(t for _i, _j, t in sched)
    for search in ("single", "lower", "bisect"):
        for prune in (False, True):
            r = oracle.min_time(spec, search=search, prune=prune)
            assert r["t_min"] == best
            # Step 4: the configuration is that of the counterexample at T_min
            c = BF.brute_check(spec, best, prune=prune, early_exit=True)
            assert (r["i"], r["j"], r["n"]) == (c["cex_i"], c["cex_j"], c["cex_n"])
            assert r["t_ini"] >= best


# ---------------------------------------------------------------- closed forms

def medium_models():
    out = []
    seed = 5000
    for P in (1, 2, 3, 4, 5):
        for rule in (FREE, GREEDY):
            out.append(W.random_small(seed, P, 3, 2, {1: 40, 2: 20, 3: 12, 4: 8, 5: 6}[P],
                                      cost_max=9, speed_max=4, rule=rule))
            seed += 1
    return out


@pytest.mark.parametrize("spec", medium_models(), ids=lambda s: f"{s.name}_P{s.P}_r{s.rule}")
def test_oracle_counts_match_closed_form(oracle, spec):
    r = oracle.check(spec, (1 << 64) - 1, prune=False, early_exit=False, widths=512)
    assert r["states"] == CF.count(spec)
    assert r["widths"] == CF.widths(spec)


@pytest.mark.parametrize("spec", medium_models(), ids=lambda s: f"{s.name}_P{s.P}_r{s.rule}")
def test_oracle_tmin_matches_closed_form(oracle, spec):
    t_min, argmins = CF.tmin(spec)
    r = oracle.min_time(spec)
    assert r["t_min"] == t_min
    assert (r["i"], r["j"]) in argmins


def test_named_workload_counts(oracle):
    assert oracle.count(W.c2(rule=GREEDY)) == CF.count(W.c2(rule=GREEDY))
    assert CF.count(W.c2_star()) == 10_385_335
    assert CF.count(W.c3_star()) == 1_072_924_481
    assert max(CF.free_widths(W.c3_star())) == 193_344_684


# ---------------------------------------------------------------- invariants

@pytest.mark.parametrize("spec", medium_models()[:6], ids=lambda s: f"{s.name}_P{s.P}_r{s.rule}")
def test_check_is_monotone_and_brackets_tmin(oracle, spec):
    t_min = oracle.min_time(spec)["t_min"]
    prev = True
    for T in range(max(0, t_min - 6), t_min + 12):
        h = oracle.check(spec, T)["holds"]
        assert h == (T < t_min)
        assert prev or not h
        prev = h


def test_pruned_counts_are_subsets(oracle):
    spec = medium_models()[4]
    full = oracle.check(spec, (1 << 64) - 1, prune=False, early_exit=False)["states"]
    last = 0
    for T in (5, 10, 20, 40, 80, 160, 1 << 40):
        r = oracle.check(spec, T, prune=True, early_exit=False)
        assert last <= r["states"] <= full
        last = r["states"]
    assert last == full


def test_simulation_draws_its_configuration(oracle):
    # counter-based splitmix64: the first two draws of walk 0 pick (i, j)
    for spec in tiny_models()[:10]:
        seed = 77
        i = W.splitmix64_mix(seed + 1 * W.SPLITMIX_GAMMA) % spec.a
        j = W.splitmix64_mix(seed + 2 * W.SPLITMIX_GAMMA) % spec.b
        t_ini = oracle.simulate(spec, seed, 1)
        times = {t for ii, jj, t in BF.schedules(spec) if (ii, jj) == (i, j)}
        assert t_ini in times
        # many walks reach the optimum of a tiny model
        best = min(t for _i, _j, t in BF.schedules(spec))
        assert oracle.simulate(spec, seed, 4000) == best


def test_swarm_runs_are_schedules_and_never_beat_tmin(oracle):
    # every swarm run is a complete schedule of its configuration, so its
    # time is one of the brute-force terminal times and never below T_min
    for spec in tiny_models()[:8]:
        sched = BF.schedules(spec)
        best = min(t for _i, _j, t in sched)
        for w in range(40):
            t, i, j = oracle.walk(spec, 99, w)
            assert t in {tt for ii, jj, tt in sched if (ii, jj) == (i, j)}
        sw = oracle.swarm(spec, 99, 64, 30)
        assert sw["best_time"] >= best and sw["first_time"] >= sw["best_time"]
        # many runs per round reach the optimum of a tiny model
        assert oracle.swarm(spec, 99, 4000, 30)["best_time"] == best


# ---------------------------------------------------------------- swarm rounds, worked by hand
# Models with one compute unit and one work-group per configuration: every
# random run of configuration i then ends at time cost[i], whatever its
# dispatch draws, so a swarm's rounds depend only on the configuration each
# run draws -- splitmix64 output number (w << 32) of the seed, modulo a
# (Section 4, Step 3's simulation; Section 5 runs many of them).  The draws
# come from the published generator in the input module; the expected best
# times, walks and round counts below are worked out from the search rule of
# Section 5 (round 0 takes the least time of its runs; round r >= 1 takes
# fresh runs r*W .. (r+1)*W - 1 and keeps one that ends at or below the best
# time minus one; the search stops after the first round that finds none).
def _one_unit_model(costs):
    return W.ModelSpec("swarm_pin", 1, [1 << i for i in range(len(costs))], [1], [1] * len(costs),
                       list(costs), [1], W.FREE)


def _drawn_config(seed, w, a):
    return W.splitmix64_mix(seed + ((w << 32) + 1) * W.SPLITMIX_GAMMA) % a


def _seed_where(pred, a, walks):
    for seed in range(1, 100000):
        if pred([_drawn_config(seed, w, a) for w in range(walks)]):
            return seed
    raise AssertionError("no seed found")


def test_swarm_stops_after_the_round_that_finds_nothing(oracle):
    # times 10, 20, 30 and 64 runs per round: round 0 draws every
    # configuration, finds 10 at its first run of configuration 0; round 1
    # looks for a time <= 9, finds none, and ends the search: two rounds
    spec = _one_unit_model([10, 20, 30])
    seed = _seed_where(lambda d: set(d[:64]) == {0, 1, 2}, 3, 64)
    first0 = [_drawn_config(seed, w, 3) for w in range(64)].index(0)
    sw = oracle.swarm(spec, seed, 64, 30)
    assert (sw["rounds"], sw["first_time"], sw["best_time"], sw["best_walk"]) == (2, 10, 10, first0)
    assert sw["walks"] == 128 and (sw["i"], sw["j"]) == (0, 0)


def test_swarm_improves_in_a_later_round_at_best_minus_one(oracle):
    # times 19 and 20, 4 runs per round, a seed whose round 0 draws only
    # configuration 1 and whose round 1 (runs 4..7, fresh) draws
    # configuration 0: round 0 finds 20, round 1 finds 19 = 20 - 1 (a run
    # ending exactly at best - 1 counts), round 2 finds nothing: three rounds.
    # A strict bound, runs reused across rounds or a late stop all fail here.
    spec = _one_unit_model([19, 20])
    seed = _seed_where(lambda d: d[:4] == [1, 1, 1, 1] and 0 in d[4:8], 2, 8)
    d = [_drawn_config(seed, w, 2) for w in range(8)]
    k = d[4:8].index(0)
    sw = oracle.swarm(spec, seed, 4, 30)
    assert (sw["rounds"], sw["first_time"], sw["best_time"], sw["best_walk"]) == (3, 20, 19, 4 + k)
    assert sw["walks"] == 12 and sw["i"] == 0
    # the round limit ends the search early with the same best
    sw2 = oracle.swarm(spec, seed, 4, 2)
    assert (sw2["rounds"], sw2["best_time"], sw2["best_walk"]) == (2, 19, 4 + k)
    sw1 = oracle.swarm(spec, seed, 4, 1)
    assert (sw1["rounds"], sw1["best_time"], sw1["best_walk"]) == (1, 20, 0)


def test_swarm_keeps_its_first_trail_when_the_next_round_misses(oracle):
    # times 19 and 20, a seed whose runs 0..7 all draw configuration 1:
    # round 0 finds 20 at run 0, round 1 (configuration 1 again, 20 > 19)
    # finds nothing: two rounds and the first trail is the answer, a miss
    # of the optimum the swarm cannot detect (optimality is not proven)
    spec = _one_unit_model([19, 20])
    seed = _seed_where(lambda d: d == [1] * 8, 2, 8)
    sw = oracle.swarm(spec, seed, 4, 30)
    assert (sw["rounds"], sw["first_time"], sw["best_time"], sw["best_walk"]) == (2, 20, 20, 0)
    assert sw["i"] == 1
