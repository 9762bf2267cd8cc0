"""Pins of the processing-element level oracle (oracle/oracle_pe.cpp).

Each check fixes the oracle to something other than itself: a separate
brute-force enumeration in Python (tests/pe_bruteforce.py), closed forms of
the model's clock, the count of a one-unit model, the reduction of a model
without PE interleavings to the cost-table GREEDY model, and the first row
of Table 1.
"""
import json
import os

import pytest

import pe_bruteforce as PB
from paper_2305_09130_gb300 import pe_workloads as PW
from paper_2305_09130_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def random_pe(seed, P, a, b, n_max=3, nwe_max=3, segs=4, ticks_max=3):
    rng = W.SplitMix64(seed)
    n, pes, progs = [], [], []
    for _ in range(a * b):
        n.append(rng.uniform(1, n_max))
        nwe = rng.uniform(1, nwe_max)
        pes.append(nwe)
        prog = []
        for _s in range(rng.uniform(1, segs)):
            prog.append((rng.uniform(0, ticks_max), rng.uniform(1, nwe)))
        if all(t == 0 for t, _m in prog):
            prog.append((1, nwe))
        progs.append(prog)
    return PW.PeSpec(f"pe_rand_{seed}", P, W.pow2_range(0, a - 1), W.pow2_range(0, b - 1), n, pes, progs,
                     {"seed": seed})


def tiny_pe_models():
    out = [PW.table1_row1(), PW.pe_minimum(16, P=2, np_=2, gmt=1)]
    seed = 7000
    for P in (1, 2, 3):
        for a, b in ((1, 1), (2, 1), (1, 2), (2, 2)):
            out.append(random_pe(seed, P, a, b, n_max=3 if P < 3 else 2, nwe_max=3 if P < 3 else 2))
            seed += 1
    return out


def tau(prog):
    return sum(t for t, _m in prog)


def tmin_closed(spec):
    """The clock of the PE model is lock-step: every work-group takes tau
    ticks and the units take them in waves, so FIN comes at
    tau * ceil(N / P) -- the same for every schedule of a configuration."""
    best = None
    for i in range(spec.a):
        for j in range(spec.b):
            k = i * spec.b + j
            t = tau(spec.programs[k]) * -(-spec.n_workgroups[k] // spec.P)
            best = min(best, (t, i, j)) if best else (t, i, j)
    return best


@pytest.mark.parametrize("spec", tiny_pe_models(), ids=lambda s: s.name + f"_P{s.P}")
def test_pe_oracle_matches_bruteforce(oracle, spec):
    levels = PB.enumerate_levels(spec)  # also asserts the graph is layered
    assert oracle.pe_count(spec) == sum(len(lv) for lv in levels)
    full = oracle.pe_check(spec, (1 << 64) - 1, prune=False, early_exit=False, widths=100000)
    assert full["widths"] == [len(lv) for lv in levels]
    times = sorted({t for ts in PB.fin_times(spec).values() for t in ts})
    probe_T = sorted({0, times[0] - 1, times[0], times[-1], times[-1] + 1, (times[0] + times[-1]) // 2})
    for T in probe_T:
        if T < 0:
            continue
        for prune in (False, True):
            for ee in (False, True):
                assert oracle.pe_check(spec, T, prune, ee) == PB.brute_check(spec, T, prune, ee), (T, prune, ee)


@pytest.mark.parametrize("spec", tiny_pe_models(), ids=lambda s: s.name + f"_P{s.P}")
def test_pe_fin_times_are_the_lockstep_closed_form(oracle, spec):
    for (i, j), ts in PB.fin_times(spec).items():
        k = i * spec.b + j
        assert ts == {tau(spec.programs[k]) * -(-spec.n_workgroups[k] // spec.P)}
    t, i, j = tmin_closed(spec)
    r = oracle.pe_min_time(spec)
    assert (r["t_min"], r["i"], r["j"]) == (t, i, j)
    assert oracle.pe_check(spec, t - 1)["holds"] and not oracle.pe_check(spec, t)["holds"]


def marks_and_barriers(prog):
    return (sum(t * m if t else m for t, m in prog), sum(1 for t, _m in prog if t == 0))


@pytest.mark.parametrize("spec", tiny_pe_models(), ids=lambda s: s.name + f"_P{s.P}")
def test_pe_fin_level_counts_every_transition(oracle, spec):
    # two selects, per work-group one dispatch plus the marks and releases of
    # its program, plus one step per clock tick
    r = oracle.pe_min_time(spec)
    k = r["i"] * spec.b + r["j"]
    N, prog = spec.n_workgroups[k], spec.programs[k]
    marks, bars = marks_and_barriers(prog)
    assert r["level"] == 2 + N * (1 + marks + bars) + tau(prog) * -(-N // spec.P)


@pytest.mark.parametrize("seed", range(4))
def test_one_unit_count_closed_form(oracle, seed):
    # one unit: per work-group, each program step has 2^pes mark states; the
    # unit is idle N+1 times (after 0..N work-groups)
    spec = random_pe(7100 + seed, 1, 2, 2, n_max=4, nwe_max=4, segs=5)
    total = 1 + spec.a
    for k, prog in enumerate(spec.programs):
        N = spec.n_workgroups[k]
        per_wg = sum((t if t else 1) * (1 << m) for t, m in prog)
        total += (N + 1) + N * per_wg
    assert oracle.pe_count(spec) == total


@pytest.mark.parametrize("seed", range(4))
def test_without_interleavings_the_greedy_cost_model_is_recovered(oracle, seed):
    # one PE per unit and no barrier: the only choice left is which idle unit
    # takes the next work-group, and work-groups last tau ticks on every
    # unit -- the cost-table GREEDY model with cost tau and speed 1
    rng = W.SplitMix64(7200 + seed)
    P, a, b = 1 + seed % 3, 2, 2
    n = [rng.uniform(1, 5) for _ in range(a * b)]
    progs = [[(rng.uniform(1, 6), 1)] for _ in range(a * b)]
    pe = PW.PeSpec("pe_plain", P, [1, 2], [1, 2], n, [1] * (a * b), progs)
    cm = W.ModelSpec("cost_plain", P, [1, 2], [1, 2], n, [tau(p) for p in progs], [1] * P, W.GREEDY)
    r_pe, r_cm = oracle.pe_min_time(pe), oracle.min_time(cm)
    assert (r_pe["t_min"], r_pe["i"], r_pe["j"]) == (r_cm["t_min"], r_cm["i"], r_cm["j"])
    for T in (r_cm["t_min"] - 1, r_cm["t_min"], r_cm["t_min"] + 3):
        assert oracle.pe_check(pe, T)["holds"] == oracle.check(cm, T)["holds"]


def test_table1_first_row(oracle):
    g = json.load(open(os.path.join(HERE, "golden", "table1_row1.json")))
    spec = PW.pe_abstract(g["size"], P=1, np_=4, gmt=g["GMT"])
    r = oracle.pe_min_time(spec)
    assert (r["t_min"], spec.ts_values[r["j"]], spec.wg_values[r["i"]]) == (g["model_time"], g["TS"], g["WG"])


def test_check_is_monotone_in_T(oracle):
    spec = PW.pe_abstract(8, P=2)
    t = oracle.pe_min_time(spec)["t_min"]
    prev = True
    for T in range(t - 5, t + 8):
        h = oracle.pe_check(spec, T)["holds"]
        assert h == (T < t) and (prev or not h)
        prev = h
