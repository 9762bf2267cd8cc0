"""GPU parity of the processing-element level model against the CPU oracle.

Counts, per-level widths, check results (holds, states, levels, the
counterexample's time, configuration and level) and min-time results must
equal the oracle's exactly; every returned trace must replay, step by step,
through the brute-force transition relation (tests/pe_bruteforce.py) to a FIN
state of time <= T.
"""
import json
import os

import pytest

import pe_bruteforce as PB
from paper_2305_09130_gb300 import pe_workloads as PW
from test_pe_oracle_pins import random_pe, tiny_pe_models

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
NO_LIMIT = (1 << 64) - 1


def gpu_state(layout, key, t):
    """The brute-force tuple of a packed GPU key (t carried by the caller)."""
    d = PB_decode(layout, key)
    if d["level"] == 0:
        return ("s0",)
    if d["level"] == 1:
        return ("wg", d["i"] - 1)
    n = tuple(u[0] for u in d["units"])
    busy = tuple(u[1] for u in d["units"])
    pc = tuple(u[2] for u in d["units"])
    mask = tuple(u[3] for u in d["units"])
    return (d["i"] - 1, d["j"] - 1, n, busy, pc, mask, t)


def PB_decode(layout, key):
    from paper_2305_09130_gb300 import mc
    return mc.decode_pe_key(layout, key)


def replay(spec, layout, trace, T):
    """Every step of the trace is a transition; it ends in FIN at time <= T."""
    M = PB.PeModel(spec)
    assert trace[0] == 0
    cur = ("s0",)
    for lvl, key in enumerate(trace[1:], start=1):
        assert PB_decode(layout, key)["level"] == lvl
        t = PB.PeModel.time(cur)
        want_same = gpu_state(layout, key, t)
        want_tick = gpu_state(layout, key, t + 1)
        nxt = M.successors(cur)
        assert want_same in nxt or want_tick in nxt, (lvl, cur, want_same)
        cur = want_same if want_same in nxt else want_tick
    assert M.is_fin(cur) and PB.PeModel.time(cur) <= T
    return cur


def run_all(mc, oracle, spec, Ts):
    lay = mc.mc_pe_model_layout(mc.mc_pe_model_create(spec, stream=0))
    for prune in (0, 1):
        for ee in (0, 1):
            m = mc.mc_pe_model_create(spec, mc.mc_options_default(prune=prune, early_exit=ee))
            for T in Ts:
                got = mc.mc_pe_check(m, T)
                exp = oracle.pe_check(spec, T, prune, ee)
                tr = got.pop("trace", None)
                for k in ("cex_wg", "cex_ts", "cex_key"):
                    got.pop(k, None)
                assert got == exp, (spec.name, T, prune, ee)
                if not exp["holds"]:
                    end = replay(spec, lay, tr, T)
                    assert (PB.PeModel.time(end), end[0], end[1]) == (exp["cex_time"], exp["cex_i"], exp["cex_j"])
                    assert len(tr) == exp["cex_level"] + 1
            mc.mc_pe_model_destroy(m)


@pytest.mark.parametrize("spec", tiny_pe_models(), ids=lambda s: s.name + f"_P{s.P}")
def test_pe_parity_tiny(mc, oracle, spec):
    m = mc.mc_pe_model_create(spec)
    assert mc.mc_pe_count_states(m) == oracle.pe_count(spec)
    full = oracle.pe_check(spec, NO_LIMIT, False, False, widths=1 << 16)
    assert mc.mc_pe_last_widths(m) == full["widths"]
    times = sorted({t for ts in PB.fin_times(spec).values() for t in ts})
    run_all(mc, oracle, spec, sorted({0, times[0] - 1, times[0], times[-1], times[-1] + 2}))
    r = mc.mc_pe_min_time(m)
    e = oracle.pe_min_time(spec)
    assert {k: r[k] for k in e} == e
    lay = mc.mc_pe_model_layout(m)
    replay(spec, lay, r["trace"], e["t_min"])


@pytest.mark.parametrize("spec", [PW.pe_abstract(8, P=2), PW.pe_minimum(32, P=4, np_=4, gmt=2),
                                  PW.pe_abstract(16, P=2), random_pe(7302, 3, 3, 3, n_max=6, nwe_max=2,
                                                                     segs=8, ticks_max=6)],
                         ids=lambda s: s.name + f"_P{s.P}")
def test_pe_parity_medium(mc, oracle, spec):
    m = mc.mc_pe_model_create(spec)
    full = oracle.pe_check(spec, NO_LIMIT, False, False, widths=1 << 16)
    assert mc.mc_pe_count_states(m) == full["states"]
    assert mc.mc_pe_last_widths(m) == full["widths"]
    e = oracle.pe_min_time(spec)
    r = mc.mc_pe_min_time(m)
    assert {k: r[k] for k in e} == e
    t = e["t_min"]
    run_all(mc, oracle, spec, [t - 1, t, t + 7])


def golden():
    return json.load(open(os.path.join(HERE, "golden", "pe_oracle_expected.json")))


@pytest.mark.parametrize("name,make", [("pe_abstract_s16_P4", lambda: PW.pe_abstract(16, P=4, np_=4, gmt=1)),
                                       ("pe_minimum_s64_P4", lambda: PW.pe_minimum(64, P=4, np_=4, gmt=2))])
def test_pe_parity_full_size(mc, name, make):
    # the 37M-state model needs the frontier log to grow twice from its
    # default 2^22 entries: the growth path runs here
    g = golden()[name]
    spec = make()
    m = mc.mc_pe_model_create(spec)
    assert mc.mc_pe_count_states(m) == g["count"]
    assert mc.mc_pe_last_widths(m, cap=1 << 20) == g["widths"]
    r = mc.mc_pe_min_time(m)
    assert {k: r[k] for k in g["min_time"]} == g["min_time"]
    lay = mc.mc_pe_model_layout(m)
    replay(spec, lay, r["trace"], g["min_time"]["t_min"])


def test_pe_explicit_small_log_reports_frontier(mc):
    spec = PW.pe_abstract(8, P=2)
    m = mc.mc_pe_model_create(spec, mc.mc_options_default(log_capacity=1000))
    with pytest.raises(mc.MCError) as e:
        mc.mc_pe_count_states(m)
    assert e.value.code == mc.MC_ERR_FRONTIER
    m2 = mc.mc_pe_model_create(spec)
    assert mc.mc_pe_count_states(m2) == 24301


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_pe_every_tile_width_agrees(mc, oracle, tile):
    for spec in (PW.pe_abstract(8, P=2), PW.pe_minimum(32, P=4, np_=4, gmt=2), tiny_pe_models()[3]):
        lanes = spec.P * max(spec.pes) + spec.P + 1
        if -(-lanes // tile) > (1 if tile == 32 else 2 if tile == 16 else 3):
            continue
        m = mc.mc_pe_model_create(spec, mc.mc_options_default(lanes_per_state=tile))
        assert mc.mc_pe_model_layout(m)["tile"] == tile
        assert mc.mc_pe_count_states(m) == oracle.pe_count(spec)
        r = mc.mc_pe_min_time(m)
        e = oracle.pe_min_time(spec)
        assert {k: r[k] for k in e} == e


def test_pe_autotune_keeps_the_answer(mc, tmp_path):
    from paper_2305_09130_gb300 import autotune as AT
    spec = PW.pe_abstract(8, P=2)
    out = AT.tune_pe(spec, space={"lanes_per_state": [8, 16, 32], "blocks_per_sm": [0, 2]}, reps=1,
                     path=str(tmp_path / "cache.json"))
    assert out["options"]["lanes_per_state"] in (8, 16, 32) and len(out["timings"]) >= 4
