"""Host-side checks of the C-ABI library (no GPU needed).

The library must load and export every function include/*.h declares.
Model creation is host-only (validation, key layout, closed-form sizing), so
it is exercised here; any query without a CUDA device must fail loudly.
"""
import os
import re

import pytest

import closed_forms as CF
from paper_2305_09130_gb300 import mc
from paper_2305_09130_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for h in sorted(os.listdir(inc)):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(inc, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(mc_[a-z_]+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return mc.load(build=True)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 19 and "mc_pe_check" in names and "mc_check_noalloc" in names
    for n in names:
        assert hasattr(lib, n), n


def test_options_default(lib):
    o = mc.mc_options_default()
    assert (o.prune, o.early_exit, o.search, o.refine, o.sim_walks, o.load_factor_pct) == (1, 1, 0, 1, 1, 25)
    assert o.sim_seed == 2305091300


def layout(spec, **kw):
    m = mc.mc_model_create(spec, mc.mc_options_default(**kw), allocator=None)
    return mc.mc_model_layout(m)


def test_layout_of_named_workloads(lib):
    l1 = layout(W.c1())
    # i+1 in 3 bits (a=5), j+1 in 2 bits (b=3), n_c in 7 bits (N <= 64), P=2
    assert (l1["wg_bits"], l1["ts_bits"], l1["n_bits"], l1["used_bits"]) == (3, 2, 7, 19)
    assert (l1["key_bits"], l1["n_shift"], l1["ts_shift"], l1["wg_shift"]) == (64, [7, 0], 14, 16)
    assert l1["state_bound"] == 8763 and l1["max_level"] == 66
    l2 = layout(W.c2_star())
    assert l2["used_bits"] == 4 + 3 + 4 * 7 and l2["key_bits"] == 64
    assert l2["state_bound"] == CF.count(W.c2_star()) == 10_385_335
    l3 = layout(W.c3_star())
    assert l3["key_bits"] == 128 and l3["used_bits"] == 4 + 3 + 8 * 6
    assert l3["state_bound"] == 1_072_924_481 and l3["max_width"] == 193_344_684
    assert l3["table_slots"] == 1 << 30 and l3["log_capacity"] == 1_072_924_481
    lit = layout(W.c3(rule=W.GREEDY))
    assert lit["used_bits"] == 4 + 3 + 8 * 13 and lit["key_bits"] == 128
    assert lit["state_bound"] >= CF.count(W.c3(rule=W.GREEDY))


@pytest.mark.parametrize("seed", range(6))
def test_free_bound_is_the_exact_count(lib, seed):
    spec = W.random_small(300 + seed, 1 + seed % 5, 3, 2, 9, rule=W.FREE)
    lay = layout(spec)
    assert lay["state_bound"] == CF.count(spec)
    assert lay["max_width"] == max(CF.widths(spec)[3:])
    g = spec.with_rule(W.GREEDY)
    assert layout(g)["state_bound"] >= CF.count(g)
    assert layout(g)["max_width"] >= max(CF.widths(g)[3:])


def test_invalid_descriptions(lib):
    ok = W.c1()
    cases = [
        (W.ModelSpec("n0", 2, [1], [1], [0], [1], [1, 1]), mc.MC_ERR_INVAL),
        (W.ModelSpec("c0", 2, [1], [1], [1], [0], [1, 1]), mc.MC_ERR_INVAL),
        (W.ModelSpec("s0", 2, [1], [1], [1], [1], [1, 0]), mc.MC_ERR_INVAL),
        (W.ModelSpec("p17", 17, [1], [1], [1], [1], [1] * 17), mc.MC_ERR_INVAL),
        (W.ModelSpec("rule", 2, [1], [1], [1], [1], [1, 1], 2), mc.MC_ERR_INVAL),
        (ok.with_key_bits(32), mc.MC_ERR_INVAL),
        (W.c3(rule=W.GREEDY).with_key_bits(64), mc.MC_ERR_OVERFLOW),
        (W.ModelSpec("clock", 2, [1], [1], [1 << 20], [1 << 19], [2, 1]), mc.MC_ERR_OVERFLOW),
        (W.ModelSpec("wide", 2, list(range(4096)), [1], [1] * 4096, [1] * 4096, [1, 1]), mc.MC_ERR_OVERFLOW),
    ]
    for spec, code in cases:
        with pytest.raises(mc.MCError) as e:
            mc.mc_model_create(spec, allocator=None)
        assert e.value.code == code, spec.name
    with pytest.raises(mc.MCError) as e:
        mc.mc_model_create(ok, mc.mc_options_default(load_factor_pct=95), allocator=None)
    assert e.value.code == mc.MC_ERR_INVAL
    with pytest.raises(mc.MCError) as e:
        mc.mc_model_create(ok, mc.mc_options_default(probe_scheme=5), allocator=None)
    assert e.value.code == mc.MC_ERR_INVAL


def test_probe_schemes_are_accepted_by_name_and_number(lib):
    for name, code in (("auto", 0), ("split", 1), ("one_call", 2), ("cas_first", 3), ("cas_clear", 4)):
        o = mc.mc_options_default(probe_scheme=name)
        assert o.probe_scheme == code == mc.PROBE[name]
        mc.mc_model_create(W.c1(), o, allocator=None)
    # AUTO resolves by key width: split for 64-bit keys, CAS first for 128-bit
    assert layout(W.c1())["probe_scheme"] == mc.PROBE["split"]
    assert layout(W.c1().with_key_bits(128))["probe_scheme"] == mc.PROBE["cas_first"]
    assert layout(W.c1(), probe_scheme="one_call")["probe_scheme"] == mc.PROBE["one_call"]
    assert layout(W.c1().with_key_bits(128), probe_scheme="split")["probe_scheme"] == mc.PROBE["split"]
    for spec in (W.c1(), W.c1().with_key_bits(128)):
        for name in ("cas_first", "cas_clear"):
            assert layout(spec, probe_scheme=name)["probe_scheme"] == mc.PROBE[name]


def test_frontier_log_tags_use_spare_key_bits(lib):
    # the level-synchronous engine: 64-bit keys with at least 8 spare top bits
    # tag their log entries (up to 16 bits)
    lv = {"engine": "level"}
    assert layout(W.c1(), **lv)["log_tag_bits"] == 16                    # 19 bits used
    assert layout(W.c2_star())["log_tag_bits"] == 16                     # 35 bits used
    assert layout(W.c2(rule=W.GREEDY), **lv)["log_tag_bits"] == 13       # 51 bits used
    # 128-bit keys: two words of 64 - t payload bits, t <= (128 - used) / 2
    assert layout(W.c1().with_key_bits(128), **lv)["log_tag_bits"] == 16  # 19 bits used
    assert layout(W.c3(rule=W.GREEDY), **lv)["log_tag_bits"] == 8         # 111 bits used
    wrap8w = W.ModelSpec("wrap8w", 10, [1], [1], [1024], [3], [1] * 10, W.GREEDY)
    assert layout(wrap8w, **lv)["used_bits"] == 112 and layout(wrap8w, **lv)["log_tag_bits"] == 8
    few128 = W.ModelSpec("few128", 10, [1, 2, 4], [1], [1024] * 3, [3] * 3, [1] * 10, W.GREEDY)
    assert layout(few128, **lv)["used_bits"] == 113 and layout(few128, **lv)["log_tag_bits"] == 0
    # a=b=1, P=6, N=256: 1 + 1 + 6 x 9 = 56 bits, 8 spare; N=512: 62 bits, too few
    wrap8 = W.ModelSpec("wrap8", 6, [1], [1], [256], [3], [1] * 6, W.GREEDY)
    assert layout(wrap8, **lv)["used_bits"] == 56 and layout(wrap8, **lv)["log_tag_bits"] == 8
    few = W.ModelSpec("few", 6, [1], [1], [512], [3], [1] * 6, W.GREEDY)
    assert layout(few, **lv)["used_bits"] == 62 and layout(few, **lv)["log_tag_bits"] == 0
    assert layout(W.c1(), no_log_tags=1, **lv)["log_tag_bits"] == 0
    # the configuration engine reads its log only after the pass: untagged
    assert layout(W.c1())["engine"] == mc.ENGINE["config"] and layout(W.c1())["log_tag_bits"] == 0
    with pytest.raises(mc.MCError):
        mc.mc_model_create(W.c1(), mc.mc_options_default(no_log_tags=2), allocator=None)


def test_engine_follows_the_width_of_one_configuration(lib):
    """AUTO takes the configuration engine when one configuration's widest
    level (closed form: C(N+P-1, P-1) under FREE, at most C(P, P/2) under
    GREEDY) fits a block's shared memory: 2048 states with 64-bit keys, 1024
    with 128-bit keys.  Its log holds one segment per configuration, as long
    as that configuration's states can be."""
    from math import comb

    c1 = layout(W.c1())  # FREE, P=2, N <= 64: the widest level of a configuration holds 65 states
    assert (c1["engine"], c1["unit_width"]) == (mc.ENGINE["config"], 65)
    assert c1["log_capacity"] == CF.count(W.c1()) - 1 - 5  # FREE: exact, without levels 0 and 1
    assert c1["unit_threads"] == 256  # 65 states x 2 lanes in one round
    c3 = layout(W.c3(rule=W.GREEDY))  # GREEDY, P=8
    assert (c3["engine"], c3["unit_width"], c3["unit_threads"]) == (mc.ENGINE["config"], comb(8, 4), 512)
    assert c3["log_capacity"] >= CF.count(W.c3(rule=W.GREEDY)) - 1 - 10
    assert layout(W.c2_star())["engine"] == mc.ENGINE["level"]  # C(83, 3) states per level
    assert layout(W.c3_star())["engine"] == mc.ENGINE["level"]
    assert layout(W.c1(), engine="level")["engine"] == mc.ENGINE["level"]
    assert layout(W.c3(rule=W.GREEDY), unit_threads=128)["unit_threads"] == 128
    # 128-bit keys halve the width the engine takes
    wide = W.ModelSpec("w", 2, [1], [1], [1500], [1], [1, 1])  # FREE, P=2: 1501 states per level
    assert layout(wide)["engine"] == mc.ENGINE["config"]
    assert layout(wide.with_key_bits(128))["engine"] == mc.ENGINE["level"]
    # forcing the configuration engine on a model it cannot take is refused
    m = mc.mc_model_create(W.c2_star(), mc.mc_options_default(engine="config"), allocator=None)
    with pytest.raises(mc.MCError) as e:
        mc.mc_reserve(m)
    assert e.value.code == mc.MC_ERR_INVAL
    for bad in ({"engine": 3}, {"unit_threads": 48}, {"unit_threads": 1024}, {"stage_chunk": 32},
                {"stage_chunk": 224}, {"stage_chunk": 100}):
        with pytest.raises(mc.MCError):
            mc.mc_model_create(W.c1(), mc.mc_options_default(**bad), allocator=None)


def test_lanes_per_state_of_the_cost_table_model(lib):
    """A power of two from P (rounded up) to 16; the configuration engine's
    threads follow the tile (one round of the widest level)."""
    c3 = W.c3(rule=W.GREEDY)  # P = 8
    for lanes in (0, 8, 16):
        assert layout(c3, lanes_per_state=lanes)["engine"] == mc.ENGINE["config"]
    assert layout(c3, lanes_per_state=16)["unit_threads"] == 512
    assert layout(W.c1(), lanes_per_state=4)["unit_threads"] == 512  # 65 states x 4 lanes in one round
    for bad in (4, 12, 32):  # below P, not a power of two, above 16
        with pytest.raises(mc.MCError) as e:
            mc.mc_model_create(c3, mc.mc_options_default(lanes_per_state=bad), allocator=None)
        assert e.value.code == mc.MC_ERR_INVAL


def test_unknown_option_names_are_rejected(lib):
    with pytest.raises(TypeError):
        mc.mc_options_default(load_factor=10)  # the field is load_factor_pct


def test_release_cached_is_safe_without_a_device(lib):
    mc.mc_release_cached()
    mc.mc_release_cached()


def test_pool_retention_is_set_without_a_device(lib):
    # no pool exists yet: the value is kept for the pools made later
    mc.mc_set_pool_retention(8 << 30)
    mc.mc_set_pool_retention(1 << 30)


def test_strerror(lib):
    assert mc.mc_strerror(mc.MC_ERR_TABLE_FULL).startswith("visited set full")
    assert mc.mc_strerror(-99) == "unknown error"


def test_queries_fail_loudly_without_a_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = mc.mc_model_create(W.c1(), allocator=None)
    with pytest.raises(mc.MCError) as e:
        mc.mc_count_states(m)
    assert e.value.code == mc.MC_ERR_CUDA


# ---------------------------------------------------------------- PE-level model
def pe_layout(spec, **kw):
    return mc.mc_pe_model_layout(mc.mc_pe_model_create(spec, mc.mc_options_default(**kw), stream=0))


def test_pe_layout(lib):
    from paper_2305_09130_gb300 import pe_workloads as PW

    lay = pe_layout(PW.table1_row1())
    # a = b = 2 (WG, TS in {2, 4}); N <= 4; longest program: TS = 2, four
    # iterations of (3 ticks, barrier, 3 ticks, barrier) and 2 ticks = 34 steps
    assert (lay["wg_bits"], lay["ts_bits"], lay["n_bits"], lay["mask_bits"]) == (2, 2, 3, 4)
    assert lay["max_steps"] == 34 and lay["pc_bits"] == 6 and lay["unit_bits"] == 3 + 1 + 6 + 4
    # 4 + 1 + 1 successors: a tile of 4 lanes, two successors per lane
    assert lay["tile"] == 4 and lay["unit_shift"] == [0]
    # deepest FIN: WG=2, TS=2: 4 work-groups of 26 ticks on one unit, 2 PEs
    assert lay["max_level"] == 2 + 4 * (1 + 2 * 26 + 2 * 8 + 8) + 4 * 26
    big = pe_layout(PW.pe_abstract(16, P=4))
    # 16 + 4 + 1 successors: a tile of 8 lanes, three successors per lane
    assert big["tile"] == 8 and big["unit_shift"] == [3 * big["unit_bits"], 2 * big["unit_bits"],
                                                        big["unit_bits"], 0]
    assert big["used_bits"] <= 128 and big["level_shift"] == 4 * big["unit_bits"]


def test_pe_invalid_descriptions(lib):
    from paper_2305_09130_gb300 import pe_workloads as PW

    ok = PW.table1_row1()

    def variant(**kw):
        d = dict(name="bad", P=ok.P, wg_values=ok.wg_values, ts_values=ok.ts_values,
                 n_workgroups=ok.n_workgroups, pes=ok.pes, programs=ok.programs)
        d.update(kw)
        return PW.PeSpec(**d)

    cases = [
        (variant(P=0), mc.MC_ERR_INVAL),
        (variant(P=9), mc.MC_ERR_INVAL),
        (variant(n_workgroups=[0, 1, 1, 1]), mc.MC_ERR_INVAL),
        (variant(pes=[9, 1, 1, 1]), mc.MC_ERR_INVAL),
        (variant(programs=[[(1, 3)]] + ok.programs[1:], pes=[2, 2, 4, 4]), mc.MC_ERR_INVAL),
        (variant(programs=[[]] + ok.programs[1:]), mc.MC_ERR_INVAL),
        (variant(programs=[[(70000, 1)]] + ok.programs[1:]), mc.MC_ERR_INVAL),
        (variant(P=8, pes=[4, 4, 4, 4]), mc.MC_ERR_INVAL),  # 8 * 4 + 8 + 1 lanes > 32
    ]
    for spec, code in cases:
        with pytest.raises(mc.MCError) as e:
            mc.mc_pe_model_create(spec, stream=0)
        assert e.value.code == code, spec
    # a tile too narrow for the model's successors, or not a tile width
    cases = [
        (PW.pe_abstract(16, P=4), 4), (PW.pe_abstract(16, P=4), 12), (PW.table1_row1(), 2),
    ]
    for spec, tile in cases:
        with pytest.raises(mc.MCError) as e:
            mc.mc_pe_model_create(spec, mc.mc_options_default(lanes_per_state=tile), stream=0)
        assert e.value.code == mc.MC_ERR_INVAL
    for tile in (8, 16, 32):
        lay = mc.mc_pe_model_layout(mc.mc_pe_model_create(PW.pe_abstract(16, P=4),
                                                          mc.mc_options_default(lanes_per_state=tile), stream=0))
        assert lay["tile"] == tile


def test_pe_queries_fail_loudly_without_a_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2305_09130_gb300 import pe_workloads as PW

    m = mc.mc_pe_model_create(PW.table1_row1(), stream=0)
    with pytest.raises(mc.MCError) as e:
        mc.mc_pe_count_states(m)
    assert e.value.code == mc.MC_ERR_CUDA


def test_random_access_measurement_checks_its_arguments(lib):
    """The measurement utility refuses an unknown operation and a buffer
    below 1 MiB before it touches the device."""
    for buffer_bytes, op in ((64 << 20, 3), (64 << 20, -1), (1 << 19, 0)):
        with pytest.raises(mc.MCError) as e:
            mc.mc_measure_random_access(buffer_bytes, 1000, op)
        assert e.value.code == mc.MC_ERR_INVAL
