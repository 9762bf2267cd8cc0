"""Served queries (continuous batching): results equal the CPU oracle's and
the single-model entry points', alone and in a mix (tolerance zero), and
requests submitted while others run are admitted at once: into jobs of the
configuration engine that overlap on the device, or (lockstep engine) into
the running device loop."""
import time

import pytest

import replay as RP
from paper_2305_09130_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("status", "holds", "levels", "states", "checks", "level", "time", "t_ini", "i", "j", "key")


def single(mc, spec, kind, T):
    m = mc.mc_model_create(spec.with_key_bits(128))
    if kind == "min_time":
        r = mc.mc_min_time(m, trace=False)
        out = {"status": 0, "holds": False, "levels": None, "states": r["states"], "checks": r["checks"],
               "level": r["level"], "time": r["t_min"], "t_ini": r["t_ini"], "i": r["i"], "j": r["j"],
               "key": r["witness_key"]}
    else:
        r = mc.mc_check(m, T, trace=False)
        out = {"status": 0, "holds": r["holds"], "levels": r["levels"], "states": r["states"], "checks": 1,
               "level": r.get("cex_level", 0), "time": r.get("cex_time", 0), "t_ini": 0,
               "i": r.get("cex_i", 0), "j": r.get("cex_j", 0), "key": r.get("cex_key", 0)}
    mc.mc_model_destroy(m)
    return out


def against_oracle(mc, oracle, spec, kind, T, r):
    """A served result against the oracle under the server's options (the
    library defaults: pruning, early exit, search SINGLE with the
    certificate check, one simulated run from the default seed): every count,
    the threshold decision, the minimal time or counterexample time, its
    configuration and level, and the witness state's work-group counts."""
    lay = mc.mc_model_layout(mc.mc_model_create(spec.with_key_bits(128)))
    assert r["status"] == 0
    if kind == "min_time":
        e = oracle.min_time(spec)
        got = (r["time"], r["t_ini"], r["states"], r["checks"], r["i"], r["j"], r["level"])
        assert got == (e["t_min"], e["t_ini"], e["states"], e["checks"], e["i"], e["j"], e["level"]), (got, e)
        assert list(RP.decode(lay, r["key"])[2]) == e["n"]
    else:
        e = oracle.check(spec, T)
        assert (r["holds"], r["states"], r["levels"]) == (e["holds"], e["states"], e["levels"]), (r, e)
        if not e["holds"]:
            got = (r["time"], r["i"], r["j"], r["level"])
            assert got == (e["cex_time"], e["cex_i"], e["cex_j"], e["cex_level"]), (got, e)
            assert list(RP.decode(lay, r["key"])[2]) == e["cex_n"]


def collect(mc, srv, n, timeout_s=120):
    got = {}
    t0 = time.time()
    while len(got) < n:
        for r in mc.mc_server_poll(srv, wait_ms=50):
            got[r["ticket"]] = r
        assert time.time() - t0 < timeout_s, mc.mc_server_status(srv)
    return got


def mix():
    specs = [W.c1(W.FREE), W.c1(W.GREEDY), W.tiny(W.GREEDY), W.c2(rule=W.GREEDY)]
    specs += W.c4_instances(24, seed=2305091377)
    queries = []
    for k, s in enumerate(specs):
        queries.append(("min_time", None) if k % 2 == 0 else ("check", 40 + 13 * k))
    return specs, queries


def test_served_results_equal_alone_and_in_mix(mc, oracle):
    specs, queries = mix()
    srv = mc.mc_server_create(slots=8, pool_bytes=4 << 30)
    tickets = {mc.mc_server_submit(srv, s, k, T): idx for idx, (s, (k, T)) in enumerate(zip(specs, queries))}
    got = collect(mc, srv, len(specs))
    for t, idx in tickets.items():
        r = got[t]
        against_oracle(mc, oracle, specs[idx], *queries[idx], r)
        exp = single(mc, specs[idx], *queries[idx])
        for key in KEYS:
            if exp[key] is not None:
                assert r[key] == exp[key], (idx, key, r, exp)
        assert r["submit_s"] <= r["admit_s"] <= r["done_s"]
    assert all(r["path"] == "config" for r in got.values())
    # the same query alone on a fresh server gives the same answer: in a job
    # of its own, and with the lockstep engine on the device loop and on the
    # latency path for a lone request
    for engine, solo, path in (("auto", 0, "config"), ("level", 1, "loop"), ("level", 0, "alone")):
        alone = mc.mc_server_create(slots=1, pool_bytes=1 << 30, solo_states=solo,
                                    options=mc.mc_options_default(engine=engine))
        for idx in (0, 3, 9):
            t = mc.mc_server_submit(alone, specs[idx], *queries[idx])
            r = collect(mc, alone, 1)[t]
            assert r["path"] == path
            assert {k: r[k] for k in KEYS} == {k: got[list(tickets)[idx]][k] for k in KEYS}
        mc.mc_server_destroy(alone)
    st = mc.mc_server_status(srv)
    assert st["fatal"] == 0 and st["queued"] == 0 and st["running"] == 0
    mc.mc_server_destroy(srv)


def test_c5_shaped_queries_in_the_benchmark_server(mc, oracle):
    """Min-time queries drawn as the served benchmark draws them (G=4096,
    P=8, a new seed each, 128-bit keys), on a server with its slot count:
    submitted together they run in configuration-engine jobs that overlap on
    the device, and each answer equals the oracle's and the single-model
    entry point's; one of them alone gives the same answer."""
    specs = [W.c3(G=4096, rule=W.GREEDY, seed=2305091305 * 1000003 + 20_000_000 + k, key_bits=128)
             for k in range(16)]
    srv = mc.mc_server_create(slots=512, pool_bytes=8 << 30)
    tickets = {mc.mc_server_submit(srv, s, "min_time"): k for k, s in enumerate(specs)}
    got = collect(mc, srv, len(specs))
    assert all(r["path"] == "config" for r in got.values())
    for t, k in tickets.items():
        r = got[t]
        against_oracle(mc, oracle, specs[k], "min_time", None, r)
        exp = single(mc, specs[k], "min_time", None)
        for key in KEYS:
            if exp[key] is not None:
                assert r[key] == exp[key], (k, key, r, exp)
    mc.mc_server_destroy(srv)
    alone = mc.mc_server_create(slots=512, pool_bytes=8 << 30)
    t = mc.mc_server_submit(alone, specs[5], "min_time")
    r = collect(mc, alone, 1)[t]
    assert r["path"] == "config"
    against_oracle(mc, oracle, specs[5], "min_time", None, r)
    exp = single(mc, specs[5], "min_time", None)
    assert {k: r[k] for k in KEYS if exp[k] is not None} == {k: exp[k] for k in KEYS if exp[k] is not None}
    mc.mc_server_destroy(alone)


@pytest.mark.parametrize("engine,path,wait_s", [("auto", "config", 0.002), ("level", "loop", 0.01)])
def test_requests_join_while_others_run(mc, engine, path, wait_s):
    # a long GREEDY search is running when small queries arrive: they are
    # admitted at once (jobs of their own on other streams, or the running
    # lockstep device loop) and finish first
    long_spec = W.c3(rule=W.GREEDY)
    srv = mc.mc_server_create(slots=16, pool_bytes=8 << 30, options=mc.mc_options_default(prune=0, engine=engine),
                              solo_states=1)
    t_long = mc.mc_server_submit(srv, long_spec, "min_time")
    time.sleep(wait_s)
    small = [mc.mc_server_submit(srv, W.c1(W.FREE), "check", 80) for _ in range(6)]
    got = collect(mc, srv, 7)
    L = got[t_long]
    assert L["status"] == 0 and L["path"] == path
    for t in small:
        r = got[t]
        assert r["status"] == 0 and not r["holds"] and r["time"] == 80
        assert r["admit_s"] < L["done_s"] and r["done_s"] < L["done_s"]
        assert r["path"] == path
    st = mc.mc_server_status(srv)
    assert st["launches"] >= 1 and st["fatal"] == 0
    mc.mc_server_destroy(srv)


def test_server_rejects_models_larger_than_its_pool(mc):
    srv = mc.mc_server_create(slots=2, pool_bytes=1 << 20)
    with pytest.raises(mc.MCError) as e:
        mc.mc_server_submit(srv, W.c2_star(), "check", 95)
    assert e.value.code == mc.MC_ERR_NOMEM
    mc.mc_server_destroy(srv)


def test_lone_requests_take_the_latency_path(mc, oracle):
    # lockstep engine: each request finds the server idle, so it runs alone
    # on the single-model explorer, with the answer of the single-model entry
    # point; a request above the latency path's bound goes through the
    # device loop
    srv = mc.mc_server_create(slots=8, pool_bytes=2 << 30, options=mc.mc_options_default(engine="level"))
    specs, queries = mix()
    for idx in (0, 1, 4, 5):
        t = mc.mc_server_submit(srv, specs[idx], *queries[idx])
        r = collect(mc, srv, 1)[t]
        assert r["path"] == "alone"
        against_oracle(mc, oracle, specs[idx], *queries[idx], r)
        exp = single(mc, specs[idx], *queries[idx])
        for key in KEYS:
            if exp[key] is not None:
                assert r[key] == exp[key], (idx, key)
    big = mc.mc_server_create(slots=8, pool_bytes=2 << 30, solo_states=1 << 12,
                              options=mc.mc_options_default(engine="level"))
    t = mc.mc_server_submit(big, specs[3], *queries[3])  # c2 literal: bound above 2^12
    assert collect(mc, big, 1)[t]["path"] == "loop"
    mc.mc_server_destroy(big)
    mc.mc_server_destroy(srv)
