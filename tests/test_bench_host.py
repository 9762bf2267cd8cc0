"""Host-side pieces of bench.py (no GPU): the DRAM-traffic lookup that fills
roofline.traffic from a committed ncu summary, and the bench's choice of
workloads."""
import bench


def _write(tmp_path, body):
    p = tmp_path / "traffic.txt"
    p.write_text(body)
    return str(p)


def test_traffic_is_read_per_load_factor_and_probe_scheme(tmp_path):
    h = bench.kernel_source_hash()
    path = _write(tmp_path, f"""# comment: 1
kernel_source_sha256_16: {h}
dram_bytes_per_launch_lf10_split: 100
dram_bytes_per_launch_lf15_split: 200
dram_bytes_per_launch_lf10_one_call: 300
""")
    assert bench.ncu_traffic_per_launch(path, 10, "split", 1e6) == 100.0
    assert bench.ncu_traffic_per_launch(path, 15, "split", 1e6) == 200.0
    assert bench.ncu_traffic_per_launch(path, 10, "one_call", 1e6) == 300.0
    assert bench.ncu_traffic_per_launch(path, 15, "one_call", 1e6) is None  # no capture for that pair
    assert bench.ncu_traffic_per_launch(path, 25, "split", 1e6) is None


def test_traffic_per_state_is_scaled_by_the_states_of_a_launch(tmp_path):
    h = bench.kernel_source_hash()
    path = _write(tmp_path, f"""kernel_source_sha256_16: {h}
dram_bytes_per_state_lf25_one_call: 512.5
""")
    assert bench.ncu_traffic_per_launch(path, 25, "one_call", 2e6) == 512.5 * 2e6
    assert bench.ncu_traffic_per_launch(path, 25, "split", 2e6) is None
    assert bench.ncu_traffic_per_launch(path, 40, "one_call", 2e6) is None


def test_traffic_is_null_for_other_kernel_sources(tmp_path):
    path = _write(tmp_path, """kernel_source_sha256_16: 0000000000000000
dram_bytes_per_launch_lf10_split: 100
""")
    assert bench.ncu_traffic_per_launch(path, 10, "split", 1.0) is None
    assert bench.ncu_traffic_per_launch(str(tmp_path / "missing.txt"), 10, "split", 1.0) is None


def test_committed_traffic_summaries_match_the_kernel_sources():
    """The ncu summaries behind roofline.traffic were taken on the exploration
    kernel as it stands (a kernel change needs new captures), and hold a line
    for every probe scheme the bench tunes over, at every load factor it may
    pick."""
    import os
    for name, lfs in (("c3_star", (15, 25)), ("c2_star", (10, 15))):
        wl = bench.WORKLOADS[name]
        path = os.path.join(bench.PROFILES, wl.traffic)
        fields = bench.read_traffic_file(path)
        assert fields["kernel_source_sha256_16"] == bench.kernel_source_hash(), wl.traffic
        schemes = wl.tune["probe_scheme"] if name == "c3_star" else ["split", "cas_clear"]
        for lf in lfs:
            for scheme in schemes:
                assert bench.ncu_traffic_per_launch(path, lf, scheme, 1e6) is not None, (name, lf, scheme)


def test_default_line_is_the_large_model_with_its_closed_form_optimum():
    """The headline is C3 at G=36 (FREE, P=8, 128-bit keys); its expected
    optimum is the closed form's (T_min = min over configurations of
    ceil(N/P) * cost with unit speeds)."""
    import closed_forms as CF

    wl = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    spec = wl.make()
    assert spec.P == 8 and spec.key_bits == 128 and spec.rule == 0
    assert CF.count(spec) == 1_072_924_481
    t, cfgs = CF.tmin(spec)
    i, j = cfgs[0]
    assert wl.expect == (t, spec.wg_values[i], spec.ts_values[j])
    assert wl.dtype == "u128"
    c2 = bench.WORKLOADS["c2_star"]
    s2 = c2.make()
    assert CF.count(s2) == 10_385_335
    t2, cfg2 = CF.tmin(s2)
    assert c2.expect == (t2, s2.wg_values[cfg2[0][0]], s2.ts_values[cfg2[0][1]])


def test_swarm_summary_reports_optimality_against_the_exact_minimum():
    runs = [{"walks": 2_000_000, "total_ms": 2.0, "first_trail_ms": 0.5, "rounds": 2, "first_time": 120,
             "best_time": 100, "wg": 8, "ts": 4},
            {"walks": 2_000_000, "total_ms": 2.0, "first_trail_ms": 0.4, "rounds": 3, "first_time": 100,
             "best_time": 100, "wg": 8, "ts": 4}]
    s = bench.swarm_summary(100, runs)
    assert s["runs_per_s"] == 4_000_000 / 0.004
    assert s["t_min_exact"] == 100
    assert [x["first_trail_optimality"] for x in s["searches"]] == [100 / 120, 1.0]
    assert [x["final_optimality"] for x in s["searches"]] == [1.0, 1.0]
