"""Host-side pieces of bench.py (no GPU): the DRAM-traffic lookup that fills
roofline.traffic from the committed ncu summary."""
import bench


def _write(tmp_path, body):
    p = tmp_path / "traffic.txt"
    p.write_text(body)
    return str(p)


def test_traffic_is_read_per_load_factor_and_probe_scheme(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _write(tmp_path, f"""# comment: 1
kernel_source_sha256_16: {h}
dram_bytes_per_launch_lf10_split: 100
dram_bytes_per_launch_lf15_split: 200
dram_bytes_per_launch_lf10_one_call: 300
"""))
    assert bench.ncu_traffic_per_launch(10, "split") == 100.0
    assert bench.ncu_traffic_per_launch(15, "split") == 200.0
    assert bench.ncu_traffic_per_launch(10, "one_call") == 300.0
    assert bench.ncu_traffic_per_launch(15, "one_call") is None  # no capture for that pair
    assert bench.ncu_traffic_per_launch(25, "split") is None


def test_traffic_is_null_for_other_kernel_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "TRAFFIC_FILE", _write(tmp_path, """kernel_source_sha256_16: 0000000000000000
dram_bytes_per_launch_lf10_split: 100
"""))
    assert bench.ncu_traffic_per_launch(10, "split") is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.txt"))
    assert bench.ncu_traffic_per_launch(10, "split") is None
