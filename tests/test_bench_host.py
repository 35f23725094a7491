"""Host-side helpers of bench.py on CPU: the clock summary, the traffic record
lookup and the roofline peak source.  No GPU is involved."""

import json

import bench


def test_clock_summary_median_max_and_reasons():
    c = bench.ClockSampler(0)
    c.samples = [
        ["2070", "2070", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["1980", "2070", "Not Active", "Not Active", "Not Active", "Active"],
        ["2055", "2070", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["[N/A]", "2070", "Not Active", "Not Active", "Not Active", "Not Active"],
    ]
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["nvidia-smi unavailable"]


def test_traffic_record_is_used_only_for_the_current_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text(
        "# tag hash launch bytes\n"
        "rows16 aaaa 1 100\n"
        "rows16 bbbb 1 200\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: "bbbb")
    assert bench._profiled_traffic("rows16") == 200.0
    monkeypatch.setattr(bench, "_kernel_source_hash", lambda: "cccc")
    assert bench._profiled_traffic("rows16") is None         # sources changed since the capture
    assert bench._profiled_traffic("other") is None


def test_peak_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6701.5}))
    assert bench._peaks() == (6701.5, "measured")


def test_cpu_baseline_one_core_and_all_cores():
    cb = bench._cpu_baseline(seconds=1.0)
    assert cb["kind"] == "oracle" and cb["unit"] == "GFLOPS" and cb["value"] > 0
    assert cb["single_core_value"] > 0 and cb["cores"] >= 1 and cb["cpu_model"]
    assert str(bench.ORACLE_LINES) in cb["sample"]


def test_sar_image_deltas_against_the_stored_fp64_metrics():
    """The bench's config-3 deltas read the oracle's stored metrics: the stored
    values themselves give zero deltas, a shifted PSLR shows up in the PSLR
    column only, and another scene gets no comparison."""
    import os
    gold = json.load(open(os.path.join(bench.ROOT, "tests", "golden", "sar_4096_image_metrics.json")))
    keys = ("pslr_range_db", "pslr_azimuth_db", "islr_range_db", "islr_azimuth_db", "width_range_cells",
            "width_azimuth_cells", "peak", "snr_db")
    m = [[g[k] for k in keys] + [0.0] * 4 for g in gold["metrics"]]
    targets = [(e, r, 1.0) for e, r in gold["targets"]]
    d = bench._golden_deltas(m, targets, 4096, 4096)
    assert d["max_abs_delta_db"] == {"pslr": 0.0, "islr": 0.0, "snr": 0.0}
    assert d["max_abs_delta_width_cells"] == 0.0
    m[1][1] += 0.05
    d = bench._golden_deltas(m, targets, 4096, 4096)
    assert abs(d["max_abs_delta_db"]["pslr"] - 0.05) < 1e-12 and d["max_abs_delta_db"]["islr"] == 0.0
    assert bench._golden_deltas(m, targets, 2048, 4096) is None
    assert bench._golden_deltas(m, targets[:-1], 4096, 4096) is None
