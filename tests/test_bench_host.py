"""Host-side helpers of bench.py that decide whether a measurement is valid:
the clock sampler's parsing of nvidia-smi rows (throttle reasons, clocks under
load) and the use of a profiled DRAM-traffic figure only while the sources it
was taken on are unchanged."""
import json
import os

import bench


def test_clock_summary_reports_median_clock_and_active_reasons():
    s = bench.ClockSampler(0)
    s.samples = [
        ["2070", "2070", "900.5", "Not Active", "Not Active", "Not Active", "Not Active"],
        ["2055", "2070", "950.0", "Not Active", "Not Active", "Not Active", "Active"],
        ["2070", "2070", "960.0", "Not Active", "Active", "Not Active", "Not Active"],
    ]
    r = bench.ClockSampler.summary(s)
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples_says_so():
    s = bench.ClockSampler(0)
    assert bench.ClockSampler.summary(s)["reasons"] == ["no nvidia-smi samples"]


def test_profiled_traffic_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    digest = bench.kernel_source_digest()
    monkeypatch.setattr(bench, "kernel_source_digest", lambda: digest)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    os.makedirs(tmp_path / "profiles")
    name = "gather_select_chain_kernel<2,2,3>"
    rec = {"kernel": name, "workload": "w", "dram_bytes_per_launch": 1.5e9, "kernel_source_digest": digest}
    path = tmp_path / "profiles" / "traffic_gather_select_chain_kernel_2_2_3_w.json"
    with open(path, "w") as f:
        json.dump(rec, f)
    assert bench.profiled_traffic(name, "w") == 1.5e9
    assert bench.profiled_traffic(name, "other") is None
    assert bench.profiled_traffic("gather_select_chain_kernel<1,2,2>", "w") is None
    # a record taken on other sources is not used
    with open(path, "w") as f:
        json.dump(dict(rec, kernel_source_digest="0000000000000000"), f)
    assert bench.profiled_traffic(name, "w") is None
