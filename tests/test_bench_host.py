"""bench.py host logic on the CPU: the DRAM-traffic lookup behind `roofline.traffic`, the
race-check kernel names, and the profiling-size workloads."""
import json
import os

import numpy as np

import bench


def test_committed_traffic_file_is_well_formed():
    t = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    assert t["captures"]
    for c in t["captures"]:
        assert c["workload"] in bench.WORKLOADS
        assert c["kernel"] in ("k_interp_plain", "k_interp_batched", "k_interp_blocks + k_interp_batched", "k_check",
                               "k_check_reg", "k_check_lean")
        assert c["unit"] in ("block", "record") and c["units"] > 0
        assert c["dram_read"] > 0 and c["dram_write"] >= 0
        assert "--clock-control none" in c["command"] and len(c["src_sha1"]) == 16


def test_traffic_is_scaled_by_unit_and_keyed_by_workload_and_source(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"captures": [
        {"workload": "reduction", "kernel": "k_check_reg", "src_sha1": "a" * 16, "unit": "block",
         "units": 100, "dram_read": 900, "dram_write": 100, "command": ""},
        {"workload": "batched", "kernel": "k_check_reg", "src_sha1": "a" * 16, "unit": "record",
         "units": 50, "dram_read": 400, "dram_write": 100, "command": ""},
    ]}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    units = {"block": 1000, "record": 500}
    assert bench.traffic_per_launch("reduction", "k_check_reg", "a" * 16, units) == 10 * 1000
    assert bench.traffic_per_launch("batched", "k_check_reg", "a" * 16, units) == 10 * 500
    # another workload, kernel or source: no number rather than a wrong one
    assert bench.traffic_per_launch("stencil2d", "k_check_reg", "a" * 16, units) is None
    assert bench.traffic_per_launch("reduction", "k_interp_plain", "a" * 16, units) is None
    assert bench.traffic_per_launch("reduction", "k_check_reg", "b" * 16, units) is None


def test_check_kernel_names():
    assert [bench.check_kernel(v) for v in (1, 2)] == ["k_check", "k_check"]
    assert [bench.check_kernel(v) for v in (0, 3, 4, 5)] == ["k_check_reg"] * 4


def test_profiling_size_batched_workload_is_a_prefix_of_the_full_one():
    # program i depends on (seed, i) only, so any smaller size is a prefix of the full batch
    small = bench.workload("batched", 0, programs=12)
    larger = bench.workload("batched", 0, programs=40)
    assert len(larger) == 40 and len(small) == 12
    for a, b in zip(small, larger):
        assert np.array_equal(a.code, b.code) and a.launches == b.launches
        assert np.array_equal(a.global_init, b.global_init)
