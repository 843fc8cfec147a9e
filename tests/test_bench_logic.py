"""Host-side helpers of bench.py (no GPU): the roofline record, the per-count
launch tally, the throughput split and the traffic record's guard."""
import json
import os

import bench


class FakeGraph:
    def __init__(self, tasks, hubs, n):
        self._i = {"num_tasks": tasks, "num_hub_roots": hubs, "n": n}

    def info(self):
        return dict(self._i)


def test_roofline_of_uses_distinct_model_and_reports_per_use():
    model = {"bytes": 2_000_000_000, "bytes_per_use": 8_000_000_000}
    r = bench.roofline_of(model, 100.0, 6498.1, "measured", "k")
    assert abs(r["achieved"] - 20.0) < 1e-9          # 2 GB in 0.1 s
    assert abs(r["frac"] - 20.0 / 6498.1) < 1e-12
    assert abs(r["per_use_model"]["frac"] - 80.0 / 6498.1) < 1e-12
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None


def test_launches_per_count():
    sch = {"hub_split": 2, "hub_split_roots": 32}
    assert bench.launches_per_count(FakeGraph(10, 5, 100), sch) == 4   # warp, hub, split finish, unrelabel
    assert bench.launches_per_count(FakeGraph(10, 0, 100), sch) == 2
    assert bench.launches_per_count(FakeGraph(0, 5, 100), dict(sch, hub_split=1)) == 2
    assert bench.launches_per_count(FakeGraph(0, 0, 0), sch) == 0


def test_rates_split():
    st = {"sets_enumerated": 10, "sets_by_signature": 90}
    r = bench.rates(st, 1000.0)
    assert r["enumerated_per_s"] == 10 and r["by_signature_per_s"] == 90


def test_traffic_record_only_for_current_kernel(tmp_path, monkeypatch):
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic_small_case.json")))
    e = rec["k4"]
    got = bench.load_traffic(4)
    if e["kernel_hash"] == bench.kernel_source_hash():
        assert got is not None and abs(got["ratio_to_algorithmic"] -
                                       e["dram_bytes_per_launch"] / e["algorithmic_bytes_of_count"]) < 1e-12
    else:
        assert got is None
    assert bench.load_traffic(3) is None


def test_full_size_traffic_record_only_for_current_kernel():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic_full_size.json")))
    e = rec["k4"]
    assert e["workload"] == bench.DEFAULT_WORKLOAD
    assert e["dram_bytes_per_launch"] == e["dram_read"] + e["dram_write"]
    got = bench.load_traffic_full(4)
    if e["kernel_hash"] == bench.kernel_source_hash():
        assert got is not None and got["dram_bytes_per_launch"] == e["dram_bytes_per_launch"]
    else:
        assert got is None
    assert bench.load_traffic_full(3) is None
