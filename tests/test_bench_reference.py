"""The reference arm of bench.py on CPU at N = 1: one JSON line with the
contract's keys, the oracle timed on the host cores (no GPU needed)."""
import argparse
import contextlib
import io
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        monkeypatch.delenv(k, raising=False)
    out = io.StringIO()
    args = argparse.Namespace(gpus=1, steps=1, warmup=3, workload=2)
    with contextlib.redirect_stdout(out):
        assert bench.run_reference(args) == 0
    lines = [l for l in out.getvalue().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["metric"] == bench.METRIC and d["impl"] == "reference"
    assert d["unit"] == "samples/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["dtype"] == "f64" and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_equal_error_time_is_where_the_error_settles():
    """Time to equal error is taken where a path's error stays at or below
    the target, not at an early dip (the error of a nearly empty volume)."""
    sys.path.insert(0, ROOT)
    import bench
    c = [{"step": 50, "rel_l2": 0.94}, {"step": 100, "rel_l2": 1.45},
         {"step": 150, "rel_l2": 0.80}, {"step": 200, "rel_l2": 0.70},
         {"step": 250, "rel_l2": 0.69}]
    assert bench.settled_at(c, 0.70)["step"] == 200
    assert bench.settled_at(c, 0.95)["step"] == 150
    assert bench.settled_at(c, 0.60) is None
    assert bench.settled_at(c, 2.0)["step"] == 50
    assert bench.settled_at([], 1.0) is None


def test_recorded_traffic_only_for_the_captured_source(tmp_path, monkeypatch):
    """The DRAM traffic a bench line reports comes from recorded counters
    only while the kernel's source is the one they were taken on: the
    current sources hash to the recorded keys, and a changed source (a copy
    of the tree with one byte more) reports null."""
    sys.path.insert(0, ROOT)
    import bench
    for kernel, entries in bench.TRAFFIC.items():
        for e in entries:
            assert bench.source_hash(e["source"]) == e["sha256_16"], kernel
    t = bench.traffic_of("tc_fwd_chain", 2, 1000, 0.0)
    assert t == bench.TRAFFIC["tc_fwd_chain"][0]["bytes_per_sample"] * 1000
    assert bench.traffic_of("tc_dw", 2, 0, 1e9) == bench.TRAFFIC["tc_dw"][0][
        "ratio_to_algorithmic"] * 1e9
    assert bench.traffic_of("tc_fwd_chain", 3, 1000, 0.0) is None   # no capture for workload 3
    assert bench.traffic_of("no_such_kernel", 2, 1000, 0.0) is None
    # a changed source: the same files under a root where one differs
    import shutil
    for p in bench.TRAFFIC["tc_fwd_chain"][0]["source"]:
        dst = tmp_path / p
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(ROOT, p), dst)
    with open(tmp_path / bench.TRAFFIC["tc_fwd_chain"][0]["source"][0], "ab") as f:
        f.write(b" ")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_of("tc_fwd_chain", 2, 1000, 0.0) is None
