"""bench.py's host-side contract, on the CPU: the reference arm's JSON line
(the oracle timed on the host cores) carries the keys the line format
requires; the DRAM-traffic record is reported only while the step kernel's
source is the one it was captured on; the defaults keep the timing rules
(N = 1, at least three warm-up steps)."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_the_line_format():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    for k in ("metric", "unit", "dtype", "data"):
        assert isinstance(line[k], str) and line[k]
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 1
    assert line["higher_is_better"] is True
    assert line["config"]["workload"]
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["sample"]
    assert cpu["value"] == line["value"] and cpu["unit"] == line["unit"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_traffic_record_follows_the_kernel_source(tmp_path, monkeypatch):
    import bench
    src = tmp_path / "kernel.cu"
    src.write_text("// one version of the kernel\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    rec = {"workload": "a10b10_1m", "dram_bytes_per_launch": 123, "source_sha256": sha}
    store = tmp_path / "traffic.json"
    store.write_text(json.dumps({"k_step": [rec]}))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(store))
    monkeypatch.setattr(bench, "STEP_SRC", [str(src)])
    assert bench.traffic_record("a10b10_1m")["dram_bytes_per_launch"] == 123
    assert bench.traffic_record("ternary_8m") is None
    src.write_text("// the kernel changed since the capture\n")
    assert bench.traffic_record("a10b10_1m") is None


def test_defaults_keep_the_timing_rules(monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    a = bench.parse()
    assert a.gpus == 1 and a.impl == "ours"
    assert a.warmup >= 3 and a.steps >= 1


def test_committed_traffic_records_name_their_capture():
    store = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    recs = json.load(open(store))
    for key in ("k_step", "k_conv_sweep"):
        for rec in recs[key]:
            assert rec["capture"].startswith("ncu ") and "--clock-control none" in rec["capture"]
            assert len(rec["source_sha256"]) == 64
