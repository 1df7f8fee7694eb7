"""bench.py's JSON contract, checked on the CPU through the reference arm (the FP64 oracle
on the host cores): one JSON line with the metric, the configuration, the CPU baseline and
the end-to-end block."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "MLUPS" and d["unit"] == "MLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["config"]["workload"] == "naca0012_a10_re6e6_ma015_6lvl_c4096"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_oracle_timing_reports_all_threads_and_one():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--oracle-timing", "--oracle-steps0", "2"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["metric"] == "oracle_MLUPS" and d["dtype"] == "f64" and d["nproc"] >= 1 and d["host"]
    runs = d["runs"]
    assert [x["threads"] for x in runs][1:] == [1] and runs[0]["threads"] >= 1
    for x in runs:
        assert x["coarse_steps"] == 2 and x["node_updates_per_step"] == 207262 and x["mlups"] > 0
