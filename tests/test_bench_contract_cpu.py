"""The measurement script's JSON contract where it runs without a GPU: the
reference arm (the oracle on the host cores) prints one line with the keys and
types the contract fixes, and the host-side helpers of the main line behave."""
import argparse
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key, typ in (("metric", str), ("value", float), ("unit", str), ("n_gpus", int), ("steps", int),
                     ("warmup", int), ("ms_per_step", float), ("higher_is_better", bool), ("scaling", str),
                     ("dtype", str), ("data", str), ("config", dict), ("cpu_baseline", dict), ("e2e", dict)):
        assert isinstance(d[key], typ), key
    assert d["metric"] == "cell-updates/s" and d["unit"] == "cell-updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 1 and d["value"] > 0 and d["vs_baseline"] is None
    assert d["config"]["workload"] == "2d_pulse_4096x2048"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_single_thread_oracle_rate_and_cpu_model():
    sys.path.insert(0, ROOT)
    import bench

    assert isinstance(bench.cpu_model(), str) and bench.cpu_model()
    r = bench.oracle_rate_one_thread(argparse.Namespace(nx=512, ny=256), rows=16, steps=1)
    assert r is not None and r["cores"] == 1 and r["value"] > 0 and "512x16" in r["sample"]
