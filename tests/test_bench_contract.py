"""bench.py's reference arm (the FP64 oracle on the host cores) runs on a CPU machine and
prints the contract's JSON line: one line, the workload's metric and config, the
oracle as cpu_baseline and an e2e entry with no host-device traffic."""
import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, check=True, timeout=600, cwd=ROOT).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("map-steps/s") and d["unit"] == "map-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["grid"] == 2048 and d["config"]["E"] == 400.0 and d["config"]["precision"] == "fp64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "map-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
