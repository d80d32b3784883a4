"""The reference arm of the bench (`bench.py --impl reference`): the float64 CPU oracle
timed on a bounded crop of the headline workload, printed as one JSON line with the same
metric, unit, direction and config as the GPU arm, a `cpu_baseline` describing the run and
an `e2e` with no host-device bytes.  Runs on the CPU (about 15 s)."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, check=True, timeout=300)
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert (line["metric"], line["unit"], line["higher_is_better"]) == ("D2Q37 MLUPS", "MLUPS", True)
    assert line["config"] == bench.headline_config(bench.LX, bench.LY, "fused", "fp64", 1)
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
