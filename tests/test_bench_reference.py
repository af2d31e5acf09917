"""The reference arm of bench.py (the CPU oracle on the host cores) keeps
the JSON contract on the step workloads and on fragment labelling: one line
with impl, metric, value, unit, e2e (no transfers) and cpu_baseline.  Run on
small sizes, CPU only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def reference_line(workload, size):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", workload, "--size", str(size), "--steps", "2",
                          "--warmup", "3"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,size,unit", [("ring_2d", 32, "cell-updates/s"),
                                                ("spall_1d", 200, "cell-updates/s"),
                                                ("ensemble_2d", 2, "cell-updates/s"),
                                                ("fragments", 24, "cells/s")])
def test_reference_arm_json_contract(workload, size, unit):
    d = reference_line(workload, size)
    assert d["impl"] == "reference"
    assert d["unit"] == unit and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["unit"] == unit and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert cb["sample"]
    assert d["config"]["workload"] and d["config"]["cells"] > 0
