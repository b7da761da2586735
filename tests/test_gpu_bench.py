"""The benchmark's JSON line on a B300, at small sizes: every key of the
contract is there and consistent (roofline, clocks, end-to-end leg, CPU
baseline, launch count, the adaptive, control-variate and alignment
sections)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def test_bench_json_line_small():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--n-db", "3000", "--steps", "3", "--warmup", "3",
           "--adaptive-db", "3000", "--cv-train", "3000", "--cv-held", "500", "--align-db", "200",
           "--fit-samples", "1024"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "clocks", "e2e", "gpu_launches", "cpu_baseline",
              "adaptive", "control_variate", "alignment"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] == 3 and line["value"] > 0
    r = line["roofline"]
    assert r["bound"] == "alu" and 0 < r["frac"] < 1.2 and abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert line["e2e"]["h2d_bytes_per_step"] > 0 and line["e2e"]["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["gpu_launches"] == 5 * line["steps"]
    a = line["adaptive"]
    assert a["frac_se_met"] + a["frac_at_cap"] >= 0.999
    assert a["with_control_variate"]["pairs_per_s"] > 0 and a["with_fitted_control_variate"]["pairs_per_s"] > 0
    assert line["alignment"]["frac_improved"] > 0.5
