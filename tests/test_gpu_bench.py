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


def a_ok(a):
    return a["pairs_per_s"] > 0 and "speedup_vs_p99_fixed" in a["with_fitted_control_variate"]


def test_eval_probe_calibration():
    import torch
    import paper_2607_20766_b300 as shp
    from paper_2607_20766_b300 import synth
    q = synth.principal_axes(synth.generate(3, [32]))
    d = synth.principal_axes(synth.generate(4, [39, 20]))
    Sq, Sd = shp.shape_set_load(q), shp.shape_set_load(d)
    for draw in (False, True):
        ev = shp.eval_probe(Sq, 0, Sd, 0, -1, draw, 8)
        torch.cuda.synchronize()
        assert ev > 0 and ev % (2 * 8 * 71) == 0
    with pytest.raises(shp.ShapeError):
        shp.eval_probe(Sq, 0, Sd, 5, -1, False, 8)
    with pytest.raises(shp.ShapeError):
        shp.eval_probe(Sq, 0, Sd, 0, 99, False, 8)


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
    c = r["loop_ceiling"]
    # the calibration loops do the screen's per-sample work without its per-pair work: at least as fast
    assert 0 < c["sample_path"]["frac"] <= c["eval_only"]["frac"] < 1.2
    assert c["sample_path"]["kernel_frac_of_it"] < 1.05
    assert a_ok(line["adaptive"])
    a = line["adaptive"]
    assert a["frac_se_met"] + a["frac_at_cap"] >= 0.999
    assert a["fixed_budget_p99"]["samples_per_direction"] <= a["fixed_budget"]["samples_per_direction"]
    assert a["self_overlaps"]["seconds"] > 0
    assert a["with_control_variate"]["pairs_per_s"] > 0 and a["with_fitted_control_variate"]["pairs_per_s"] > 0
    assert line["alignment"]["frac_improved"] > 0.5
    # every kernel family's roofline is there and plausible
    for arm in ("union_crn", "hybrid_fo_closed"):
        assert 0.0 < line["alignment"][arm]["roofline"]["frac"] < 1.5
    assert 0.0 < line["control_variate"]["train_roofline"]["frac"] < 1.5
    assert 0.0 < a["roofline"]["frac"] < 1.5 and 0.0 < a["first_order_kernel"]["roofline"]["frac"] < 1.5
    for pf in a["first_order_prefilter"]:
        assert pf["kept_pairs_equal_unfiltered_at_its_self_precision"] and pf["molecules_kept"] > 0
        assert 0.0 <= pf["recall_at_100"]["min"] <= 1.0 and pf["frac_se_met"] > 0.99


@pytest.mark.parametrize("case, keys", [("align", ("union_crn_ms", "fo_closed_ms")),
                                        ("prefilter", ("fo_tanimoto_ms", "select_ms")),
                                        ("self", ("self_ms",)), ("train", ("epoch_ms", "atoms")),
                                        ("load", ("load_ms", "host_ms"))])
def test_profile_cases(case, keys):
    """The small standalone cases that the profiler captures run and report
    their timings (one JSON line)."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--profile-case", case], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["case"] == case and all(line[k] > 0 for k in keys)
