"""The JSON line of bench.py, checked on the CPU: bench.main() runs with the
library and CUDA faked (tests/bench_fakes.py, in a process of its own) and
the line must carry every key of the bench contract, with values that follow
from the fake timings by the formulas the line states."""
import json
import os
import subprocess
import sys

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H = W = 4096
EVENT_MS = 2.0          # every fake timed region
K3_MS = 1.9             # the fake kernel-timing hook's forward entry


@pytest.fixture(scope="module")
def line():
    from paper_1203_5128_gb300 import build
    build.build()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bench_fakes.py"),
                        "--steps", "2", "--warmup", "3", "--oracle-rows", "128"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return json.loads(lines[0])


def test_top_level_keys(line):
    for k in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"]:
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 2 and line["warmup"] == 3
    assert line["unit"] == "Mpixel/s" and line["higher_is_better"] is True
    assert line["scaling"] == "weak" and line["vs_baseline"] is None
    assert line["data"] == "synthetic" and "workload" in line["config"]


def test_value_and_step_time(line):
    assert line["ms_per_step"] == pytest.approx(EVENT_MS)
    assert line["value"] == pytest.approx(H * W / (EVENT_MS * 1e3))
    assert line["gpu_launches"] == 4 * 2


def test_roofline(line):
    r = line["roofline"]
    for k in ["bound", "achieved", "peak", "unit", "frac", "traffic"]:
        assert k in r, k
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    assert r["achieved"] == pytest.approx(r["algorithmic_flops_per_launch"] / (K3_MS * 1e-3) / 1e12)


def test_cpu_baseline_and_e2e(line):
    c = line["cpu_baseline"]
    assert c["kind"] == "oracle" and c["unit"] == "Mpixel/s" and c["cores"] >= 1
    assert c["value"] > 0 and "rows 0..127" in c["sample"]
    e = line["e2e"]
    assert e["unit"] == "Mpixel/s" and e["value"] > 0
    assert e["h2d_bytes_per_step"] == 4 * H * W and e["d2h_bytes_per_step"] == 4 * H * W


def test_extra_legs(line):
    for k in ["tuned", "plain", "tuned_fp32", "tuned_yvv", "batch", "backward", "box"]:
        assert k in line, k
    for planes in ["fp16", "fp32"]:
        b = line["box"][planes]
        assert b["value"] == pytest.approx(H * W / (EVENT_MS * 1e3))
    assert line["tuned_fp32"]["roofline"]["bound"] == "alu"
    assert line["tuned_yvv"]["roofline_hbm"]["bound"] == "hbm"


def test_parity_and_sweep_legs(line):
    t = line["tuned"]
    assert t["every_pixel"]["outputs"] == 128 * W and t["every_pixel"]["max_abs"] >= 0
    assert "recheck" in t["kernel_ms"]
    for planes in ["fp32", "bf16", "fp16"]:
        e = line["precision"][planes]
        assert e["value"] == pytest.approx(H * W / (EVENT_MS * 1e3)) and e["max_abs"] >= 0
    cells = line["config1"]["cells"]
    assert sorted((c["sigma_s"], c["sigma_r"]) for c in cells) == \
        [(5.0, 10.0), (5.0, 20.0), (10.0, 10.0), (10.0, 20.0)]
    for c in cells:
        assert c["speedup_tile"] == pytest.approx(c["accel_tile"]["value"] / c["plain"]["value"])
    for k in ["poly_fixed", "poly_tile", "cosine_fixed", "cosine_tile"]:
        assert line["poly"][k]["value"] > 0
    assert line["nlm"]["value"] > 0 and line["nlm"]["max_abs"] >= 0
    d = line["divergence"]
    for k in ["vs_direct_gaussian", "vs_plain_parameters"]:
        assert d[k]["max_abs"] >= 0 and d[k]["mse"] >= 0
