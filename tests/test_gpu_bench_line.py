"""The benchmark's JSON line on a GPU: one short run of bench.py (the headline
and its precision variants; the long legs and the CPU oracle switched off),
checked for the keys and the consistency the line promises."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def line():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device for a gpu-marked test")
    from paper_1709_08018_gb300 import build
    build.build()
    cmd = [sys.executable, "bench.py", "--steps", "3", "--warmup", "3", "--no-batch", "--no-lod",
           "--no-tiling", "--no-scan", "--no-maskit", "--no-multiseed", "--no-cull",
           "--no-cpu-baseline"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_headline_keys(line):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "clocks",
              "roofline", "e2e", "gpu_launches", "counters"):
        assert k in line, k
    assert line["n_gpus"] == 1 and line["steps"] == 3 and line["warmup"] == 3
    assert line["dtype"] == "f64" and line["higher_is_better"] is True
    assert "8192x8192" in line["config"]["workload"]
    assert line["config"]["words_per_step"] == 4 * 3 ** 19


def test_value_matches_its_step_time(line):
    words = line["config"]["words_per_step"]
    assert line["value"] == pytest.approx(words / (line["ms_per_step"] / 1000.0), rel=1e-6)
    c = line["counters"]
    assert c["in_window"] + c["dropped"] == words


def test_roofline_and_e2e(line):
    r = line["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-9)
    assert 0.3 < r["frac"] < 1.05
    # the kernel is the step, all but the parts and combine launches
    assert 0.9 < r["kernel_share_of_step"] <= 1.0
    e = line["e2e"]
    assert e["unit"] == line["unit"] and 0 < e["value"] <= 1.05 * line["value"]
    assert e["d2h_bytes_per_step"] >= 8192 * 8192 * 4 and e["h2d_bytes_per_step"] > 0
    assert line["gpu_launches"] == 3 * line["steps"]


def test_precision_variants(line):
    df, mx = line["df64_nearcusp_d20"], line["mixed_nearcusp_d20"]
    assert df["roofline"]["ops_per_word"] == 117 and mx["roofline"]["ops_per_word"] == 12
    assert df["speedup_over_fp64"] > 2 and mx["speedup_over_fp64"] > 10
    for v in (df, mx, line["mixed_gasket_d18"]):
        assert v["counters"]["in_window"] + v["counters"]["dropped"] == v["words_per_step"]
    a = line["l2_atomics"]
    assert a["peak_per_s"] > 1e9 and 0 < a["fp64_nearcusp_d20_frac"] < 1
