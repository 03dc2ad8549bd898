"""The bench's CPU-side pieces: the reference arm (the FP64 oracle timed on host cores) runs
end to end and prints one JSON line with the contract's keys; the work counts behind the
roofline figures follow from the workload's shapes.  CPU only."""
import json
import math
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          "small", "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and 1 <= cb["cores"] <= cb["host_cores"] == (os.cpu_count() or 1)
    assert cb["cores"] == min(os.cpu_count() or 1, 1) and cb["cpu_model"]  # one timed step, one process
    assert cb["value"] == d["value"] and cb["seconds"] > 0


def test_default_workload_is_the_largest_single_gpu_one():
    """With no flags the bench measures the 1024 x 1024 x 256 slab under 1500 views."""
    import bench
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert 'choices=list(WORKLOAD_TEXT), default="slab"' in src
    assert "1024x1024x256" in bench.WORKLOAD_TEXT["slab"] and "1500" in bench.WORKLOAD_TEXT["slab"]


def test_work_counts_follow_the_shapes():
    import bench

    class Plan:  # the two attributes the counts read
        padded = 512

    cfg = {"nu": 256, "nv": 256, "nz_layers": 32, "grid": (256, 256, 256)}
    counts = [120, 120, 120]
    half = 257
    fft = 5.0 * 512 * math.log2(512)
    assert bench.cols_flops(cfg, Plan, counts) == 360 * half * (33 * fft + 32 * 2.0 * 512)
    b = bench.algorithmic_bytes(cfg, Plan, 4, counts)
    spec = 120 * 256 * half * 8
    inter = 120 * 32 * 256 * half * 8
    stack = 120 * 32 * 258 * 258 * 4
    V = 256 ** 3
    assert np.allclose(b, [3 * (120 * 256 * 256 * 4 + spec), 3 * (spec + inter), 3 * (inter + stack),
                           3 * stack + V * 4 + 2 * V * 8])
    assert bench.aggregate_rate(6.0e9, 10, 2, 100.0) == 2 * 6.0e9 * 10 / 0.1


def test_pair_filter_option_is_refused_outside_single_axis_layered_runs():
    """The opposite-pair filter needs every view's opposite: only the single-axis workloads
    (views respread over 360 degrees) in the layered form take it."""
    import bench
    for extra in (["--workload", "slab"], ["--workload", "learned"], ["--workload", "mid", "--form", "swap"],
                  ["--workload", "mid", "--impl", "reference"]):
        out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--filter", "pair"] + extra,
                             capture_output=True, text=True, timeout=120, cwd=ROOT)
        assert out.returncode == 2 and "--filter pair" in out.stderr, (extra, out.stderr[-500:])
    # the stage-A traffic captures are of the Tikhonov kernels only
    assert bench.ncu_traffic("k_cols", "mid", "f32", "pair") is None
    assert bench.ncu_traffic("k_cols", "mid", "f32", "tikhonov") is not None
    assert bench.ncu_traffic("k_backproject", "mid", "f32", "pair") is not None
