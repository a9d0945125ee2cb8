"""The benchmark's GPU arm prints one JSON line carrying the contract's keys, with figures
that agree with each other: a short run on the 5-point Laplacian 256x256."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_gpu_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload",
                        "laplacian_256", "--quick", "--no-cpu-baseline", "--steps", "20",
                        "--warmup", "3"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-4000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout[-4000:]
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "roofline", "e2e", "gpu_launches", "clocks", "paper_protocol"):
        assert k in d, k
    assert d["unit"] == "GFLOP/s" and d["n_gpus"] == 1 and d["steps"] == 20
    assert d["dtype"] == "f64" and d["config"]["workload"] == "laplacian_256"
    nnz = d["config"]["nnz"]
    # value is 2*NNZ per step over the per-step time (ms_per_step is printed to 5 decimals,
    # a few microseconds here)
    assert d["value"] == pytest.approx(2 * nnz / (d["ms_per_step"] * 1e-3) / 1e9, rel=2e-2)
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s"
    assert rf["achieved"] == pytest.approx(rf["alg_bytes"] / (d["ms_per_step"] * 1e-3) / 1e9,
                                           rel=2e-2)
    assert rf["frac"] == pytest.approx(rf["achieved"] / rf["peak"], rel=1e-3)
    e2e = d["e2e"]
    assert e2e["h2d_bytes_per_step"] == 8 * 65536 and e2e["d2h_bytes_per_step"] == 8 * 65536
    assert 0 < e2e["value"]
    assert d["gpu_launches"] >= d["steps"]
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    t = d["tune"]
    # the grid-searched setting the profile route ran with, and Fig. 3's one-pass class set
    # beside the two-pass one
    assert t["setting"]["source"] in ("calibrated", "library defaults")
    assert set(t["classes_fig3_one_pass"]) <= {"MB", "ML", "IMB", "CMP"}
    # the second pass only adds classes to the first pass's set
    assert set(t["classes"]) >= set(t["classes_fig3_one_pass"])
    # FP64 arithmetic: the FP64 pipe's ceiling measured by the FMA probe in the same run
    fp = d["fp64_pipe"]
    assert fp["probe_gfma_per_s"] > 0 and fp["fp64_ops_per_spmv"] >= nnz
    assert fp["frac"] == pytest.approx(fp["achieved_g_ops_per_s"] / fp["probe_gfma_per_s"],
                                       rel=2e-2)
    pp = d["paper_protocol"]
    assert pp["runs"] == 5 and pp["spmvs_per_run"] == 128 and len(pp["gflops_per_run"]) == 5
    assert min(pp["gflops_per_run"]) - 0.1 <= pp["gflops_harmonic_mean"] <= \
        max(pp["gflops_per_run"]) + 0.1
