"""The benchmark's reference arm (the oracle on the host cores) prints one JSON line with the
contract's keys; it needs no GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "laplacian_256", "--steps", "3", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "GFLOP/s" and d["steps"] == 3 and d["warmup"] >= 3
    assert d["config"]["workload"] == "laplacian_256"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_algorithmic_bytes_closed_forms():
    """The roofline's algorithmic bytes: P_MB's compulsory traffic per variant."""
    b = _bench_module()
    n, c, z = 1000, 1200, 7000
    # plain CSR, FP64 values and vectors: 4(N+1) + (4 + 8) NNZ + 8 (N + N_cols)
    assert b.alg_bytes(n, c, z, (0, 0, 0, 0, 0, 0, 0), 0, 0) == 4 * (n + 1) + 12 * z + 8 * (n + c)
    # 16-bit deltas: 2 bytes per column index plus a 4-byte base per row
    assert (b.alg_bytes(n, c, z, (0, 1, 0, 1, 1, 32, 0), 0, 0)
            == 4 * (n + 1) + 10 * z + 4 * n + 8 * (n + c))
    # FP32 storage and vectors
    assert b.alg_bytes(n, c, z, (0, 0, 0, 0, 0, 0, 0), 1, 1) == 4 * (n + 1) + 8 * z + 4 * (n + c)
    # column panels: P row-pointer sets, y passed over 2P - 1 times
    p = 3
    assert (b.alg_bytes(n, c, z, (0, 0, p, 0, 2, 0, 0), 0, 0)
            == 4 * p * (n + 1) + 12 * z + 8 * c + 8 * n * (2 * p - 1))
    # double-float storage moves 8 bytes per value
    assert b.alg_bytes(n, c, z, (0, 0, 0, 0, 0, 0, 0), 3, 0) == b.alg_bytes(
        n, c, z, (0, 0, 0, 0, 0, 0, 0), 0, 0)


def test_whole_job_rate_and_dtype_sizes():
    b = _bench_module()
    assert b.dtype_bytes(0) == 8 and b.dtype_bytes(1) == 4 and b.dtype_bytes(2) == 2
    assert b.dtype_bytes(3) == 8
    # N replicas of the same work in the max-over-ranks time
    assert b.whole_job_rate(2e9, 1.0, 4) == 4 * 2e9 / 1e-3 / 1e9


def test_reference_arm_batched_line():
    """The batched workload's reference arm: the oracle's SpMM over every matrix of the batch,
    with the GPU arm's metric and unit."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "batched_512", "--batch-count", "6", "--steps", "2",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GFLOP/s" and d["higher_is_better"] is True
    assert d["metric"].startswith("batched SpMV/SpMM GFLOP/s")
    assert d["config"]["workload"] == "batched_6" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_batched_and_cg_lines_carry_the_oracle_baseline(monkeypatch, capsys):
    """main() attaches the oracle's cpu_baseline to the batched and CG lines at N = 1 (the
    GPU runs are replaced by stubs here; the baselines themselves run on the host)."""
    b = _bench_module()
    monkeypatch.setattr(b, "run_batched", lambda args, rank, world: {"metric": "batched"})
    monkeypatch.setattr(b, "run_cg", lambda args, rank, world:
                        {"metric": "cg", "solves": {"tuned_f64": {"iters": 300}}})
    small = b.synth.laplacian_27pt
    monkeypatch.setattr(b.synth, "laplacian_27pt", lambda n: small(24))
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    for wl, unit in (("batched_512", "GFLOP/s"), ("cg27_160", "ms")):
        monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", wl, "--batch-count", "4"])
        b.main()
        d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
        cb = d["cpu_baseline"]
        assert cb["kind"] == "oracle" and cb["unit"] == unit and cb["value"] > 0
        assert cb["cores"] >= 1 and cb["sample"]
