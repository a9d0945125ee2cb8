"""Benchmark: adaptive CSR SpMV GFLOP/s and HBM-roofline fraction on one GB300.

Default workload: the bandwidth-bound 27-point stencil on a 160^3 grid (N = 4,096,000,
NNZ = 109,215,352), FP64 values, FP64 x. A step is one y = A x through the tuned handle
(the amortized hot loop); tuning and preprocessing happen once before the timed region and
are reported as t_pre. The plain CSR-vector baseline and the FP32 / BF16 storage variants
are timed beside it. Inputs (about 1.2 GB) are larger than L2, so no flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs an independent replica (the method does not shard: one
matrix, one GPU); rank 0 prints one JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0


def _peaks():
    try:
        with open(MEASURED) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# ------------------------------------------------------------------------ clocks -----
class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# ---------------------------------------------------------------------- workloads ----
WORKLOADS = {
    "stencil27_160": dict(desc="27-point 3-D stencil, 160^3 grid, natural order, FP64 values "
                               "U[-1,1] off-diagonal with a dominant diagonal, FP64 x",
                          make=lambda: synth.stencil_27pt(160), x_seed=synth.SEED_BASE + 12),
    "stencil27_100": dict(desc="27-point 3-D stencil, 100^3 grid (profiling-size case), FP64",
                          make=lambda: synth.stencil_27pt(100), x_seed=synth.SEED_BASE + 12),
    "laplacian_256": dict(desc="5-point 2-D Laplacian 256x256, FP64", make=lambda: synth.laplacian_2d(256),
                          x_seed=synth.SEED_BASE + 11),
    "powerlaw_4m": dict(desc="power-law rows Zipf(1.8) clipped at 200,000, N=4,000,000, FP32",
                        make=lambda: synth.power_law(4_000_000), x_seed=synth.SEED_BASE + 13),
    "scattered_16m": dict(desc="16,000,000 rows x 8 uniform random columns, FP64",
                          make=lambda: synth.scattered(16_000_000, 8), x_seed=synth.SEED_BASE + 14),
    "powerlaw_1m": dict(desc="power-law rows Zipf(1.8) clipped at 200,000, N=1,000,000, FP32 "
                             "(profiling-size case)",
                        make=lambda: synth.power_law(1_000_000), x_seed=synth.SEED_BASE + 13),
    "scattered_4m": dict(desc="4,000,000 rows x 8 uniform random columns, FP64 (profiling-size "
                              "case)", make=lambda: synth.scattered(4_000_000, 8),
                         x_seed=synth.SEED_BASE + 14),
}


CALIBRATION = os.path.join(ROOT, "paper_1711_05487_gb300", "data", "calibration_gb300.json")


def route_opts() -> dict:
    """Tune options of the grid-searched setting (Section III-C: thresholds tuned on the target
    platform, here with the uneven-rows ratio and the row decomposition limits) when the
    calibration file is present; the library's defaults otherwise."""
    try:
        with open(CALIBRATION) as fh:
            c = json.load(fh)
        return {"t_imb": float(c["t_imb"]), "t_ml": float(c["t_ml"]), "t_mb": float(c["t_mb"]),
                "long_row_ratio": float(c["long_ratio"]), "bin_med": int(c["bin_med"]),
                "bin_chunk": int(c["bin_chunk"])}
    except (OSError, KeyError, ValueError):
        return {}


def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's time (the timed region ends when every replica is done)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_replica: float, ms_max: float, world: int) -> float:
    """Units all replicas processed per second (weak scaling: every rank runs the full
    workload), in giga-units."""
    return world * units_per_replica / (ms_max * 1e-3) / 1e9


def measured_traffic(workload: str, variant) -> dict | None:
    """DRAM bytes per launch of the dominant kernel from an ncu capture (profiles/), valid only
    for the same variant and unchanged kernel sources (the files the entry lists)."""
    try:
        from paper_1711_05487_gb300.buildlib import source_digest
        with open(TRAFFIC) as fh:
            t = json.load(fh).get(workload)
        if (t and list(t["variant"]) == list(variant)
                and t["source_digest"] == source_digest(t.get("sources"))):
            return t
    except Exception:
        return None
    return None


def dtype_bytes(code):
    return {0: 8, 1: 4, 2: 2, 3: 8}[code]


def alg_bytes(n_rows, n_cols, nnz, variant, storage, vec, handle=None):
    """Compulsory traffic of one SpMV with the variant's own format (P_MB's M_min):
    row pointers, column indices (int32 or 16-bit deltas + per-row base), values, x, y.
    Column panels (xpath = P >= 2) read P sets of row pointers and pass over y 2P - 1 times
    (written once, then read and written by every later pass). Sliced rows (partition 3)
    read their padded positions and one 8-byte offset per 32-row slice."""
    if variant[0] == 3 and handle is not None:
        from paper_1711_05487_gb300 import _abi
        try:
            positions, bits = _abi.spmv_get_sell(handle)
        except _abi.SpmvError:      # the handle has since been re-tuned without slices
            positions, bits = nnz, (16 if variant[1] == 1 else 0)
        vb = 8 if storage == 3 else dtype_bytes(storage)
        ib = bits // 8 if bits else 4
        extra = 4 * n_rows if bits else 0
        return (4 * (n_rows + 1) + 8 * ((n_rows + 31) // 32 + 1) + (ib + vb) * positions
                + extra + dtype_bytes(vec) * (n_rows + n_cols))
    if len(variant) > 2 and variant[2] >= 2:
        p = variant[2]
        vb = 8 if storage == 3 else dtype_bytes(storage)
        return (4 * p * (n_rows + 1) + (4 + vb) * nnz + dtype_bytes(vec) * n_cols
                + dtype_bytes(vec) * n_rows * (2 * p - 1))
    idx = 2 if variant[1] == 1 else 4
    extra = 4 * n_rows if variant[1] == 1 else 0
    return (4 * (n_rows + 1) + (idx + dtype_bytes(storage)) * nnz + extra
            + dtype_bytes(vec) * (n_rows + n_cols))


def launches_per_spmv(A, variant) -> int:
    """Kernel launches of one SpMV with the installed variant."""
    from paper_1711_05487_gb300 import _abi
    if len(variant) > 2 and variant[2] >= 2:
        return variant[2]                                  # one pass per column panel
    if variant[0] == 1:
        n_tiles, _ = _abi.spmv_get_merge_path(A.handle)
        return 1 + (n_tiles > 1)                           # tiles, then the carry fixup
    if variant[0] == 2:
        n_med, n_long, n_ch = _abi.spmv_get_row_bins(A.handle)
        return 1 + (n_long > 0)                            # rows and warp items, fixup
    return 1


# --------------------------------------------------------------------------- ours ----
def run_ours(args, rank, world):
    import torch

    from paper_1711_05487_gb300 import api

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    wl = WORKLOADS[args.workload]
    t0 = time.time()
    m = wl["make"]()
    gen_s = time.time() - t0
    x_host = synth.uniform_vector(m.n_cols, wl["x_seed"])
    stream = torch.cuda.Stream()
    A = api.SpmvMatrix.from_csr(m, stream=stream)
    vec_t = torch.float64 if m.val.dtype == np.float64 else torch.float32
    if m.val.dtype != np.float64:
        A.set_precision("f32", "f32", "f32", stream=stream)
    elif args.precision == "df64":
        A.set_precision("df64", "f64", "df64", stream=stream)
    elif args.precision in ("f32", "bf16"):
        A.set_precision(args.precision, "f32", "f32", stream=stream)
        vec_t = torch.float32
    x = torch.from_numpy(x_host).to(vec_t).cuda()
    y = torch.empty(m.n_rows, dtype=vec_t, device="cuda")
    flops = 2.0 * m.nnz

    def timed(K, W, tag="timed"):
        with torch.cuda.stream(stream):
            for _ in range(W):
                A.run(x, y, stream=stream)
            stream.synchronize()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push(tag)
            e0.record(stream)
            for _ in range(K):
                A.run(x, y, stream=stream)
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
            e1.synchronize()
            torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), world) / K

    # plain CSR-vector baseline
    A.set_variant(stream=stream)
    base_ms = timed(args.steps, args.warmup)
    # adaptive: profile-guided classification + Table II variant + autotuned width
    # (--fixed-variant installs a given variant instead, so that a run under a profiler, whose
    # inflated timings would steer the tuner elsewhere, executes the kernel a plain run picks)
    if args.fixed_variant:
        knobs = [int(v) for v in args.fixed_variant.split(",")]
        rep = A.tune("fixed", stream=stream, fixed=api.variant(*knobs))
    else:
        rep = A.tune("profile", stream=stream, **route_opts())
    peak, peak_kind = _peaks()
    clocks = ClockSampler(dev)
    clocks.start()
    # keep the GPU loaded for ~1.5 s before the timed region so that the clock samples
    # (100 ms apart) see the kernel running; these steps are not timed
    t_load = time.time()
    with torch.cuda.stream(stream):
        while time.time() - t_load < 1.5:
            for _ in range(50):
                A.run(x, y, stream=stream)
            stream.synchronize()
    ms = timed(args.steps, args.warmup, tag="bench_timed")
    clocks.stop()
    # Section IV-A's protocol beside the contract's figure: 5 runs of 128 back-to-back SpMVs,
    # harmonic mean of the per-run rates
    run_rates = [flops / (timed(128, 1) * 1e-3) / 1e9 for _ in range(5)]
    protocol = {"runs": 5, "spmvs_per_run": 128,
                "gflops_harmonic_mean": round(len(run_rates) / sum(1.0 / r for r in run_rates), 2),
                "gflops_per_run": [round(r, 1) for r in run_rates]}
    storage = A.storage
    traffic = measured_traffic(args.workload + ("" if args.precision == "native"
                                                 else "/" + args.precision), rep.variant)
    ab = alg_bytes(m.n_rows, m.n_cols, m.nnz, rep.variant, storage, A.vec, A.handle)
    achieved = ab / (ms * 1e-3) / 1e9
    csr_bytes = alg_bytes(m.n_rows, m.n_cols, m.nnz, (0, 0, 0, 0, 0), storage, A.vec)
    value = whole_job_rate(flops, ms, world)
    # end to end through the C ABI with host buffers (x in, y out, copies inside the timing)
    xh = torch.from_numpy(x_host).to(vec_t).pin_memory()
    yh = torch.empty(m.n_rows, dtype=vec_t).pin_memory()
    for _ in range(max(1, args.warmup)):
        A.run_host(xh, yh, stream=stream)
    te = time.perf_counter()
    for _ in range(args.steps):
        A.run_host(xh, yh, stream=stream)
    e2e_ms = max_over_ranks((time.perf_counter() - te) * 1e3 / args.steps, world)
    # Section IV-D: solver iterations that amortize each route's tuning over the plain
    # CSR-vector, N_iters,min = t_pre / (t_base - t_opt)
    def n_iters(t_pre_ms, t_opt_ms):
        return round(t_pre_ms / (base_ms - t_opt_ms), 1) if base_ms > t_opt_ms else None

    amort = {"profile": {"t_pre_ms": round(rep.t_pre_ms, 2), "t_spmv_ms": round(ms, 5),
                         "n_iters_min": n_iters(rep.t_pre_ms, ms)}}
    sel_path = os.path.join(ROOT, "paper_1711_05487_gb300", "data", "selector_gb300.npz")
    if not args.quick and os.path.exists(sel_path) and not args.fixed_variant:
        sel = api.Selector.load(sel_path)
        for route, kw in (("learned", dict(selector=sel)), ("features", {})):
            r_l = A.tune(route, stream=stream, **kw, **route_opts())
            t_l = timed(max(8, args.steps // 4), args.warmup)
            amort[route] = {"t_pre_ms": round(r_l.t_pre_ms, 2), "t_spmv_ms": round(t_l, 5),
                            "classes": r_l.class_names, "variant": list(r_l.variant),
                            "n_iters_min": n_iters(r_l.t_pre_ms, t_l)}
            if route == "learned":
                # margin -1: the matrix lies outside the selector's training range and the
                # route profiled it instead
                amort[route]["decided_by"] = ("mlp" if r_l.mode_used == 2 else "profile")
                amort[route]["margin"] = round(r_l.margin, 4)
                amort[route]["t_learned_over_t_profile"] = round(t_l / ms, 4)
        # Section IV-D's trivial optimizers: try every single optimization (5) or also every
        # pair of them (15 in all), 64 timed SpMVs each, keep the fastest; t_pre is the whole
        # search including each candidate's preprocessing
        singles = {"delta16": dict(index=1, vec=1), "xl2": dict(xpath=1),
                   "merge": dict(partition=1), "vector": dict(vec=1), "tile": dict(vec=1, vs=1)}
        names = list(singles)
        pairs = [(a, b) for i, a in enumerate(names) for b in names[i + 1:]]

        def trivial(cands):
            t0 = time.perf_counter()
            best = None
            for knobs in cands:
                A.set_variant(stream=stream, **knobs)
                t_c = timed(64, 2)
                if best is None or t_c < best[0]:
                    best = (t_c, knobs)
            t_pre = (time.perf_counter() - t0) * 1e3
            return {"t_pre_ms": round(t_pre, 2), "t_spmv_ms": round(best[0], 5),
                    "candidates": len(cands), "best": best[1],
                    "n_iters_min": n_iters(t_pre, best[0])}

        single_c = [singles[n] for n in names]
        amort["trivial_single"] = trivial(single_c)
        amort["trivial_combined"] = trivial(single_c + [{**singles[a], **singles[b]}
                                                       for a, b in pairs])
        A.tune("fixed", stream=stream, fixed=api.variant(*rep.variant))
    # every pool variant timed on this matrix: the paper's "oracle" (perfect optimizer)
    sweep = {}
    if not args.quick:
        pool = {"csr_vector": dict(), "vector_w4": dict(vec=1, vs=4),
                "tile_i32": dict(vec=1, vs=1), "tile_delta16": dict(index=1, vec=1, vs=1),
                "tile_i32_xl2": dict(vec=1, vs=1, xpath=1),
                "subwarp_delta16": dict(index=1, vec=1, vs=4), "merge_path": dict(partition=1),
                "col_panels_2": dict(xpath=2, vs=2), "sliced_delta16": dict(partition=3, index=1)}
        for name, knobs in pool.items():
            A.set_variant(stream=stream, **knobs)
            t_v = timed(max(8, args.steps // 4), args.warmup)
            vb = alg_bytes(m.n_rows, m.n_cols, m.nnz,
                           (knobs.get("partition", 0), knobs.get("index", 0),
                            knobs.get("xpath", 0)), storage, A.vec)
            sweep[name] = {"gflops": round(flops / (t_v * 1e-3) / 1e9, 1),
                           "frac_hbm": round(vb / (t_v * 1e-3) / 1e9 / peak, 3)}
        A.tune("fixed", stream=stream, fixed=api.variant(*rep.variant))
    # reduced-precision value storage on the same matrix (FP64 originals rounded once)
    extra = {}
    if m.val.dtype == np.float64 and not args.quick:
        for st, vt, at in (("df64", "f64", "df64"), ("f32", "f64", "f64"), ("f32", "f64", "df64"),
                           ("bf16", "f64", "df64"), ("f32", "f32", "f32"), ("bf16", "f32", "f32")):
            A.set_precision(st, vt, at, stream=stream)
            r2 = A.tune("profile", stream=stream, **route_opts())
            xv = x.to(torch.float64 if vt == "f64" else torch.float32)
            yv = torch.empty(m.n_rows, dtype=xv.dtype, device="cuda")
            x_old, y_old = x, y
            x, y = xv, yv
            t2 = timed(args.steps, args.warmup)
            x, y = x_old, y_old
            b2 = alg_bytes(m.n_rows, m.n_cols, m.nnz, r2.variant, A.storage, A.vec, A.handle)
            extra[f"{st}/{vt}/{at}"] = {
                "gflops": round(flops / (t2 * 1e-3) / 1e9, 1),
                "variant": list(r2.variant), "classes": r2.class_names,
                "frac_hbm": round(b2 / (t2 * 1e-3) / 1e9 / peak, 3)}
        A.set_precision("f64", "f64", "f64", stream=stream)
    fp64_pipe = None
    if storage == 0:
        # the FP64 pipe's ceiling measured now by the register-only FMA probe (4 chains per
        # thread, 32 warps per SM); the SpMV spends one FMA per nonzero, plus one add per row
        # where delta-coded tile rows are summed in two chains
        from paper_1711_05487_gb300 import _abi
        r_fma = _abi.spmv_probe_fma(8, 4, 32, 5, stream.cuda_stream)
        v = rep.variant
        adds = m.n_rows if (v[0] == 0 and v[1] != 0 and v[4] == 1) else 0
        ops = m.nnz + adds
        fp64_pipe = {"probe_gfma_per_s": round(r_fma / 1e9, 1),
                     "probe": "spmv_probe_fma(8 bytes, 4 chains, 32 warps per SM)",
                     "fp64_ops_per_spmv": int(ops), "dfma": int(m.nnz), "dadd": int(adds),
                     "achieved_g_ops_per_s": round(ops / (ms * 1e-3) / 1e9, 1),
                     "t_min_ms": round(ops / r_fma * 1e3, 5),
                     "frac": round(ops / (ms * 1e-3) / r_fma, 4),
                     "frac_of_nominal_625_gfma": round(ops / (ms * 1e-3) / 625e9, 4)}
    out = {
        "metric": "SpMV GFLOP/s (2*nnz/t), adaptive (profile-guided) vs plain CSR-vector",
        "value": round(value, 2),
        "unit": "GFLOP/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {0: "f64", 1: "f32", 2: "bf16", 3: "df64"}[storage],
        "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "desc": wl["desc"], "n_rows": m.n_rows,
                   "nnz": m.nnz, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (no flush needed)" if csr_bytes > 200e6
                   else "L2-resident working set"},
        "baseline_csr_vector": {"gflops": round(flops / (base_ms * 1e-3) / 1e9, 2),
                                "ms": round(base_ms, 5),
                                "frac_hbm": round(csr_bytes / (base_ms * 1e-3) / 1e9 / peak, 3)},
        "speedup_vs_csr_vector": round(base_ms / ms, 3),
        "paper_protocol": protocol,
        "tune": {"classes": rep.class_names, "variant": list(rep.variant),
                 "setting": {"source": "calibrated" if route_opts() else "library defaults",
                             **route_opts()},
                 "classes_fig3_one_pass": fig3_one_pass(rep.p) if rep.p["P_CSR"] > 0 else None,
                 "p_gflops": {k: round(v, 1) for k, v in rep.p.items()},
                 "b_max_gbs": round(rep.b_max_gbs, 1), "t_pre_ms": round(rep.t_pre_ms, 2)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "traffic": traffic["dram_bytes_per_launch"] if traffic else None,
                     "traffic_source": traffic["source"] if traffic else None,
                     "peak_kind": peak_kind, "alg_bytes": ab,
                     "frac_of_nominal_8tbs": round(achieved / NOMINAL_HBM_GBS, 4),
                     "csr_fp64_bytes_frac": round(csr_bytes / (ms * 1e-3) / 1e9 / peak, 4)},
        "e2e": {"value": round(whole_job_rate(flops, e2e_ms, world), 2), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(xh.numel() * xh.element_size()),
                "d2h_bytes_per_step": int(yh.numel() * yh.element_size()),
                "ms_per_step": round(e2e_ms, 4)},
        "gpu_launches": args.steps * launches_per_spmv(A, rep.variant),
        "precision_variants": extra,
        "variant_sweep": sweep,
        "amortization": amort,
        "fp64_pipe": fp64_pipe,
        "clocks": clocks.summary(),
        "gen_s": round(gen_s, 1),
    }
    return out, m


def run_batched(args, rank, world):
    """512 mixed FP32 matrices (N log-uniform in [1e3, 2e5]) with k in {1, 4, 16} right-hand
    sides each: one graph-captured persistent launch per step, against the same products
    launched matrix by matrix."""
    import concurrent.futures as cf

    import torch

    from paper_1711_05487_gb300 import api

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    specs = synth.batched_specs(args.batch_count)
    t0 = time.time()
    with cf.ThreadPoolExecutor(max_workers=max(2, (os.cpu_count() or 4) - 2)) as ex:
        mats = list(ex.map(lambda sp: synth.make_from_spec(sp, dtype=np.float32), specs))
    gen_s = time.time() - t0
    stream = torch.cuda.Stream()
    sel_path = os.path.join(ROOT, "paper_1711_05487_gb300", "data", "selector_gb300.npz")
    sel = api.Selector.load(sel_path) if os.path.exists(sel_path) else None
    As, Xs, Ys, ks = [], [], [], []
    flops = 0.0
    nbytes = 0
    t_tune = 0.0
    by_mlp = 0
    for sp, m in zip(specs, mats):
        A = api.SpmvMatrix.from_csr(m, stream=stream)
        A.set_precision("f32", "f32", "f32", stream=stream)
        if sel is not None:
            r = A.tune("learned", stream=stream, selector=sel, **route_opts())
            t_tune += r.t_pre_ms
            by_mlp += r.mode_used == 2
        else:
            A.set_variant(stream=stream)
        k = sp["k"]
        X = torch.from_numpy(synth.uniform_vector(m.n_cols * k, sp["seed"], np.float32)
                             ).reshape(m.n_cols, k).cuda()
        As.append(A)
        Xs.append(X)
        Ys.append(torch.empty((m.n_rows, k), dtype=torch.float32, device="cuda"))
        ks.append(k)
        flops += 2.0 * m.nnz * k
        nbytes += 4 * (m.n_rows + 1) + 8 * m.nnz + 4 * k * (m.n_rows + m.n_cols)
    B = api.Batch(As, Xs, Ys, ks, stream=stream)
    # the batch's work plan (items per warp, chunk length of split rows) by its autotuner
    t0 = time.perf_counter()
    plan = B.tune(reps=5, stream=stream)
    t_plan = (time.perf_counter() - t0) * 1e3

    def timed(fn, K, W, tag):
        with torch.cuda.stream(stream):
            for _ in range(W):
                fn(stream=stream)
            stream.synchronize()
            if world > 1:
                torch.distributed.barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.nvtx.range_push(tag)
            e0.record(stream)
            for _ in range(K):
                fn(stream=stream)
            e1.record(stream)
            torch.cuda.nvtx.range_pop()
            e1.synchronize()
        return max_over_ranks(e0.elapsed_time(e1), world) / K

    peak, peak_kind = _peaks()
    seq_ms = timed(B.run_sequential, max(4, args.steps // 8), args.warmup, "batched_sequential")
    clocks = ClockSampler(dev)
    clocks.start()
    t_load = time.time()
    with torch.cuda.stream(stream):
        while time.time() - t_load < 1.5:
            B.run(stream=stream)
            stream.synchronize()
    ms = timed(B.run, args.steps, args.warmup, "bench_timed")
    clocks.stop()
    achieved = nbytes / (ms * 1e-3) / 1e9
    total_nnz = sum(m.nnz for m in mats)
    # the measured ceiling of the x-row gathers: one 32-byte L2 sector per nonzero for k = 1
    # and k = 4 (4- and 16-byte rows), two for k = 16 (64-byte rows), at the random-gather
    # rate of an L2-resident array
    from paper_1711_05487_gb300 import _abi
    sectors = sum(m.nnz * (2 if k == 16 else 1) for m, k in zip(mats, ks))
    t_g = _abi.spmv_probe_gather(4 << 20, 4, sectors, 5)
    learned = None
    if sel is not None:
        # the same batch with every matrix tuned by the profile route instead (what the
        # learned route is compared with), at the same work plan
        t_prof = 0.0
        for A in As:
            t_prof += A.tune("profile", stream=stream, **route_opts()).t_pre_ms
        B.close()
        B = api.Batch(As, Xs, Ys, ks, stream=stream)
        B.set_plan(*plan)
        ms_p = timed(B.run, args.steps, args.warmup, "batched_profile_route")
        learned = {"decided_by_mlp": int(by_mlp), "matrices": len(As),
                   "t_pre_ms_total": round(t_tune, 1),
                   "profile_route": {"gflops": round(flops / (ms_p * 1e-3) / 1e9, 2),
                                     "ms": round(ms_p, 5), "t_pre_ms_total": round(t_prof, 1)},
                   "t_learned_over_t_profile": round(ms / ms_p, 4)}
    out = {
        "metric": "batched SpMV/SpMM GFLOP/s (sum of 2*nnz*k / t), one persistent launch",
        "value": round(whole_job_rate(flops, ms, world), 2), "unit": "GFLOP/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": f"batched_{len(mats)}", "matrices": len(mats),
                   "total_nnz": total_nnz,
                   "k_hist": {str(k): ks.count(k) for k in (1, 4, 16)},
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (no flush needed)"},
        "sequential_launches": {"gflops": round(flops / (seq_ms * 1e-3) / 1e9, 2),
                                "ms": round(seq_ms, 4)},
        "speedup_vs_sequential": round(seq_ms / ms, 3),
        "tune": {"route": "learned" if sel is not None else "fixed",
                 "t_pre_ms_total": round(t_tune, 1),
                 "plan": {"item_nnz": plan[0], "chunk_nnz": plan[1],
                          "t_tune_ms": round(t_plan, 1)}},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_kind": peak_kind, "alg_bytes": nbytes},
        "gpu_launches": args.steps * 2,
        "gather_ceiling": {"x_row_sectors": int(sectors), "probe_ms": round(t_g, 5),
                           "frac": round(t_g / ms, 4)},
        "learned": learned,
        "clocks": clocks.summary(),
        "gen_s": round(gen_s, 1),
    }
    B.close()
    return out


# The other full-size workloads of the method, measured in the same run as the headline so
# that one line carries them all: each matrix is generated, tuned by the profile route and
# timed like the headline, then tuned again by the learned route and timed.
OTHER_WORKLOADS = ("powerlaw_4m", "scattered_16m", "batched_512")
CLASS_NAMES = ("MB", "ML", "IMB", "CMP")


def _names(mask):
    return [n for b, n in enumerate(CLASS_NAMES) if mask >> b & 1]


def time_spmv(A, x, y, stream, K, W, world):
    """Milliseconds per SpMV over K back-to-back runs between CUDA events on `stream`, after W
    untimed ones (the slowest rank's time)."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(W):
            A.run(x, y, stream=stream)
        stream.synchronize()
        if world > 1:
            torch.distributed.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            A.run(x, y, stream=stream)
        e1.record(stream)
        e1.synchronize()
    return max_over_ranks(e0.elapsed_time(e1), world) / K


def fig3_one_pass(p: dict) -> list:
    """The class set of Fig. 3's rules on the first profiling pass alone (the paper's
    classifier), beside the two-pass set the profile route installs; same thresholds."""
    from paper_1711_05487_gb300 import _abi
    v = np.array([p[k] for k in ("P_CSR", "P_MB", "P_ML", "P_IMB", "P_CMP", "P_peak")])
    o = route_opts()
    thr = (o["t_imb"], o["t_ml"], o["t_mb"]) if o else (1.24, 1.25, 0.75)
    return _names(_abi.spmv_classify(v.ctypes.data, *thr))


def workload_summary(name, args, world, peak, sel):
    """One of the other full-size workloads: GFLOP/s, variant and classes of the profile
    route, algorithmic bytes and HBM roofline fraction, and the learned route beside it."""
    import torch

    from paper_1711_05487_gb300 import api
    if name == "batched_512":
        b = run_batched(args, 0, world)
        return {"desc": "512 mixed FP32 matrices, N log-uniform in [1e3, 2e5], k in {1, 4, 16}",
                "gflops": b["value"], "ms_per_step": b["ms_per_step"],
                "alg_bytes": b["roofline"]["alg_bytes"], "roofline_frac": b["roofline"]["frac"],
                "total_nnz": b["config"]["total_nnz"], "k_hist": b["config"]["k_hist"],
                "sequential_launches": b["sequential_launches"],
                "speedup_vs_sequential": b["speedup_vs_sequential"], "plan": b["tune"]["plan"],
                "learned": b["learned"], "gpu_launches": b["gpu_launches"],
                "gather_ceiling": b["gather_ceiling"],
                "clocks": b["clocks"], "gen_s": b["gen_s"]}
    wl = WORKLOADS[name]
    t0 = time.time()
    m = wl["make"]()
    gen_s = time.time() - t0
    stream = torch.cuda.Stream()
    A = api.SpmvMatrix.from_csr(m, stream=stream)
    vec_t = torch.float64 if m.val.dtype == np.float64 else torch.float32
    if m.val.dtype != np.float64:
        A.set_precision("f32", "f32", "f32", stream=stream)
    x = torch.from_numpy(synth.uniform_vector(m.n_cols, wl["x_seed"])).to(vec_t).cuda()
    y = torch.empty(m.n_rows, dtype=vec_t, device="cuda")
    flops = 2.0 * m.nnz
    A.set_variant(stream=stream)
    base_ms = time_spmv(A, x, y, stream, args.steps, args.warmup, world)
    rep = A.tune("profile", stream=stream, **route_opts())
    ms = time_spmv(A, x, y, stream, args.steps, args.warmup, world)
    ab = alg_bytes(m.n_rows, m.n_cols, m.nnz, rep.variant, A.storage, A.vec, A.handle)
    out = {"desc": wl["desc"], "n_rows": m.n_rows, "nnz": m.nnz,
           "dtype": {0: "f64", 1: "f32", 2: "bf16", 3: "df64"}[A.storage],
           "gflops": round(flops / (ms * 1e-3) / 1e9, 2), "ms_per_step": round(ms, 5),
           "variant": list(rep.variant), "classes": rep.class_names,
           "classes_fig3_one_pass": fig3_one_pass(rep.p), "t_pre_ms": round(rep.t_pre_ms, 2),
           "alg_bytes": ab, "achieved_gbs": round(ab / (ms * 1e-3) / 1e9, 1),
           "roofline_frac": round(ab / (ms * 1e-3) / 1e9 / peak, 4),
           "csr_vector": {"gflops": round(flops / (base_ms * 1e-3) / 1e9, 2),
                          "ms": round(base_ms, 5)},
           "speedup_vs_csr_vector": round(base_ms / ms, 3),
           "gpu_launches": args.steps * launches_per_spmv(A, rep.variant),
           "gen_s": round(gen_s, 1)}
    # the measured ceiling of this matrix's random x gathers: as many gathers, uniform over
    # an L2-resident x (at most 64 MB; the rate any variant that keeps its gathers in the L2,
    # such as column panels, can reach), and over an x of the matrix's own size; frac =
    # probe time / SpMV time
    if name in ("powerlaw_4m", "scattered_16m"):
        from paper_1711_05487_gb300 import _abi
        eb = 8 if vec_t == torch.float64 else 4
        n_l2 = min(m.n_cols, (64 << 20) // eb)
        t_g = _abi.spmv_probe_gather(n_l2, eb, m.nnz, 5)
        t_full = t_g if n_l2 == m.n_cols else _abi.spmv_probe_gather(m.n_cols, eb, m.nnz, 5)
        out["gather_ceiling"] = {"probe_ms": round(t_g, 5), "x_bytes": n_l2 * eb,
                                 "g_gathers_per_s": round(m.nnz / (t_g * 1e-3) / 1e9, 1),
                                 "frac": round(t_g / ms, 4),
                                 "full_x_probe_ms": round(t_full, 5)}
    if sel is not None:
        r_l = A.tune("learned", stream=stream, selector=sel, **route_opts())
        t_l = time_spmv(A, x, y, stream, args.steps, args.warmup, world)
        out["learned"] = {"decided_by": "mlp" if r_l.mode_used == 2 else "profile",
                          "margin": round(r_l.margin, 4), "classes": r_l.class_names,
                          "variant": list(r_l.variant), "t_pre_ms": round(r_l.t_pre_ms, 2),
                          "gflops": round(flops / (t_l * 1e-3) / 1e9, 2),
                          "ms_per_step": round(t_l, 5),
                          "t_learned_over_t_profile": round(t_l / ms, 4)}
    A.close()
    del x, y
    torch.cuda.synchronize()
    return out


def run_cg(args, rank, world):
    """Conjugate gradients on the SPD 27-point operator 160^3 (Section IV-D's solver setting):
    time to rtol with the plain CSR-vector handle and with tuned handles, and the iterations
    after which tuning pays for itself."""
    import torch

    from paper_1711_05487_gb300 import api

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    t0 = time.time()
    m = synth.laplacian_27pt(160)
    gen_s = time.time() - t0
    b = torch.from_numpy(synth.uniform_vector(m.n_rows, synth.SEED_BASE + 15)).cuda()
    rtol, max_iters, check = 1e-8, 5000, 25
    solves = max(1, min(args.steps, 5))
    peak, peak_kind = _peaks()

    def solve_runs(A):
        A.cg(b, max_iters=max_iters, rtol=rtol, check_every=check)       # warm-up
        times, rep = [], None
        for _ in range(solves):
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            _, rep = A.cg(b, max_iters=max_iters, rtol=rtol, check_every=check)
            times.append(max_over_ranks(rep["t_ms"], world))
        return float(np.median(times)), rep

    res = {}
    A = api.SpmvMatrix.from_csr(m)
    A.set_variant()
    t_plain, rep_plain = solve_runs(A)
    res["csr_vector"] = {"ms": round(t_plain, 3), "iters": rep_plain["iters"],
                         "ms_per_iter": round(t_plain / max(1, rep_plain["iters"]), 5),
                         "t_pre_ms": 0.0}
    clocks = ClockSampler(dev)
    clocks.start()
    tuned = None
    for name, prec in (("tuned_f64", None), ("tuned_df64", "df64")):
        if prec:
            A.set_precision(prec, "f64", prec)
        tr = A.tune("profile", **route_opts())
        t, rep = solve_runs(A)
        it = max(1, rep["iters"])
        gain = t_plain / max(1, rep_plain["iters"]) - t / it
        res[name] = {"ms": round(t, 3), "iters": rep["iters"], "ms_per_iter": round(t / it, 5),
                     "t_pre_ms": round(tr.t_pre_ms, 2), "variant": list(tr.variant),
                     "classes": tr.class_names, "converged": rep["converged"],
                     "breakeven_iters": round(tr.t_pre_ms / gain, 1) if gain > 0 else None,
                     "ms_with_tuning": round(t + tr.t_pre_ms, 3)}
        if tuned is None:
            tuned = (t, rep, tr)
    clocks.stop()
    t, rep, tr = tuned
    it = max(1, rep["iters"])
    spmv_b = alg_bytes(m.n_rows, m.n_cols, m.nnz, tr.variant, 0, 0)
    iter_b = spmv_b + 88 * m.n_rows     # + dot(p,Ap) 16N, x/r update 48N, p update 24N
    achieved = iter_b / (t / it * 1e-3) / 1e9
    return {
        "metric": "CG solve time to rtol 1e-8, SPD 27-point operator 160^3, tuned handle",
        "value": round(t, 3), "unit": "ms", "n_gpus": world, "steps": solves,
        "warmup": 1, "ms_per_step": round(t, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
        "config": {"workload": "cg27_160", "n_rows": m.n_rows, "nnz": m.nnz, "rtol": rtol,
                   "check_every": check, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (no flush needed)"},
        "solves": res,
        "speedup_vs_csr_vector": round(t_plain / t, 3),
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "peak_kind": peak_kind, "alg_bytes_per_iter": iter_b},
        "gpu_launches": solves * (it * 6 + 5),
        "clocks": clocks.summary(),
        "gen_s": round(gen_s, 1),
    }


def _time_rates(fn, nnz, budget_s):
    t = time.perf_counter()
    fn()
    one = time.perf_counter() - t
    reps = max(1, min(20, int(budget_s / max(one, 1e-6))))
    rates = []
    for _ in range(reps):
        t = time.perf_counter()
        fn()
        rates.append(2.0 * nnz / (time.perf_counter() - t) / 1e9)
    return rates


def cpu_baseline(m, x_host, budget_s=8.0):
    """The oracle's FP64 CSR SpMV on the host: the paper's static nnz-balanced baseline on all
    host cores (the headline), and the single-threaded loop."""
    import oracle
    oracle.lib()
    cores = os.cpu_count() or 1
    used = [1]

    def par():
        used[0] = oracle.spmv_static(m.rowptr, m.colind, m.val, x_host, cores)[1]

    rates = _time_rates(par, m.nnz, budget_s)
    rates1 = _time_rates(lambda: oracle.spmv(m.rowptr, m.colind, m.val, x_host), m.nnz, budget_s)
    return {"value": round(oracle.harmonic_mean(rates), 4), "unit": "GFLOP/s",
            "cores": used[0], "kind": "oracle", "build": "gcc " + " ".join(oracle.BUILD_FLAGS),
            "sample": f"full matrix, {len(rates)} SpMVs, harmonic mean of per-SpMV rates; "
                      "static nnz-balanced row partition, one range per thread",
            "single_thread": {"value": round(oracle.harmonic_mean(rates1), 4), "cores": 1,
                              "sample": f"full matrix, {len(rates1)} SpMVs"}}


# ---------------------------------------------------------------------- reference ----
def _oracle_build_flags():
    import oracle
    return "gcc " + " ".join(oracle.BUILD_FLAGS)


def _reference_line(args, metric, value, unit, higher, ms, config, cores, sample):
    return {
        "impl": "reference", "metric": metric, "value": value, "unit": unit,
        "n_gpus": args.gpus, "device": "host CPU (the oracle; no GPU work)",
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": higher, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)", "config": config,
        "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle",
                         "sample": sample, "build": _oracle_build_flags()},
        "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference_batched(args):
    """The batched workload on the oracle: each step is one pass of FP64 SpMM products over
    all matrices (FP32 values and X widened exactly), matrices spread over the host cores."""
    import concurrent.futures as cf

    import oracle
    oracle.lib()
    specs = synth.batched_specs(args.batch_count)
    cores = os.cpu_count() or 1
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        mats = list(ex.map(lambda sp: synth.make_from_spec(sp, dtype=np.float32), specs))
    Xs = [synth.uniform_vector(m.n_cols * sp["k"], sp["seed"], np.float32).reshape(m.n_cols, sp["k"])
          for sp, m in zip(specs, mats)]
    flops = sum(2.0 * m.nnz * sp["k"] for sp, m in zip(specs, mats))
    work = list(zip(mats, Xs))

    def one_pass(ex):
        list(ex.map(lambda mx: oracle.spmm(mx[0].rowptr, mx[0].colind, mx[0].val, mx[1]), work))

    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        for _ in range(args.warmup):
            one_pass(ex)
        t = time.perf_counter()
        for _ in range(args.steps):
            one_pass(ex)
        dt = (time.perf_counter() - t) / args.steps
    v = round(flops / dt / 1e9, 4)
    return _reference_line(
        args, "batched SpMV/SpMM GFLOP/s (sum of 2*nnz*k / t), one persistent launch", v,
        "GFLOP/s", True, round(dt * 1e3, 3),
        {"workload": f"batched_{len(mats)}", "matrices": len(mats), "flops_per_step": flops},
        cores, f"all {len(mats)} matrices per step, one FP64 SpMM per matrix, matrices spread "
               f"over {cores} threads")


def run_reference_cg(args):
    """Conjugate gradients on the oracle (single-threaded plain C): the iterations to rtol
    1e-8 come from one full solve; each step is a bounded sample of 25 iterations, and the
    reported time per solve is the sample's time per iteration times that count."""
    import oracle
    oracle.lib()
    m = synth.laplacian_27pt(160)
    b = synth.uniform_vector(m.n_rows, synth.SEED_BASE + 15)
    rtol, sample = 1e-8, 25
    _, iters, conv, _ = oracle.cg(m.rowptr, m.colind, m.val, b, max_iters=5000, rtol=rtol)
    for _ in range(args.warmup):
        oracle.cg(m.rowptr, m.colind, m.val, b, max_iters=sample, rtol=0.0)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.cg(m.rowptr, m.colind, m.val, b, max_iters=sample, rtol=0.0)
    per_iter = (time.perf_counter() - t) / (args.steps * sample)
    ms = round(per_iter * iters * 1e3, 3)
    return _reference_line(
        args, "CG solve time to rtol 1e-8, SPD 27-point operator 160^3, tuned handle", ms, "ms",
        False, ms, {"workload": "cg27_160", "n_rows": m.n_rows, "nnz": m.nnz, "rtol": rtol,
                    "iters": iters, "converged": bool(conv)},
        1, f"{sample} CG iterations per step, scaled to the {iters} iterations the oracle "
           f"needs to reach rtol {rtol}")


def cpu_baseline_batched(args):
    """The oracle's side of the batched line: two timed passes of FP64 SpMM products over the
    whole batch on the host cores (the reference arm's computation)."""
    import argparse as _ap
    ref = run_reference_batched(_ap.Namespace(batch_count=args.batch_count, warmup=1, steps=2,
                                              gpus=1))
    cb = dict(ref["cpu_baseline"])
    cb["sample"] = "whole batch, 2 passes: " + cb["sample"]
    return cb


def cpu_baseline_cg(iters, sample=25):
    """The oracle's side of the CG line: time per iteration of the oracle's conjugate
    gradients (single-threaded) over `sample` iterations, times the timed solve's count."""
    import oracle
    oracle.lib()
    m = synth.laplacian_27pt(160)
    b = synth.uniform_vector(m.n_rows, synth.SEED_BASE + 15)
    oracle.cg(m.rowptr, m.colind, m.val, b, max_iters=2, rtol=0.0)          # warm-up
    t = time.perf_counter()
    oracle.cg(m.rowptr, m.colind, m.val, b, max_iters=sample, rtol=0.0)
    per_iter = (time.perf_counter() - t) / sample
    return {"value": round(per_iter * iters * 1e3, 3), "unit": "ms", "cores": 1,
            "kind": "oracle", "build": _oracle_build_flags(),
            "sample": f"{sample} CG iterations of the oracle on the same operator, scaled to "
                      f"the {iters} iterations of the timed solve"}


def run_reference(args):
    """The oracle (plain FP64 CPU CSR SpMV over the paper's static nnz-balanced row
    partition, one range per host core), timed on the host: --steps SpMVs of the same
    workload after --warmup untimed ones."""
    if args.workload == "batched_512":
        return run_reference_batched(args)
    if args.workload == "cg27_160":
        return run_reference_cg(args)
    import oracle
    oracle.lib()
    wl = WORKLOADS[args.workload]
    m = wl["make"]()
    x = synth.uniform_vector(m.n_cols, wl["x_seed"]).astype(np.float64)
    cores = os.cpu_count() or 1
    used = 1
    for _ in range(args.warmup):
        used = oracle.spmv_static(m.rowptr, m.colind, m.val, x, cores)[1]
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.spmv_static(m.rowptr, m.colind, m.val, x, cores)
    dt = (time.perf_counter() - t) / args.steps
    v = 2.0 * m.nnz / dt / 1e9
    return {
        "impl": "reference", "metric": "SpMV GFLOP/s (2*nnz/t), adaptive (profile-guided) vs "
        "plain CSR-vector", "value": round(v, 4), "unit": "GFLOP/s", "n_gpus": args.gpus,
        "device": "host CPU (the oracle; no GPU work)",
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": args.workload, "desc": wl["desc"], "n_rows": m.n_rows,
                   "nnz": m.nnz},
        "cpu_baseline": {"value": round(v, 4), "unit": "GFLOP/s", "cores": used,
                         "kind": "oracle", "build": _oracle_build_flags(),
                         "sample": f"full matrix, {args.steps} SpMVs, static nnz-balanced "
                                   "row partition, one range per thread"},
        "e2e": {"value": round(v, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=128)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS) + ["batched_512", "cg27_160"],
                    default="stencil27_160")
    ap.add_argument("--batch-count", type=int, default=512,
                    help="matrices in the batched workload (512; fewer for profiling)")
    ap.add_argument("--quick", action="store_true", help="skip the precision variants")
    ap.add_argument("--precision", choices=["native", "df64", "f32", "bf16"], default="native",
                    help="FP64 workloads: native FP64 arithmetic, double-float (df64) storage "
                         "and arithmetic, or FP32 / BF16 value storage with FP32 x and "
                         "accumulation, for the timed line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--probe-gather", action="store_true",
                    help="print the random-gather ceiling for x sizes from 4 MB to 1 GB (one "
                         "JSON line per size) and exit")
    ap.add_argument("--probe-fma", action="store_true",
                    help="print the FP64 and FP32 FMA rates of register-only chains by chains "
                         "per thread and warps per SM (one JSON line each) and exit")
    ap.add_argument("--fixed-variant", default=None,
                    help="install this variant instead of tuning: partition,index,xpath,vec,"
                         "vs,tile_rows,tile_pipe")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.probe_gather:
        import torch

        from paper_1711_05487_gb300 import _abi
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        count = 1 << 27
        for n_x, eb in ((1 << 20, 4), (4 << 20, 4), (16 << 20, 4), (4 << 20, 8), (8 << 20, 8),
                        (12 << 20, 8), (16 << 20, 8), (64 << 20, 8), (1 << 28, 4)):
            ms = _abi.spmv_probe_gather(n_x, eb, count, 5)
            print(json.dumps({"n_x": n_x, "elem_bytes": eb, "x_mb": n_x * eb / 2 ** 20,
                              "gathers": count, "ms": round(ms, 5),
                              "g_gathers_per_s": round(count / (ms * 1e-3) / 1e9, 1)}),
                  flush=True)
        return
    if args.probe_fma:
        import torch

        from paper_1711_05487_gb300 import _abi
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        for eb in (8, 4):
            for w in (4, 8, 16, 24, 32, 48, 64):
                for c in (1, 2, 4):
                    r = _abi.spmv_probe_fma(eb, c, w, 5)
                    print(json.dumps({"elem_bytes": eb, "chains": c, "warps_per_sm": w,
                                      "g_fma_per_s": round(r / 1e9, 1)}), flush=True)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            # bounded samples: the default run ends within a few minutes on the host cores
            cap = 3 if args.workload == "batched_512" else (5 if args.workload == "cg27_160"
                                                            else 20)
            args.steps = max(1, min(args.steps, cap))
            print(json.dumps(run_reference(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    if args.workload in ("batched_512", "cg27_160"):
        out = (run_batched if args.workload == "batched_512" else run_cg)(args, rank, world)
        if rank == 0:
            if not args.no_cpu_baseline and world == 1:      # the oracle baseline: N = 1 only
                out["cpu_baseline"] = (
                    cpu_baseline_batched(args) if args.workload == "batched_512"
                    else cpu_baseline_cg(out["solves"]["tuned_f64"]["iters"]))
            print(json.dumps(out), flush=True)
        return
    out, m = run_ours(args, rank, world)
    if rank == 0 and not args.no_cpu_baseline and world == 1:   # the oracle: N = 1 only
        wl = WORKLOADS[args.workload]
        out["cpu_baseline"] = cpu_baseline(m, synth.uniform_vector(m.n_cols, wl["x_seed"]))
    del m
    if args.workload == "stencil27_160" and not args.quick and not args.fixed_variant:
        from paper_1711_05487_gb300 import api
        sel_path = os.path.join(ROOT, "paper_1711_05487_gb300", "data", "selector_gb300.npz")
        sel = api.Selector.load(sel_path) if os.path.exists(sel_path) else None
        peak, _ = _peaks()
        out["workloads"] = {name: workload_summary(name, args, world, peak, sel)
                            for name in OTHER_WORKLOADS}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
