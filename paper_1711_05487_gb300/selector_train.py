"""Learned selector: training data, GPU training and evaluation.

The paper trains its feature-guided classifier on matrices labelled by the profile-guided
classifier (Section III-D, "Training Data Labeling") and scores it with the exact and partial
match ratios (Section IV-B) and by the speed of the optimizations it selects (Section IV-C,
against the "oracle" that always picks the best). This module does the same with an MLP
trained on the GPU by the library's own kernels:

  1. for each seeded mixed matrix: Table I features (GPU), the profile route's class set (the
     label), and the time of every pool variant the class sets can select (the exhaustive
     sweep that measures regret);
  2. standardize the MLP inputs on the training split and train with full-batch Adam
     (spmv_mlp_train: forward, backward and update kernels);
  3. on the held-out split: match ratios against the profile labels, and the geometric means
     of t(MLP choice) / t(profile choice), t(MLP choice) / t(best variant) and
     t(plain CSR-vector) / t(MLP choice).

Run as a module to build a dataset, train, evaluate and save the selector:

  python -m paper_1711_05487_gb300.selector_train --count 2000 --out DIR
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import math
import os
import time

import numpy as np
import torch

from . import _abi
from .api import Selector, SpmvMatrix

# Every variant a class set can select (partition, index, xpath, vec) with the pool's
# sub-warp width heuristic; index 0 is the plain CSR-vector.
CANDIDATES = ((0, 0, 0, 0), (0, 0, 0, 1), (0, 1, 0, 1), (0, 0, 1, 0), (0, 0, 1, 1),
              (0, 1, 1, 1), (1, 0, 0, 0), (1, 0, 1, 0), (2, 0, 0, 1), (2, 0, 1, 1))
SIZES = (12, 32, 32, 4)


def _time_variant(A: SpmvMatrix, x, y, knobs, reps: int, bin_med: int = 0,
                  bin_chunk: int = 0) -> float:
    A.set_variant(partition=knobs[0], index=knobs[1], xpath=knobs[2], vec=knobs[3],
                  bin_med=bin_med if knobs[0] == 2 else 0,
                  bin_chunk=bin_chunk if knobs[0] == 2 else 0)
    for _ in range(2):
        A.run(x, y)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        A.run(x, y)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_matrix(m, reps: int = 5) -> dict:
    """Features, profile label and the time of every candidate variant for one matrix."""
    A = SpmvMatrix.from_csr(m)
    t0 = time.perf_counter()
    f, _ = A.features()
    torch.cuda.synchronize()
    t_feat = (time.perf_counter() - t0) * 1e3
    rep = A.tune("profile", reps=reps, autotune=0)
    x = torch.ones(m.n_cols, dtype=A.vec_dtype, device="cuda")
    y = torch.empty(m.n_rows, dtype=A.vec_dtype, device="cuda")
    times = [_time_variant(A, x, y, c, reps) for c in CANDIDATES]
    lens = np.diff(m.rowptr)
    # the row decomposition at every pair of limits the grid search tries, for matrices
    # uneven enough that some ratio of the grid sends them to the decomposition
    from .calibrate import BIN_GRID, GRID
    t_bins = np.zeros((2, len(BIN_GRID)))
    uneven = lens.size and lens.max() > min(GRID["long_ratio"]) * lens.mean()
    for xp in (0, 1):
        base = times[CANDIDATES.index((2, 0, xp, 1))]
        for b, (l_med, chunk) in enumerate(BIN_GRID):
            t_bins[xp, b] = (_time_variant(A, x, y, (2, 0, xp, 1), reps, l_med, chunk)
                             if uneven else base)
    feat16 = np.concatenate([f, [float(m.n_rows), float(m.nnz)]])
    out = {"feat16": feat16, "classes": rep.classes, "p": [rep.p[k] for k in rep.p],
           "p2": list(rep.p2), "times": times, "times_bins": t_bins,
           "t_pre_profile_ms": rep.t_pre_ms, "t_features_ms": t_feat,
           "nnz_avg": float(lens.mean()) if lens.size else 0.0,
           "nnz_max": float(lens.max()) if lens.size else 0.0, "name": m.name}
    A.close()
    return out


def build_dataset(count: int, seed: int, n_lo: int, n_hi: int, reps: int = 5,
                  workers: int = 8, log=print) -> dict:
    """Generates the mixed set on host threads (numpy releases the GIL) while the GPU
    measures the matrices in order."""
    import synth
    specs = [synth.mixed_spec(i, seed=seed, n_lo=n_lo, n_hi=n_hi) for i in range(count)]
    rows = []
    t0 = time.time()
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {}
        nxt = 0
        for i in range(count):
            while nxt < count and nxt < i + 2 * workers:
                futs[nxt] = ex.submit(synth.make_from_spec, specs[nxt])
                nxt += 1
            m = futs.pop(i).result()
            r = measure_matrix(m, reps)
            r["family"] = specs[i]["family"]
            rows.append(r)
            del m
            if log and (i + 1) % 100 == 0:
                log(f"measured {i + 1}/{count} in {time.time() - t0:.0f}s")
    return {
        "feat16": np.stack([r["feat16"] for r in rows]),
        "classes": np.array([r["classes"] for r in rows], dtype=np.int32),
        "p": np.array([r["p"] for r in rows]),
        "p2": np.array([r["p2"] for r in rows]),
        "times": np.array([r["times"] for r in rows]),
        "times_bins": np.stack([r["times_bins"] for r in rows]),
        "t_pre_profile_ms": np.array([r["t_pre_profile_ms"] for r in rows]),
        "t_features_ms": np.array([r["t_features_ms"] for r in rows]),
        "nnz_avg": np.array([r["nnz_avg"] for r in rows]),
        "nnz_max": np.array([r["nnz_max"] for r in rows]),
        "family": np.array([r["family"] for r in rows]),
    }


# ----------------------------------------------------------------------- training ----
def _inputs(feat16: np.ndarray, mu=None, inv=None) -> np.ndarray:
    f = torch.from_numpy(np.ascontiguousarray(feat16, dtype=np.float64)).cuda()
    X = torch.empty((feat16.shape[0], _abi.MLP_INPUTS), dtype=torch.float32, device="cuda")
    mud = None if mu is None else torch.from_numpy(np.asarray(mu, np.float32)).cuda()
    ivd = None if inv is None else torch.from_numpy(np.asarray(inv, np.float32)).cuda()
    _abi.spmv_mlp_inputs(f.data_ptr(), feat16.shape[0], None if mud is None else mud.data_ptr(),
                         None if ivd is None else ivd.data_ptr(), X.data_ptr(), 0)
    torch.cuda.synchronize()
    return X.cpu().numpy()


def class_bits(classes: np.ndarray) -> np.ndarray:
    c = np.asarray(classes, dtype=np.int64)
    return np.stack([(c >> b) & 1 for b in range(4)], axis=1).astype(np.float32)


def init_params(sizes=SIZES, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for i in range(3):
        fan_in, fan_out = sizes[i], sizes[i + 1]
        parts.append(rng.standard_normal(fan_out * fan_in) * math.sqrt(2.0 / fan_in))
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def train(feat16: np.ndarray, classes: np.ndarray, steps: int = 3000, lr: float = 3e-3,
          seed: int = 0, sizes=SIZES):
    """Standardize inputs on this (training) set and train with full-batch Adam on the GPU.
    Returns (params, mu, inv_sigma, loss history)."""
    raw = _inputs(feat16)
    mu = raw.mean(axis=0).astype(np.float32)
    sd = raw.std(axis=0)
    inv = (1.0 / np.where(sd > 1e-3, sd, 1.0)).astype(np.float32)
    X = torch.from_numpy(_inputs(feat16, mu, inv)).cuda()
    Y = torch.from_numpy(class_bits(classes)).cuda()
    sizes_h = np.asarray(sizes, dtype=np.int32)
    w = torch.from_numpy(init_params(sizes, seed)).cuda()
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    hist = torch.empty(steps, dtype=torch.float32, device="cuda")
    _abi.spmv_mlp_train(sizes_h.ctypes.data, w.data_ptr(), m.data_ptr(), v.data_ptr(),
                        X.shape[0], X.data_ptr(), Y.data_ptr(), steps, 0, lr, 0.9, 0.999, 1e-8,
                        hist.data_ptr(), 0)
    return w.cpu().numpy(), mu, inv, hist.cpu().numpy()


def predict(params, mu, inv, feat16, sizes=SIZES) -> tuple[np.ndarray, np.ndarray]:
    """Class sets (logit > 0 per class) and logits for a batch, computed on the GPU."""
    X = torch.from_numpy(_inputs(feat16, mu, inv)).cuda()
    w = torch.from_numpy(np.asarray(params, np.float32)).cuda()
    L = torch.empty((feat16.shape[0], sizes[3]), dtype=torch.float32, device="cuda")
    sizes_h = np.asarray(sizes, dtype=np.int32)
    _abi.spmv_mlp_logits(sizes_h.ctypes.data, w.data_ptr(), feat16.shape[0], X.data_ptr(),
                         L.data_ptr(), 0)
    torch.cuda.synchronize()
    lg = L.cpu().numpy()
    masks = np.zeros(lg.shape[0], dtype=np.int32)
    for b in range(lg.shape[1]):
        masks |= (lg[:, b] > 0).astype(np.int32) << b
    return masks, lg


# --------------------------------------------------------------------- evaluation ----
def family_times(t: np.ndarray) -> np.ndarray:
    """Times with each merge-path candidate replaced by the faster of it and the row
    decomposition with the same x path: the autotuner picks between the two decompositions
    for IMB matrices."""
    t = np.array(t, dtype=np.float64, copy=True)
    if t.shape[1] < len(CANDIDATES):
        return t
    for xp in (0, 1):
        m, b = CANDIDATES.index((1, 0, xp, 0)), CANDIDATES.index((2, 0, xp, 1))
        t[:, m] = np.minimum(t[:, m], t[:, b])
    return t


def candidate_of(classes: int, nnz_avg: float, nnz_max: float, long_ratio: float = 32.0) -> int:
    """Index in CANDIDATES of the variant Table II maps the class set to."""
    v = _abi.spmv_variant_for_classes(int(classes), nnz_avg, nnz_max, long_ratio)
    if v.partition == 1:          # merge-path tiles use neither the delta index nor widths
        return CANDIDATES.index((1, 0, v.xpath, 0))
    return CANDIDATES.index((v.partition, v.index, v.xpath, v.vec))


def _gmean(a) -> float:
    a = np.asarray(a, dtype=np.float64)
    return float(np.exp(np.mean(np.log(a)))) if a.size else float("nan")


def match_ratios(pred: np.ndarray, lab: np.ndarray, bits: int = 0xF) -> tuple[float, float]:
    """Section IV-B: exact match ratio (every class of the set right) and partial match
    ratio (at least one class in common, or both sets empty), over the class bits in
    `bits`."""
    p, q = np.asarray(pred) & bits, np.asarray(lab) & bits
    emr = float(np.mean(p == q)) if p.size else float("nan")
    pmr = float(np.mean(((p & q) != 0) | ((p == 0) & (q == 0)))) if p.size else float("nan")
    return emr, pmr


def varying_bits(lab: np.ndarray) -> int:
    """The class bits that are not the same in every label (a bit every label carries, or
    none does, makes every prediction that copies it match trivially)."""
    lab = np.asarray(lab)
    bits = 0
    for b in range(4):
        v = (lab >> b) & 1
        if v.size and v.min() != v.max():
            bits |= 1 << b
    return bits


def evaluate(ds: dict, idx: np.ndarray, pred: np.ndarray) -> dict:
    """Section IV-B match ratios (over all four classes, and over the classes whose bit
    varies among the labels) and Section IV-C speed of the selected variants: regret of the
    profile route's and of the MLP's choice against the best candidate."""
    from .calibrate import times_at
    lab = ds["classes"][idx]
    ratio = float(ds.get("long_ratio", 32.0))
    emr, pmr = match_ratios(pred, lab)
    vb = varying_bits(ds["classes"])
    emr_v, pmr_v = match_ratios(pred, lab, vb)
    t = times_at(ds, idx, tuple(ds.get("bins", (64, 4096))))
    ch_ml = np.array([candidate_of(c, a, mx, ratio) for c, a, mx in
                      zip(pred, ds["nnz_avg"][idx], ds["nnz_max"][idx])])
    ch_pr = np.array([candidate_of(c, a, mx, ratio) for c, a, mx in
                      zip(lab, ds["nnz_avg"][idx], ds["nnz_max"][idx])])
    r = np.arange(len(idx))
    t_ml, t_pr, t_best, t_base = t[r, ch_ml], t[r, ch_pr], t.min(axis=1), t[:, 0]
    names = ("MB", "ML", "IMB", "CMP")
    return {"n": int(len(idx)), "exact_match_ratio": emr, "partial_match_ratio": pmr,
            "varying_classes": [names[b] for b in range(4) if vb >> b & 1],
            "exact_match_ratio_varying": emr_v, "partial_match_ratio_varying": pmr_v,
            "class_accuracy": {names[b]: float(np.mean(((pred >> b) & 1) == ((lab >> b) & 1)))
                               for b in range(4)},
            "gmean_t_mlp_over_t_profile": _gmean(t_ml / t_pr),
            "gmean_t_mlp_over_t_best": _gmean(t_ml / t_best),
            "gmean_t_profile_over_t_best": _gmean(t_pr / t_best),
            "frac_mlp_within_5pct_of_best": float(np.mean(t_ml <= 1.05 * t_best)),
            "frac_profile_within_5pct_of_best": float(np.mean(t_pr <= 1.05 * t_best)),
            "max_t_mlp_over_t_profile": float(np.max(t_ml / t_pr)) if len(idx) else float("nan"),
            "gmean_speedup_mlp_vs_csr_vector": _gmean(t_base / t_ml),
            "gmean_speedup_profile_vs_csr_vector": _gmean(t_base / t_pr),
            "gmean_speedup_best_vs_csr_vector": _gmean(t_base / t_best),
            "label_histogram": {int(k): int(v) for k, v in
                                zip(*np.unique(lab, return_counts=True))}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=171105487 + 40)
    ap.add_argument("--n-lo", type=int, default=1_000)
    ap.add_argument("--n-hi", type=int, default=4_000_000)
    ap.add_argument("--slack", type=float, default=1.0,
                    help="standardized units an input may leave the training range by")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--train-frac", type=float, default=0.8)
    ap.add_argument("--workers", type=int, default=12)
    ap.add_argument("--dataset", default=None, help="reuse a saved dataset (.npz)")
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    t0 = time.time()
    if args.dataset:
        z = np.load(args.dataset, allow_pickle=False)
        ds = {k: z[k] for k in z.files}
    else:
        ds = build_dataset(args.count, args.seed, args.n_lo, args.n_hi, args.reps, args.workers)
        np.savez(os.path.join(args.out, "selector_dataset.npz"), **ds)
    t_data = time.time() - t0
    n = ds["classes"].shape[0]
    # split by seed order: the first train_frac of the indices train, the rest test
    n_tr = int(round(args.train_frac * n))
    tr, te = np.arange(n_tr), np.arange(n_tr, n)
    # thresholds of the profile route calibrated on the training split (Section III-C grid
    # search), then the labels the network learns are the calibrated route's class sets
    cal = None
    if "p2" in ds:
        from . import calibrate
        cal = calibrate.calibrate(ds, tr, te)
        ds = dict(ds)
        ds["classes_paper"] = ds["classes"]
        ds["classes"] = calibrate.classes_for(ds, np.arange(n),
                                              [cal[k] for k in calibrate.KEYS])
        ds["long_ratio"] = cal["long_ratio"]
        ds["bins"] = (cal["bin_med"], cal["bin_chunk"])
    t1 = time.time()
    params, mu, inv, hist = train(ds["feat16"][tr], ds["classes"][tr], steps=args.steps)
    t_train = time.time() - t1
    pred_te, _ = predict(params, mu, inv, ds["feat16"][te])
    pred_tr, _ = predict(params, mu, inv, ds["feat16"][tr])
    res = {"train": evaluate(ds, tr, pred_tr), "test": evaluate(ds, te, pred_te),
           "calibration": cal,
           "loss_first": float(hist[0]), "loss_last": float(hist[-1]),
           "t_dataset_s": t_data, "t_train_s": t_train, "count": int(n),
           "t_pre_profile_ms_median": float(np.median(ds["t_pre_profile_ms"])),
           "t_features_ms_median": float(np.median(ds["t_features_ms"]))}
    # the training range of the standardized inputs: the learned route profiles matrices
    # outside it instead of extrapolating
    x_tr = _inputs(ds["feat16"][tr], mu, inv)
    sel = Selector(SIZES, params, mu, inv, x_tr.min(axis=0), x_tr.max(axis=0), args.slack)
    sel.save(os.path.join(args.out, "selector_gb300.npz"))
    te_in = np.array([sel.predict(f)[1] >= 0.0 for f in ds["feat16"][te]])
    res["test_inside_training_range"] = float(np.mean(te_in))
    if cal is not None:
        with open(os.path.join(args.out, "calibration_gb300.json"), "w") as fh:
            json.dump(cal, fh, indent=1)
    with open(os.path.join(args.out, "selector_metrics.json"), "w") as fh:
        json.dump(res, fh, indent=1)
    print(json.dumps(res))


if __name__ == "__main__":
    main()
