"""Calibration of the profile route's thresholds on the target GPU.

The paper sets T_ML and T_IMB by an exhaustive grid search that maximizes the average
performance gain of the optimizations selected on a large matrix set (Section III-C). With
the per-matrix P-vectors (both profiling passes) and the measured time of every candidate
variant, each threshold triple (T_IMB, T_ML, T_MB) is scored by classifying every matrix with
the library's own classifier (spmv_classify2), mapping the class set to its variant (Table
II) and averaging t(plain CSR-vector) / t(selected variant).
"""
from __future__ import annotations

import itertools

import numpy as np

from . import _abi

PAPER = (1.24, 1.25, 0.75)
GRID = {
    "t_imb": (1.05, 1.1, 1.15, 1.24, 1.35, 1.5, 2.0, 3.0),
    "t_ml": (1.02, 1.05, 1.1, 1.15, 1.25, 1.4, 1.6, 2.0),
    "t_mb": (0.4, 0.5, 0.6, 0.7, 0.75, 0.8, 0.9, 1.01),
}


def classes_for(ds: dict, idx, thr) -> np.ndarray:
    t_imb, t_ml, t_mb = thr
    out = np.zeros(len(idx), dtype=np.int32)
    for k, i in enumerate(idx):
        p = np.ascontiguousarray(ds["p"][i], dtype=np.float64)
        p2 = np.ascontiguousarray(ds["p2"][i], dtype=np.float64)
        out[k] = _abi.spmv_classify2(p.ctypes.data, p2.ctypes.data, t_imb, t_ml, t_mb)
    return out


def _candidate(cls, nnz_avg, nnz_max):
    from .selector_train import candidate_of
    return candidate_of(int(cls), float(nnz_avg), float(nnz_max))


def mean_gain(ds: dict, idx, thr) -> float:
    idx = np.asarray(idx)
    cls = classes_for(ds, idx, thr)
    ch = np.array([_candidate(c, a, m) for c, a, m in
                   zip(cls, ds["nnz_avg"][idx], ds["nnz_max"][idx])])
    from .selector_train import family_times
    t = family_times(ds["times"][idx])
    return float(np.mean(t[:, 0] / t[np.arange(len(idx)), ch]))


def grid_search(ds: dict, idx) -> dict:
    best, best_gain = PAPER, -1.0
    table = []
    for thr in itertools.product(GRID["t_imb"], GRID["t_ml"], GRID["t_mb"]):
        g = mean_gain(ds, idx, thr)
        table.append((thr, g))
        if g > best_gain + 1e-12:
            best, best_gain = thr, g
    return {"best": tuple(float(v) for v in best), "best_gain": best_gain,
            "paper_gain": mean_gain(ds, idx, PAPER), "table": table}
