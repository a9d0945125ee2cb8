"""The Section III-C grid search (calibrate.py) on a synthetic label set whose best setting is
known by construction.

Each synthetic matrix has a P-vector whose class set flips at exactly one grid threshold and
candidate times that make one side of the flip the better one, so the setting that maximizes
the mean gain is unique: T_IMB = 1.15, T_ML = 1.25, T_MB = 0.8, uneven-rows ratio 16 and row
decomposition limits (128, 2048). A held-out copy with perturbed P-vectors is scored beside
the paper's setting. Runs on the CPU: the classifier and the class-to-variant map are the
library's host functions."""
import numpy as np
import pytest

from paper_1711_05487_gb300 import calibrate
from paper_1711_05487_gb300.selector_train import CANDIDATES, match_ratios, varying_bits

BEST = (1.15, 1.25, 0.8, 16.0, 128, 2048)
I_MERGE, I_BINS, I_ML, I_MB = (CANDIDATES.index((1, 0, 0, 0)), CANDIDATES.index((2, 0, 0, 1)),
                               CANDIDATES.index((0, 0, 1, 0)), CANDIDATES.index((0, 1, 0, 1)))


def _matrix(p, nnz_max, times=None, bins=1.0):
    t = np.ones(len(CANDIDATES))
    for k, v in (times or {}).items():
        t[k] = v
    tb = np.full((2, len(calibrate.BIN_GRID)), float(bins) if np.isscalar(bins) else 1.0)
    if not np.isscalar(bins):
        tb[0] = bins
    return dict(p=np.array(p, float), p2=np.zeros(2), times=t, times_bins=tb,
                nnz_avg=10.0, nnz_max=float(nnz_max))


def _dataset(imb=(1.2, 1.12), ml=(1.3, 1.2), mb=(8.5, 7.8)):
    b_star = calibrate.BIN_GRID.index((128, 2048))
    r1_bins = np.full(len(calibrate.BIN_GRID), 0.5)
    r1_bins[b_star] = 0.25
    rows = [
        # IMB flips at T_IMB = P_IMB / P_CSR; merge-path tiles help the first, hurt the second
        _matrix([1, 10, 1, imb[0], 20, 30], 1000, {I_MERGE: 0.5}),
        _matrix([1, 10, 1, imb[1], 20, 30], 1000, {I_MERGE: 2.0, I_BINS: 2.0}, bins=2.0),
        # ML flips at T_ML = P_ML / P_CSR
        _matrix([1, 10, ml[0], 1, 20, 30], 10, {I_ML: 0.5}),
        _matrix([1, 10, ml[1], 1, 20, 30], 10, {I_ML: 2.0}),
        # MB flips at T_MB = P_CSR / P_MB (P_MB < P_CMP < P_peak holds)
        _matrix([mb[0], 10, 1, 1, 20, 30], 10, {I_MB: 0.5}),
        _matrix([mb[1], 10, 1, 1, 20, 30], 10, {I_MB: 2.0}),
        # always IMB; the decomposition is taken when nnz_max > ratio * nnz_avg: it helps at
        # ratio 20 (fastest at limits (128, 2048)), hurts at ratio 12
        _matrix([1, 10, 1, 5, 20, 30], 200, {I_MERGE: 2.0, I_BINS: 0.5}, bins=r1_bins),
        _matrix([1, 10, 1, 5, 20, 30], 120, {I_MERGE: 2.0, I_BINS: 2.0}, bins=2.0),
    ]
    return {k: np.stack([r[k] for r in rows]) for k in rows[0]}


def _concat(a, b):
    return {k: np.concatenate([a[k], b[k]]) for k in a}


def test_grid_search_finds_the_constructed_optimum():
    ds = _dataset()
    res = calibrate.grid_search(ds, np.arange(8))
    assert res["best"] == BEST
    # the best setting's gain, recomputed directly: 2 + 1 + 2 + 1 + 2 + 1 + 4 + 1 over 8
    assert res["best_gain"] == pytest.approx(14 / 8)
    assert calibrate.mean_gain(ds, np.arange(8), BEST) == pytest.approx(14 / 8)
    # the paper's setting: no IMB flip at 1.24, MB taken for both at 0.75, no decomposition
    # at ratio 32: 1 + 1 + 2 + 1 + 2 + 0.5 + 1 + 1 over 8
    assert res["paper_gain"] == pytest.approx(9.5 / 8)
    # the optimum is unique: every other setting scores lower
    gains = sorted((g for _, g in res["table"]), reverse=True)
    assert gains[0] > gains[1] + 1e-9


def test_calibrate_scores_the_held_out_split():
    train = _dataset()
    test = _dataset(imb=(1.19, 1.11), ml=(1.28, 1.18), mb=(8.3, 7.7))   # same sides of the flips
    ds = _concat(train, test)
    rec = calibrate.calibrate(ds, np.arange(8), np.arange(8, 16))
    assert tuple(rec[k] for k in calibrate.KEYS) == BEST
    assert rec["test_mean_gain"] == pytest.approx(14 / 8)
    assert rec["paper_test_mean_gain"] == pytest.approx(9.5 / 8)
    assert rec["n_train"] == 8 and rec["n_test"] == 8


def test_grid_search_without_bin_timings_keeps_default_limits():
    ds = _dataset()
    del ds["times_bins"]
    res = calibrate.grid_search(ds, np.arange(8))
    assert res["best"][4:] == (64, 4096)
    assert res["best"][:3] == BEST[:3]


def test_match_ratios_over_varying_bits():
    # every label carries CMP (bit 8): over all bits any prediction with CMP matches
    # partially; over the varying bits only real matches count
    lab = np.array([8 | 4, 8 | 1, 8, 8 | 2])
    pred = np.array([8, 8, 8, 8])
    assert match_ratios(pred, lab) == (0.25, 1.0)
    vb = varying_bits(lab)
    assert vb == 1 | 2 | 4
    assert match_ratios(pred, lab, vb) == (0.25, 0.25)
