"""Pins of the oracle's Table I features, Section III-B bounds, Fig. 3 classifier,
Table II map, Section IV metrics and the MLP selector's arithmetic."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


# --------------------------------------------------------------------- features
def test_features_hand_example():
    # rows: [0,1,2,5], [], [7], [1,3,4,7]; 8 columns; a "cache line" of 2 elements
    rp = np.array([0, 4, 4, 5, 9], np.int32)
    ci = np.array([0, 1, 2, 5, 7, 1, 3, 4, 7], np.int32)
    f, isum = oracle.features(4, 8, rp, ci, line_elems=2, ws_bytes=10, llc_bytes=10)
    d = dict(zip(oracle.FEATURE_NAMES, f))
    assert d["size"] == 1.0
    assert d["density"] == 9 / 32
    assert (d["nnz_min"], d["nnz_max"], d["nnz_avg"]) == (0, 4, 2.25)
    assert d["nnz_sd"] == math.sqrt(3.1875)
    assert (d["bw_min"], d["bw_max"], d["bw_avg"]) == (0, 7, 3.5)
    assert d["bw_sd"] == math.sqrt(9.25)
    scatter = [Fraction(4, 6), 0, Fraction(1), Fraction(4, 7)]
    exact_avg = float(sum(scatter) / 4)
    assert abs(d["scatter_avg"] - exact_avg) <= 2 ** -24
    mean = sum(scatter) / 4
    exact_sd = math.sqrt(float(sum((s - mean) ** 2 for s in scatter) / 4))
    assert abs(d["scatter_sd"] - exact_sd) <= 2 ** -22
    assert d["clustering_avg"] == 0.5625        # (1/2 + 0 + 1 + 3/4) / 4
    assert d["misses_avg"] == 1.25              # (2 + 0 + 1 + 2) / 4
    assert isum[0] == 9 and isum[1] == 14 and isum[4] == 5 and isum[5] == 6


def test_features_laplacian_closed_forms():
    n = 256
    m = synth.laplacian_2d(n)
    f, _ = oracle.features(m.n_rows, m.n_cols, m.rowptr, m.colind, line_elems=16,
                           ws_bytes=1 << 40, llc_bytes=1 << 20)
    d = dict(zip(oracle.FEATURE_NAMES, f))
    assert d["size"] == 0.0
    assert (d["nnz_min"], d["nnz_max"]) == (3, 5)
    assert d["nnz_avg"] == 326656 / 65536
    assert d["bw_max"] == 2 * n + 1
    assert d["bw_min"] == n + 1           # corner rows: [r, r+1, r+n] or [r-n, r-1, r]
    # first and last grid rows have 2 misses, all others 3 (the jumps of n columns)
    assert d["misses_avg"] == (2 * n * 2 + (n - 2) * n * 3) / (n * n)
    # interior rows form 3 groups out of 5 elements
    assert 0.55 < d["clustering_avg"] < 0.7


def test_features_sd_matches_two_pass():
    m = synth.power_law(20000, seed=9)
    f, _ = oracle.features(m.n_rows, m.n_cols, m.rowptr, m.colind)
    lens = np.diff(m.rowptr.astype(np.int64))
    assert f[4] == lens.sum() / lens.size
    assert abs(f[5] - np.std(lens)) <= 1e-12 * np.std(lens)
    c = m.colind.astype(np.int64)
    bw = np.where(lens > 0, c[np.maximum(m.rowptr[1:] - 1, 0)] - c[np.minimum(m.rowptr[:-1], len(c) - 1)] + 1, 0)
    assert abs(f[9] - np.std(bw)) <= 1e-12 * np.std(bw)
    sc = np.where(lens > 0, lens / np.maximum(bw, 1), 0.0)
    assert abs(f[10] - sc.mean()) <= 2 ** -24
    assert abs(f[11] - sc.std()) <= 2 ** -20


# ----------------------------------------------------------------------- bounds
def test_bounds_closed_form():
    p_mb, p_peak, ws = oracle.bounds(4, 4, 10, 4, 8, 8, 100.0)
    assert ws == 4 * 5 + 12 * 10 + 64
    assert p_mb == pytest.approx(20 * 100 / 204, rel=1e-15)
    assert p_peak == pytest.approx(20 * 100 / 144, rel=1e-15)


def test_select_bmax():
    assert oracle.select_bmax(100, 100, 1.0, 5.0) == 5.0
    assert oracle.select_bmax(101, 100, 1.0, 5.0) == 1.0


# --------------------------------------------------------------------- classify
def _p_vector(imb, ml, mb, cmp_):
    """P-vector that makes each Fig. 3 predicate take the requested value; mb and cmp_
    cannot both hold (P_MB < P_CMP < P_peak excludes P_MB > P_CMP or P_CMP > P_peak)."""
    p_csr = 100.0
    p_imb = 200.0 if imb else 110.0
    p_ml = 200.0 if ml else 110.0
    if mb:
        p_mb, p_cmp, p_peak = 110.0, 150.0, 300.0
    elif cmp_:
        p_mb, p_cmp, p_peak = 150.0, 110.0, 300.0
    else:
        p_mb, p_cmp, p_peak = 400.0, 450.0, 500.0     # ordered, but P_CSR far below P_MB
    return p_csr, p_mb, p_ml, p_imb, p_cmp, p_peak


@pytest.mark.parametrize("imb,ml,mb,cmp_", [c for c in itertools.product([0, 1], repeat=4)
                                            if not (c[2] and c[3])])
def test_classify_truth_table(imb, ml, mb, cmp_):
    want = (4 if imb else 0) | (2 if ml else 0) | (1 if mb else 0) | (8 if cmp_ else 0)
    assert oracle.classify(*_p_vector(imb, ml, mb, cmp_)) == want


def test_classify_thresholds_are_strict_and_cmp_above_peak():
    assert oracle.classify(100, 500, 125, 124, 550, 600) == 0     # ratios equal T: no class
    assert oracle.classify(100, 500, 125.0001, 124.0001, 550, 600) == 6
    assert oracle.classify(100, 110, 100, 100, 700, 600) == 8     # P_CMP > P_peak -> CMP
    assert oracle.classify(100, 133.4, 100, 100, 150, 600) == 0   # P_CSR/P_MB < 0.75
    assert oracle.classify(100, 133.3, 100, 100, 150, 600) == 1


def test_variant_map_table2():
    for cls in range(16):
        part, idx, xp, vec = oracle.variant_for_classes(cls, nnz_avg=10, nnz_max=1000)
        assert part == (1 if cls & 4 else 0)
        assert idx == (1 if cls & 1 else 0)
        assert xp == (1 if cls & 2 else 0)
        assert vec == (1 if cls & 9 else 0)
    # IMB without highly uneven rows keeps the dynamic (sub-warp row) schedule
    assert oracle.variant_for_classes(4, nnz_avg=10, nnz_max=100)[0] == 0
    assert oracle.variant_for_classes(5, nnz_avg=10, nnz_max=100)[:2] == (0, 1)


def test_amortization_and_metrics():
    assert oracle.amortization_iters(10.0, 3.0, 1.0) == 5.0
    assert math.isinf(oracle.amortization_iters(10.0, 1.0, 1.0))
    assert oracle.exact_match_ratio([1, 2, 6, 0], [1, 3, 6, 8]) == 0.5
    assert oracle.partial_match_ratio([1, 2, 6, 0], [1, 3, 4, 8]) == 0.75
    assert oracle.partial_match_ratio([0], [0]) == 1.0
    assert oracle.harmonic_mean([1.0, 4.0, 4.0]) == 2.0


# -------------------------------------------------------------------------- MLP
SIZES = [5, 7, 6, 4]


def _params(seed, sizes=SIZES):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(oracle.mlp_nparams(sizes)) * 0.5


def test_mlp_gradient_central_differences():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((9, SIZES[0]))
    Y = (rng.random((9, SIZES[3])) < 0.5).astype(np.float64)
    w = _params(4)
    _, g, _ = oracle.mlp_loss_grad(SIZES, w, X, Y)
    h = 1e-6
    for i in range(w.size):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (oracle.mlp_loss_grad(SIZES, wp, X, Y, False)[0]
              - oracle.mlp_loss_grad(SIZES, wm, X, Y, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), i


def test_mlp_loss_is_bce_of_sigmoid():
    sizes = [1, 1, 1, 1]
    # W1=1, b1=0, W2=1, b2=0, W3=2, b3=-1 -> z = 2 relu(relu(x)) - 1
    w = np.array([1.0, 0.0, 1.0, 0.0, 2.0, -1.0])
    loss, _, probs = oracle.mlp_loss_grad(sizes, w, np.array([[1.5]]), np.array([[1.0]]))
    z = 2.0
    assert probs[0, 0] == pytest.approx(1 / (1 + math.exp(-z)), rel=1e-15)
    assert loss == pytest.approx(-math.log(1 / (1 + math.exp(-z))), rel=1e-14)


def test_mlp_training_reduces_loss_on_separable_set():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((64, SIZES[0]))
    Y = np.stack([X[:, 0] > 0, X[:, 1] > 0, X[:, 0] + X[:, 2] > 0, X[:, 3] < 0], 1) * 1.0
    w = _params(6) * 0.5
    l0 = oracle.mlp_loss_grad(SIZES, w, X, Y, False)[0]
    for _ in range(300):
        _, g, _ = oracle.mlp_loss_grad(SIZES, w, X, Y)
        w -= 0.5 * g
    l1, _, probs = oracle.mlp_loss_grad(SIZES, w, X, Y, False)
    assert l1 < 0.5 * l0
    assert np.mean((probs > 0.5) == (Y > 0.5)) > 0.9


def test_mlp_logits_f32_exact_small_net():
    sizes = [2, 2, 2, 1]
    # every product and sum below is exact in FP32
    w = np.array([1, 2, -1, 0.5, 0.25, -0.5,      # W1 (2x2), b1
                  1, 1, 2, -1, 0, 1,               # W2 (2x2), b2
                  0.5, 4, -3], dtype=np.float32)   # W3 (1x2), b3
    x = np.array([[2.0, 3.0], [-1.0, 1.0]], dtype=np.float32)
    got = oracle.mlp_logits_f32(sizes, w, x)
    # sample 0: h1 = relu([0.25+2+6, -0.5-2+1.5]) = [8.25, 0]; h2 = relu([8.25, 16.5+1]) ;
    #           z = 0.5*8.25 + 4*17.5 - 3
    # sample 1: h1 = relu([0.25-1+2, -0.5+1+0.5]) = [1.25, 1]; h2 = relu([2.25, 2.5-1+1])
    #           z = 0.5*2.25 + 4*2.5 - 3
    assert got[:, 0].tolist() == [0.5 * 8.25 + 4 * 17.5 - 3, 0.5 * 2.25 + 4 * 2.5 - 3]


def test_mlp_logits_f32_close_to_f64_forward():
    rng = np.random.default_rng(7)
    w = _params(8).astype(np.float32)
    X = rng.standard_normal((50, SIZES[0])).astype(np.float32)
    lg = oracle.mlp_logits_f32(SIZES, w, X)
    _, _, probs = oracle.mlp_loss_grad(SIZES, w.astype(np.float64), X.astype(np.float64),
                                       np.zeros((50, SIZES[3])), False)
    z64 = np.log(probs / (1 - probs))
    assert np.max(np.abs(lg - z64)) < 1e-4


def test_log2p1_accuracy_and_exact_powers():
    v = np.concatenate([np.logspace(-6, 9, 5000), [0.5, 1.0, 3.0, 7.0, 1023.0]]).astype(np.float32)
    got = oracle.log2p1_f32(v)
    ref = np.log2(1.0 + v.astype(np.float64))
    # forming w = 1 + v in FP32 costs up to 2^-24 relative in w, i.e. 2^-24 / ln 2 absolute
    assert np.all(np.abs(got - ref) <= 2e-6 * np.abs(ref) + 2.0 ** -24 / math.log(2) * 1.01)
    for k in range(1, 20):
        assert oracle.log2p1_f32(np.float32(2 ** k - 1))[0] == float(k)
    assert oracle.log2p1_f32(np.float32(0.0))[0] == 0.0
    assert oracle.log2p1_f32(np.float32(-3.0))[0] == 0.0


def test_feature_rules_each_branch():
    base = np.zeros(14)
    def f(size=0.0, nnz_max=10.0, nnz_avg=10.0, misses=1.0):
        v = base.copy()
        v[0], v[3], v[4], v[13] = size, nnz_max, nnz_avg, misses
        return v
    l2 = 100 << 20
    assert oracle.feature_rules(f(), 10 ** 6, 8, l2) == 1                    # MB
    assert oracle.feature_rules(f(nnz_max=400), 10 ** 6, 8, l2) == 4         # IMB
    assert oracle.feature_rules(f(misses=6.0), 10 ** 8, 8, l2) == 2          # ML: big x
    assert oracle.feature_rules(f(misses=6.0), 10 ** 6, 8, l2) == 1          # x fits: MB
    assert oracle.feature_rules(f(size=1.0), 10 ** 6, 8, l2) == 8            # CMP
    assert oracle.feature_rules(f(nnz_avg=3.0, nnz_max=3.0), 10 ** 6, 8, l2) == 8
    assert oracle.feature_rules(f(nnz_max=400, misses=6.0), 10 ** 8, 8, l2) == 6


def test_mlp_inputs_definition():
    feat = np.zeros(16)
    feat[:14] = [1, 0.5, 1, 63, 1, 3, 3, 255, 15, 3, 0.25, 0.125, 0.75, 0.5]
    feat[14], feat[15] = 1023.0, 1023.0
    x = oracle.mlp_inputs(feat)[0]
    # log2(1 + v) is exact at v = 2^k - 1; the other entries are exact FP32 values
    assert x.tolist() == [10.0, 1.0, 2.0, 6.0, 6.0, 4.0, 2.0, 0.25, 0.125, 0.75, 0.5, 1.0]
    mu = np.full(12, 1.0, np.float32)
    inv = np.full(12, 0.5, np.float32)
    y = oracle.mlp_inputs(feat, mu, inv)[0]
    assert np.array_equal(y, (x - 1.0) * 0.5)
    z = np.zeros(16)
    assert oracle.mlp_inputs(z)[0].tolist() == [0.0] * 12


def test_classify2_second_pass_truth_table():
    cmp_only = [100.0, 150.0, 110.0, 110.0, 110.0, 300.0]     # Fig. 3 -> {CMP}
    assert oracle.classify(*cmp_only) == 8
    assert oracle.classify2(cmp_only) == 8                    # no second pass
    # P_CSR' = 120 (120 / P_MB 150 = 0.8 >= 0.75 -> MB); P_ML' = 200 (ratio 1.67 -> ML)
    assert oracle.classify2(cmp_only, [120.0, 200.0]) == 8 | 1 | 2
    assert oracle.classify2(cmp_only, [100.0, 110.0]) == 8    # 0.667 < 0.75, ratio 1.1
    assert oracle.classify2(cmp_only, [112.5, 112.5]) == 8 | 1  # exactly 0.75 -> MB
    assert oracle.classify2(cmp_only, [100.0, 125.0]) == 8    # ML needs a strict excess
    # without CMP in the first pass the second pass changes nothing
    mb_only = [100.0, 110.0, 100.0, 100.0, 150.0, 300.0]
    assert oracle.classify2(mb_only, [1.0, 1000.0]) == oracle.classify(*mb_only) == 1
