"""Randomized properties of the oracle on small CSR matrices: each check is derived from the
definition of the operation (a dense product, the CSR definition, the delta-index rules of
Section III-E, the merge-path item count, the sliced-row and column-panel layouts, round to
nearest even), not from the oracle's own code, so that a dropped term, a wrong index or an
off-by-one in the oracle fails one of them."""
import numpy as np
import pytest

import oracle
import synth

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
from hypothesis import given, settings  # noqa: E402

SETTINGS = dict(max_examples=60, deadline=None)


def random_csr(seed, n_rows, n_cols, max_len, gap_scale):
    m = synth.random_gaps(n_rows, n_cols, max_len, gap_scale, seed)
    return m.rowptr, m.colind


csr_args = dict(seed=st.integers(0, 2**31 - 1), n_rows=st.integers(0, 64),
                n_cols=st.integers(1, 400_000), max_len=st.integers(0, 40),
                gap_scale=st.sampled_from([1.0, 30.0, 300.0, 3000.0, 100_000.0]))


def dense(rowptr, colind, val, n_cols):
    n = rowptr.size - 1
    A = np.zeros((n, n_cols), dtype=val.dtype)
    for i in range(n):
        A[i, colind[rowptr[i]:rowptr[i + 1]]] = val[rowptr[i]:rowptr[i + 1]]
    return A


@settings(**SETTINGS)
@given(**csr_args)
def test_generated_csr_is_valid_and_each_corruption_has_its_code(seed, n_rows, n_cols, max_len,
                                                                  gap_scale):
    rp, ci = random_csr(seed, n_rows, n_cols, max_len, gap_scale)
    assert oracle.validate_csr(n_rows, n_cols, rp, ci) == 0
    if n_rows == 0:
        return
    bad = rp.copy()
    bad[0] = 1                                   # rowptr[0] != 0 (code 1)
    assert oracle.validate_csr(n_rows, n_cols, bad, ci) == 1
    if n_rows >= 2:
        bad = rp.copy()
        bad[1] = bad[2] + 1                      # rowptr decreases after row 0 (code 2)
        assert oracle.validate_csr(n_rows, n_cols, bad, ci) == 2
    # the last row pointer must equal the number of nonzeros (code 3)
    bad = rp.copy()
    bad[-1] = rp[-1] + 1
    assert oracle.validate_csr(n_rows, n_cols, bad, ci) == 3
    if ci.size:
        # a column at n_cols is out of range (code 4)
        c = ci.copy()
        c[-1] = n_cols
        assert oracle.validate_csr(n_rows, n_cols, rp, c) == 4
        # a repeated column inside a row breaks "sorted, unique" (code 5)
        lens = np.diff(rp)
        r = int(np.argmax(lens))
        if lens[r] >= 2:
            c = ci.copy()
            c[rp[r] + 1] = c[rp[r]]
            assert oracle.validate_csr(n_rows, n_cols, rp, c) == 5


@settings(**SETTINGS)
@given(**csr_args)
def test_spmv_equals_dense_product_exactly_on_integers(seed, n_rows, n_cols, max_len, gap_scale):
    """Fig. 1 on integer data is exact in FP64: y = A x and s = |A| |x| as dense products."""
    n_cols = min(n_cols, 5000)
    rp, ci = random_csr(seed, n_rows, n_cols, max_len, gap_scale)
    rng = np.random.default_rng(seed + 1)
    val = rng.integers(-8, 9, ci.size).astype(np.float64)
    x = rng.integers(-8, 9, n_cols).astype(np.float64)
    y, s = oracle.spmv(rp, ci, val, x)
    A = dense(rp, ci, val, n_cols).astype(np.int64)
    xi = x.astype(np.int64)
    assert np.array_equal(y, (A @ xi).astype(np.float64))
    assert np.array_equal(s, (np.abs(A) @ np.abs(xi)).astype(np.float64))
    # SpMM column by column is the SpMV
    X = rng.integers(-8, 9, (n_cols, 3)).astype(np.float64)
    Y, S = oracle.spmm(rp, ci, val, X)
    for q in range(3):
        yq, sq = oracle.spmv(rp, ci, val, X[:, q])
        assert np.array_equal(Y[:, q], yq) and np.array_equal(S[:, q], sq)


def _row_max_gap(rp, ci, i):
    seg = ci[rp[i]:rp[i + 1]].astype(np.int64)
    return int(np.diff(seg).max()) if seg.size >= 2 else 0


@settings(**SETTINGS)
@given(**csr_args)
def test_delta_index_escape_rule_width_rule_and_round_trip(seed, n_rows, n_cols, max_len,
                                                           gap_scale):
    """Section III-E's delta index: a row is an escape row exactly when one of its gaps does
    not fit the width; the others store their first column as base; the width is the one
    with fewer index bytes (1 or 2 per nonzero of fitting rows, 4 per nonzero of escape
    rows), 16 on a tie; decoding gives the columns back."""
    rp, ci = random_csr(seed, n_rows, n_cols, max_len, gap_scale)
    lens = np.diff(rp.astype(np.int64))
    gaps = np.array([_row_max_gap(rp, ci, i) for i in range(n_rows)], np.int64)
    nbytes = {}
    for bits, enc, dec, limit in ((16, oracle.delta16_encode, oracle.delta16_decode, 65535),
                                  (8, oracle.delta8_encode, oracle.delta8_decode, 255)):
        base, delta, esc = enc(rp, ci)
        escape = gaps > limit
        assert np.array_equal(base < 0, escape)
        for i in np.flatnonzero(~escape):
            if lens[i]:
                assert base[i] == ci[rp[i]]
                assert delta[rp[i]] == 0
            else:
                assert base[i] == 0
        assert esc.size == int(lens[escape].sum())
        assert np.array_equal(dec(rp, base, delta, esc), ci)
        nbytes[bits] = (bits // 8) * int(lens[~escape].sum()) + 4 * int(lens[escape].sum())
    want = 8 if nbytes[8] < nbytes[16] else 16
    assert oracle.delta_width(rp, ci) == want


@settings(**SETTINGS)
@given(**csr_args, d=st.integers(1, 50))
def test_merge_path_tiles_take_exactly_their_items(seed, n_rows, n_cols, max_len, gap_scale, d):
    """Every merge-path tile consumes d merge items (row ends + nonzeros), the last one the
    remainder; boundaries move monotonically from (0, 0) to (N, NNZ) and never consume a
    nonzero of a row before the end of the rows above it."""
    rp, ci = random_csr(seed, n_rows, n_cols, max_len, gap_scale)
    co = oracle.merge_path(rp, d).astype(np.int64)
    nnz = int(rp[-1])
    assert tuple(co[0]) == (0, 0) and tuple(co[-1]) == (n_rows, nnz)
    steps = np.diff(co, axis=0)
    assert (steps >= 0).all()
    items = steps.sum(axis=1)
    assert (items[:-1] == d).all() and 0 < items[-1] <= d if items.size else n_rows + nnz == 0
    for i, j in co:
        assert rp[i] <= j
        if i < n_rows:
            assert j <= rp[i + 1]


@settings(**SETTINGS)
@given(**csr_args)
def test_sliced_rows_place_every_element_once(seed, n_rows, n_cols, max_len, gap_scale):
    """SELL-32: slice s is 32 x (its longest row) positions; element k of row 32 s + l sits
    at soff[s] + 32 k + l; every CSR position appears once, the rest is padding (-1)."""
    rp, ci = random_csr(seed, n_rows, n_cols, max_len, gap_scale)
    soff, perm = oracle.sell32(rp)
    lens = np.diff(rp.astype(np.int64))
    ns = (n_rows + 31) // 32
    assert soff.size == ns + 1 and soff[0] == 0
    for s in range(ns):
        assert soff[s + 1] - soff[s] == 32 * int(lens[32 * s:32 * s + 32].max())
    for r in range(n_rows):
        s, lane = divmod(r, 32)
        for k in range(lens[r]):
            assert perm[soff[s] + 32 * k + lane] == rp[r] + k
    real = perm[perm >= 0]
    assert np.array_equal(np.sort(real), np.arange(int(rp[-1])))


@settings(**SETTINGS)
@given(**csr_args, n_panels=st.integers(2, 6))
def test_column_panels_split_each_row_by_column_slice(seed, n_rows, n_cols, max_len, gap_scale,
                                                      n_panels):
    """Panel p holds, row by row and in column order, exactly the nonzeros whose columns lie
    in [p w, (p + 1) w); the panels together hold every nonzero once."""
    rp, ci = random_csr(seed, n_rows, n_cols, max_len, gap_scale)
    prow, perm, w = oracle.col_panels(rp, ci, n_cols, n_panels)
    assert w % 32 == 0 and w * n_panels >= n_cols
    for p in range(n_panels):
        for i in range(n_rows):
            got = perm[prow[p, i]:prow[p, i + 1]]
            seg = np.arange(rp[i], rp[i + 1])
            want = seg[(ci[seg] >= p * w) & (ci[seg] < (p + 1) * w)]
            assert np.array_equal(got, want)
    assert np.array_equal(np.sort(perm), np.arange(ci.size))


finite = st.floats(allow_nan=False, allow_infinity=False, width=64)


@settings(max_examples=200, deadline=None)
@given(a=finite, b=finite)
def test_bf16_rounding_is_monotone_and_idempotent(a, b):
    """Round to nearest even from FP64 to BF16 never reorders two values and leaves a BF16
    value unchanged."""
    lo, hi = min(a, b), max(a, b)
    bits = oracle.round_bf16_bits(np.array([lo, hi]))
    v = oracle.bf16_bits_to_f64(bits)
    if np.isfinite(v).all():
        assert v[0] <= v[1]
        assert np.array_equal(oracle.round_bf16_bits(v), bits)


@settings(max_examples=200, deadline=None)
@given(a=finite)
def test_f32_rounding_matches_numpy_and_is_idempotent(a):
    r = oracle.round_f32(np.array([a]))
    with np.errstate(over="ignore"):             # beyond the FP32 range both give infinity
        want = np.array([a]).astype(np.float32)
    assert r.view(np.uint32)[0] == want.view(np.uint32)[0]
    assert oracle.round_f32(r.astype(np.float64)).view(np.uint32)[0] == r.view(np.uint32)[0]


@settings(**SETTINGS)
@given(**csr_args, line=st.sampled_from([2, 16, 32]), fits=st.booleans())
def test_table1_features_against_a_direct_computation(seed, n_rows, n_cols, max_len, gap_scale,
                                                      line, fits):
    """Table I per row: nnz, bandwidth (last - first + 1), scatter nnz/bw, clustering (runs
    of consecutive columns / nnz) and misses (the first element and every gap larger than a
    cache line); averages and population deviations over all N rows (empty rows count as
    zeros); size = working set within the last-level cache, density = NNZ / (N N_cols).
    Ratios are compared within the oracle's 2^-24 quantization."""
    n_rows = max(n_rows, 1)
    rp, ci = random_csr(seed, n_rows, n_cols, max_len, gap_scale)
    f, _ = oracle.features(n_rows, n_cols, rp, ci, line_elems=line,
                           ws_bytes=100 if fits else 1000, llc_bytes=500)
    d = dict(zip(oracle.FEATURE_NAMES, f))
    nnz, bw, sc, cl, ms = (np.zeros(n_rows) for _ in range(5))
    for i in range(n_rows):
        c = ci[rp[i]:rp[i + 1]].astype(np.int64)
        if c.size == 0:
            continue
        g = np.diff(c)
        nnz[i] = c.size
        bw[i] = c[-1] - c[0] + 1
        sc[i] = c.size / bw[i]
        cl[i] = (1 + np.count_nonzero(g != 1)) / c.size
        ms[i] = 1 + np.count_nonzero(g > line)
    assert d["size"] == (1.0 if fits else 0.0)
    assert d["density"] == pytest.approx(rp[-1] / (n_rows * n_cols), rel=1e-15)
    assert (d["nnz_min"], d["nnz_max"]) == (nnz.min(), nnz.max())
    assert d["nnz_avg"] == pytest.approx(nnz.mean(), rel=1e-15)
    assert d["nnz_sd"] == pytest.approx(nnz.std(), rel=1e-12, abs=1e-12)
    assert (d["bw_min"], d["bw_max"]) == (bw.min(), bw.max())
    assert d["bw_avg"] == pytest.approx(bw.mean(), rel=1e-15)
    assert d["bw_sd"] == pytest.approx(bw.std(), rel=1e-12, abs=1e-9)
    assert abs(d["scatter_avg"] - sc.mean()) <= 2 ** -24
    assert abs(d["scatter_sd"] - sc.std()) <= 2 ** -20
    assert abs(d["clustering_avg"] - cl.mean()) <= 2 ** -24
    assert d["misses_avg"] == pytest.approx(ms.mean(), rel=1e-15)


@settings(**SETTINGS)
@given(**csr_args, l_med=st.integers(1, 10), extra=st.integers(1, 14))
def test_row_decomposition_bins_and_chunks(seed, n_rows, n_cols, max_len, gap_scale, l_med,
                                           extra):
    """Fig. 5's A = A_short + A_long with a medium bin: rows shorter than l_med are short,
    rows of l_med..chunk-1 nonzeros medium (listed in order), longer rows long (listed in
    order) and cut into consecutive chunks of `chunk` nonzeros, the last one the remainder;
    a chunk's start column is the row's first column for its first chunk, else the column
    before the chunk (the base its deltas start from)."""
    chunk = l_med + extra
    rp, ci = random_csr(seed, n_rows, n_cols, max_len, gap_scale)
    lens = np.diff(rp.astype(np.int64))
    med, lng, first, ch = oracle.row_bins(rp, ci, l_med=l_med, chunk=chunk)
    assert np.array_equal(med, np.flatnonzero((lens >= l_med) & (lens < chunk)))
    assert np.array_equal(lng, np.flatnonzero(lens >= chunk))
    assert first.size == lng.size + 1 and first[0] == 0 and first[-1] == ch.shape[0]
    for i, r in enumerate(lng):
        cs = ch[first[i]:first[i + 1]].astype(np.int64)
        starts = np.arange(rp[r], rp[r + 1], chunk)
        assert np.array_equal(cs[:, 0], np.full(starts.size, r))
        assert np.array_equal(cs[:, 1], starts)
        assert np.array_equal(cs[:, 2], np.minimum(starts + chunk, rp[r + 1]))
        want_c0 = np.where(starts > rp[r], ci[np.maximum(starts - 1, 0)], ci[rp[r]])
        assert np.array_equal(cs[:, 3], want_c0)
