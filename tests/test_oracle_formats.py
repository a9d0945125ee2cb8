"""Pins of the oracle's value rounding, delta-index format and merge-path coordinates."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth


# ------------------------------------------------------------------ value precision
def test_round_f32_matches_numpy():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-40, 40, 10000),
                        [0.0, -0.0, 1e-46, 3.4028235677973366e38, 3.5e38, np.inf, -np.inf]])
    with np.errstate(over="ignore"):
        ref = v.astype(np.float32)
    assert np.array_equal(oracle.round_f32(v).view(np.uint32), ref.view(np.uint32))


def _bf16_exact(v: float) -> int:
    """Brute-force round-to-nearest-even of v to bf16, in exact rational arithmetic."""
    if v == 0.0:
        return 0x8000 if np.signbit(v) else 0
    sign = 0x8000 if v < 0 else 0
    a = Fraction(abs(v))
    e = 0
    while a >= 2 ** (e + 1):
        e += 1
    while a < 2 ** e:
        e -= 1
    e = max(e, -126)
    quantum = Fraction(2) ** (e - 7)
    q = round(a / quantum)                # Fraction rounding: ties to even
    r = q * quantum
    if r >= 2 ** 128:
        return sign | 0x7F80
    f = np.float32(float(r))
    return sign | int(np.array([f]).view(np.uint32)[0] >> 16)


def test_round_bf16_against_exact_rationals():
    rng = np.random.default_rng(1)
    v = rng.standard_normal(3000) * 2.0 ** rng.integers(-140, 128, 3000)
    # exact halfway points and their neighbours
    half = [1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -40, 1 + 2 ** -8 - 2 ** -40,
            -(1 + 2 ** -8), 2.0 ** -133, 2.0 ** -134, 3 * 2.0 ** -134, 2.0 ** -127 * 1.5,
            (2 - 2 ** -8) * 2.0 ** 127, (2 - 2 ** -9) * 2.0 ** 127, 3.3895313892515355e38]
    v = np.concatenate([v, half])
    got = oracle.round_bf16_bits(v)
    want = np.array([_bf16_exact(float(t)) for t in v], dtype=np.uint16)
    assert np.array_equal(got, want)


def test_round_bf16_known_bits():
    got = oracle.round_bf16_bits(np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.0,
                                           (2 - 2 ** -8) * 2.0 ** 127, np.inf, np.nan]))
    assert [hex(int(b)) for b in got] == ["0x3f80", "0x3f80", "0x3f82", "0xc000",
                                         "0x7f80", "0x7f80", "0x7fc0"]


# ------------------------------------------------------------------ delta16 format
def test_delta16_hand_example():
    rp = np.array([0, 3, 3, 5, 6, 8], np.int32)
    ci = np.array([2, 3, 10, 0, 70000, 5, 100, 65635], np.int32)
    base, delta, esc = oracle.delta16_encode(rp, ci)
    assert list(base) == [2, 0, -1, 5, 100]
    assert list(delta) == [0, 1, 7, 0, 0, 0, 0, 65535]
    assert list(esc) == [0, 70000]
    assert np.array_equal(oracle.delta16_decode(rp, base, delta, esc), ci)


def test_delta16_gap_limit():
    rp = np.array([0, 2, 4], np.int32)
    ci = np.array([0, 65535, 0, 65536], np.int32)
    base, delta, esc = oracle.delta16_encode(rp, ci)
    assert list(base) == [0, -1] and list(esc) == [0, 65536]


@pytest.mark.parametrize("gen", [lambda: synth.stencil_27pt(12),
                                 lambda: synth.scattered(300_000, 4, seed=3),
                                 lambda: synth.power_law(50_000, seed=4),
                                 lambda: synth.identity(1)])
def test_delta16_round_trip(gen):
    m = gen()
    base, delta, esc = oracle.delta16_encode(m.rowptr, m.colind)
    assert np.array_equal(oracle.delta16_decode(m.rowptr, base, delta, esc), m.colind)


def test_delta16_stencil_has_no_escape_rows():
    m = synth.stencil_27pt(20)
    _, _, esc = oracle.delta16_encode(m.rowptr, m.colind)
    assert esc.size == 0


def test_delta8_hand_example_and_gap_limit():
    rp = np.array([0, 3, 3, 5, 6, 8], np.int32)
    ci = np.array([2, 3, 10, 0, 300, 5, 100, 355], np.int32)
    base, delta, esc = oracle.delta8_encode(rp, ci)
    assert list(base) == [2, 0, -1, 5, 100]          # row 2's gap 300 escapes, 255 fits
    assert list(delta) == [0, 1, 7, 0, 0, 0, 0, 255]
    assert list(esc) == [0, 300]
    assert np.array_equal(oracle.delta8_decode(rp, base, delta, esc), ci)


@pytest.mark.parametrize("gen", [lambda: synth.banded(3000, 40, 0.5, seed=5),
                                 lambda: synth.laplacian_2d(200),
                                 lambda: synth.power_law(20_000, seed=6)])
def test_delta8_round_trip(gen):
    m = gen()
    base, delta, esc = oracle.delta8_encode(m.rowptr, m.colind)
    assert np.array_equal(oracle.delta8_decode(m.rowptr, base, delta, esc), m.colind)


def test_delta_width_choice():
    # every gap of the 2-D Laplacian on a 200-wide grid is 1 or 199: 8 bits fit everywhere
    assert oracle.delta_width(*_rc(synth.laplacian_2d(200))) == 8
    # the 27-point stencil's plane gaps (~n^2) escape 8 bits: 16
    assert oracle.delta_width(*_rc(synth.stencil_27pt(20))) == 16
    # one row of 4 nonzeros with a 256 gap (16 bytes escaped at 8 bits, 8 at 16 bits) next
    # to short-gap rows: 8 bits win only when the fitting rows save more than the escape
    # costs. Rows: [0,1,2,300] and k rows [0,1,2,3]: bytes8 = 16 + 4k, bytes16 = 8 + 8k
    for k, want in ((1, 16), (2, 16), (3, 8)):
        rows = [[0, 1, 2, 300]] + [[0, 1, 2, 3]] * k
        rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
        ci = np.concatenate(rows).astype(np.int32)
        assert oracle.delta_width(rp, ci) == want, k


def _rc(m):
    return m.rowptr, m.colind


# -------------------------------------------------------------------- merge path
def test_merge_path_hand_example():
    rp = np.array([0, 2, 2, 5], np.int32)
    c = oracle.merge_path(rp, 2)
    assert c.tolist() == [[0, 0], [0, 2], [2, 2], [2, 4], [3, 5]]


def _check_merge_coordinates(rp, c, d):
    n, nnz = rp.shape[0] - 1, int(rp[-1])
    assert c[0].tolist() == [0, 0] and c[-1].tolist() == [n, nnz]
    for t, (a, b) in enumerate(c.tolist()):
        if t < len(c) - 1:
            assert a + b == t * d
        # consumed nonzeros precede every unconsumed row end ...
        if a < n and b > 0:
            assert b - 1 < rp[a + 1]
        # ... and consumed row ends precede every unconsumed nonzero
        if a > 0 and b < nnz:
            assert rp[a] <= b
    assert np.all(np.diff(c[:, 0]) >= 0) and np.all(np.diff(c[:, 1]) >= 0)
    assert np.all(np.diff(c.sum(axis=1))[:-1] == d) and np.diff(c.sum(axis=1))[-1] <= d


@pytest.mark.parametrize("gen,d", [(lambda: synth.power_law(20_000, seed=5), 256),
                                   (lambda: synth.laplacian_2d(30), 64),
                                   (lambda: synth.uniform_random(5000, 3, 6, min_per_row=0), 7),
                                   (lambda: synth.identity(1), 2048)])
def test_merge_path_splits_characterised(gen, d):
    m = gen()
    _check_merge_coordinates(m.rowptr, oracle.merge_path(m.rowptr, d), d)


def test_merge_path_empty_matrix():
    c = oracle.merge_path(np.zeros(1, np.int32), 16)
    assert c.tolist() == [[0, 0]]


# ------------------------------------------------------------------ double-float split
def _f32_bits(x: float) -> int:
    return int(np.array([x], dtype=np.float32).view(np.uint32)[0])


def _df_exact(v: float) -> tuple[int, int]:
    """The split from the 53-bit integer significand M of v: hi = the top 24 bits of M,
    lo = the next 23, each scaled back to v's exponent (exact rational arithmetic)."""
    import math
    if v == 0.0:
        return (0x80000000 if math.copysign(1.0, v) < 0 else 0, 0)
    if not math.isfinite(v):
        return (0x7FC00000, 0)
    _, e2 = math.frexp(abs(v))
    e = e2 - 1
    if e < -40 or e > 40:
        return (0x7FC00000, 0)
    M = Fraction(abs(v)) / Fraction(2) ** (e - 52)
    assert M.denominator == 1 and 2 ** 52 <= M < 2 ** 53
    M = int(M)
    sign = -1 if v < 0 else 1
    hi = sign * Fraction(M >> 29) * Fraction(2) ** (e - 23)
    lo_int = (M >> 6) & (2 ** 23 - 1)
    lo = sign * Fraction(lo_int) * Fraction(2) ** (e - 46)
    return (_f32_bits(float(hi)), _f32_bits(float(lo)) if lo_int else 0)


def test_df_split_against_integer_significand():
    rng = np.random.default_rng(3)
    v = rng.standard_normal(4000) * 2.0 ** rng.integers(-45, 46, 4000)
    edge = [1.0, -1.0, 1 + 2 ** -30, 1 + 2 ** -52, -3.75, 2.0 ** -40, 2.0 ** 41,
            2.0 ** 41 - 2.0 ** -12, 2.0 ** -41, (2 - 2 ** -52) * 2.0 ** -41, 0.0, -0.0,
            np.inf, -np.inf, np.nan, 1 + 2 ** -23 + 2 ** -24 + 2 ** -47, -(1 + 2 ** -46)]
    v = np.concatenate([v, edge])
    got = oracle.df_split_bits(v)
    want = np.array([_df_exact(float(t)) for t in v], dtype=np.uint32)
    assert np.array_equal(got, want)


def test_df_split_known_bits_and_error_bound():
    got = oracle.df_split_bits(np.array([1.0, 1 + 2 ** -30, 1 + 2 ** -52, -3.75, 2.0 ** -40,
                                         2.0 ** 41, 0.0, -0.0, np.nan]))
    assert [tuple(hex(int(b)) for b in r) for r in got] == [
        ("0x3f800000", "0x0"), ("0x3f800000", "0x30800000"), ("0x3f800000", "0x0"),
        ("0xc0700000", "0x0"), ("0x2b800000", "0x0"), ("0x7fc00000", "0x0"),
        ("0x0", "0x0"), ("0x80000000", "0x0"), ("0x7fc00000", "0x0")]
    rng = np.random.default_rng(4)
    v = rng.uniform(-1, 1, 20000) * 2.0 ** rng.integers(-39, 40, 20000)
    v = v[(np.abs(v) >= 2.0 ** -40) & (np.abs(v) < 2.0 ** 41)]
    pair = oracle.df_split_bits(v).view(np.float32).astype(np.float64)
    hi, lo = pair[:, 0], pair[:, 1]
    r = np.array([float(Fraction(a) - Fraction(b) - Fraction(c)) for a, b, c in zip(v, hi, lo)])
    assert np.all(np.abs(r) < 2.0 ** -46 * np.abs(v))
    assert np.all(np.sign(r) * np.sign(v) >= 0)          # truncation toward zero


# ------------------------------------------------------------------ row decomposition
def test_row_bins_hand_example():
    # row lengths 1, 5, 0, 12, 3, 9 with l_med = 3 and chunk = 5: rows 0 and 2 are short,
    # row 4 (length 3) is medium, rows 1, 3 and 5 are long and cut into chunks of 5
    lens = [1, 5, 0, 12, 3, 9]
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    ci = np.concatenate([np.arange(n) * 3 + 7 for n in lens]).astype(np.int32)
    med, lng, first, ch = oracle.row_bins(rp, ci, l_med=3, chunk=5)
    assert list(med) == [4]
    assert list(lng) == [1, 3, 5]
    assert list(first) == [0, 1, 4, 6]
    # start column: the row's first column for a first chunk, else the previous column
    assert [tuple(c) for c in ch] == [(1, 1, 6, 7), (3, 6, 11, 7), (3, 11, 16, 19),
                                      (3, 16, 18, 34), (5, 21, 26, 7), (5, 26, 30, 19)]


def test_row_bins_partition_the_matrix_exactly():
    """A_short + A_medium + A_long = A: every nonzero belongs to exactly one short row,
    medium row or chunk, and rebuilding the product from the pieces gives the oracle's y."""
    m = synth.power_law(30_000, alpha=1.4, clip=30_000, seed=17, dtype=np.float64)
    med, lng, first, ch = oracle.row_bins(m.rowptr, m.colind, l_med=64, chunk=4096)
    lens = np.diff(m.rowptr)
    owner = np.full(m.nnz, -1, np.int64)
    for r in np.where(lens < 64)[0]:
        owner[m.rowptr[r]:m.rowptr[r + 1]] = 0
    for r in med:
        assert 64 <= lens[r] < 4096
        assert np.all(owner[m.rowptr[r]:m.rowptr[r + 1]] == -1)
        owner[m.rowptr[r]:m.rowptr[r + 1]] = 1
    assert len(lng) > 0 and np.all(lens[lng] >= 4096)
    for i, r in enumerate(lng):
        cs = ch[first[i]:first[i + 1]]
        assert np.all(cs[:, 0] == r)
        assert cs[0, 1] == m.rowptr[r] and cs[-1, 2] == m.rowptr[r + 1]
        assert np.all(cs[1:, 1] == cs[:-1, 2])
        assert np.all(cs[:-1, 2] - cs[:-1, 1] == 4096) and 0 < cs[-1, 2] - cs[-1, 1] <= 4096
        for _, b, e, c0 in cs:
            assert np.all(owner[b:e] == -1)
            owner[b:e] = 2
            assert c0 == m.colind[b - 1 if b > m.rowptr[r] else b]
    assert np.all(owner >= 0)
    x = synth.uniform_vector(m.n_cols, 18)
    y, _ = oracle.spmv(m.rowptr, m.colind, m.val, x)
    prod = m.val * x[m.colind]
    y2 = np.zeros(m.n_rows)
    rows_of = np.repeat(np.arange(m.n_rows), lens)
    np.add.at(y2, rows_of, prod)
    assert np.allclose(y2, y, rtol=0, atol=1e-9)


# ------------------------------------------------------------------ column panels
def test_panel_width_closed_forms():
    # ceil(n_cols / P) rounded up to a multiple of 32
    assert oracle.panel_width(100, 1) == 128
    assert oracle.panel_width(1000, 4) == 256
    assert oracle.panel_width(64, 2) == 32
    assert oracle.panel_width(65, 2) == 64
    assert oracle.panel_width(16_000_000, 2) == 8_000_000
    assert oracle.panel_width(16_000_000, 3) == 5_333_344
    assert oracle.panel_width(40, 4) == 32      # panels 2 and 3 are empty
    assert oracle.panel_width(0, 2) == 32


def test_col_panels_hand_example():
    # 3 rows over 70 columns, 3 panels of 32 columns: [0, 32), [32, 64), [64, 96)
    rp = np.array([0, 4, 4, 7], np.int32)
    ci = np.array([1, 31, 32, 69, 5, 40, 63], np.int32)
    prow, perm, w = oracle.col_panels(rp, ci, 70, 3)
    assert w == 32
    assert prow.tolist() == [[0, 2, 2, 3], [3, 4, 4, 6], [6, 7, 7, 7]]
    assert perm.tolist() == [0, 1, 4, 2, 5, 6, 3]


def _dense(n_rows, n_cols, rp, ci, v):
    d = np.zeros((n_rows, n_cols))
    for i in range(n_rows):
        for j in range(rp[i], rp[i + 1]):
            d[i, ci[j]] += v[j]
    return d


@pytest.mark.parametrize("n_panels", [1, 2, 3, 5, 16])
@pytest.mark.parametrize("gen", [lambda: synth.uniform_random(300, 40, seed=31),
                                 lambda: synth.scattered(500, 8, seed=32),
                                 lambda: synth.banded(400, 30, 0.5, seed=33),
                                 lambda: synth.dense_random(60, 90, 0.03, seed=36)])
def test_col_panels_against_dense_masks(gen, n_panels):
    """Panel p, read as a CSR of its own, is A with every column outside [p*w, (p+1)*w) set
    to zero; perm is a bijection; columns keep their order inside each row."""
    m = gen()
    prow, perm, w = oracle.col_panels(m.rowptr, m.colind, m.n_cols, n_panels)
    assert prow.shape == (n_panels, m.n_rows + 1)
    assert np.array_equal(np.sort(perm), np.arange(m.nnz))
    dense = _dense(m.n_rows, m.n_cols, m.rowptr, m.colind, m.val)
    pc, pv = m.colind[perm], m.val[perm]
    cols = np.arange(m.n_cols)
    total = np.zeros_like(dense)
    for p in range(n_panels):
        r = prow[p]
        assert np.all(np.diff(r) >= 0)
        if p > 0:
            assert r[0] == prow[p - 1][-1]
        for i in range(m.n_rows):
            assert np.all(np.diff(pc[r[i]:r[i + 1]]) > 0)
        d = _dense(m.n_rows, m.n_cols, r, pc, pv)
        inside = (cols >= p * w) & (cols < (p + 1) * w)
        assert np.array_equal(d, dense * inside[None, :])
        total += d
    assert np.array_equal(total, dense)
    assert prow[0][0] == 0 and prow[-1][-1] == m.nnz
    if n_panels == 1:
        assert np.array_equal(prow[0], m.rowptr) and np.array_equal(perm, np.arange(m.nnz))


def test_col_panels_spmv_by_passes_is_exact_on_integers():
    # integer values and x: every partial sum is exact, so summing the passes in order
    # equals the one-pass product bit for bit
    m = synth.scattered(2000, 8, seed=34)
    rng = np.random.default_rng(35)
    val = rng.integers(-9, 10, m.nnz).astype(np.float64)
    x = rng.integers(-9, 10, m.n_cols).astype(np.float64)
    y, _ = oracle.spmv(m.rowptr, m.colind, val, x)
    prow, perm, _ = oracle.col_panels(m.rowptr, m.colind, m.n_cols, 3)
    acc = np.zeros(m.n_rows)
    for p in range(3):
        yp, _ = oracle.spmv(prow[p] - prow[p][0], m.colind[perm][prow[p][0]:prow[p][-1]],
                            val[perm][prow[p][0]:prow[p][-1]], x)
        acc += yp
    assert np.array_equal(acc, y)


# ------------------------------------------------------------------ sliced rows (SELL-32)
def test_sell32_hand_example():
    # 3 rows of lengths 2, 0, 3 in one slice of width 3: element k of row l at 32 k + l
    rp = np.array([0, 2, 2, 5], np.int32)
    soff, perm = oracle.sell32(rp)
    assert soff.tolist() == [0, 96]
    want = np.full(96, -1)
    want[[0, 32]] = [0, 1]
    want[[2, 34, 66]] = [2, 3, 4]
    assert perm.tolist() == want.tolist()


@pytest.mark.parametrize("gen", [lambda: synth.uniform_random(1000, 40, seed=41, min_per_row=0),
                                 lambda: synth.stencil_27pt(9),
                                 lambda: synth.power_law(3000, alpha=1.6, clip=500, seed=42,
                                                         dtype=np.float64),
                                 lambda: synth.dense_random(70, 50, 0.1, seed=43),
                                 lambda: synth.Csr(0, 4, np.zeros(1, np.int32),
                                                   np.zeros(0, np.int32), np.zeros(0), "empty")])
def test_sell32_against_dense_and_widths(gen):
    """Reading every slice position back (value and column of perm, zero for padding)
    rebuilds A; each slice is as wide as its longest row; every CSR element appears once,
    rows in order down their lane."""
    m = gen()
    soff, perm = oracle.sell32(m.rowptr)
    ns = (m.n_rows + 31) // 32
    lens = np.diff(m.rowptr)
    assert soff.shape == (ns + 1,) and soff[0] == 0
    for s in range(ns):
        assert soff[s + 1] - soff[s] == 32 * lens[32 * s:32 * s + 32].max()
    real = perm[perm >= 0]
    assert np.array_equal(np.sort(real), np.arange(m.nnz))
    dense = np.zeros((m.n_rows, m.n_cols))
    for s in range(ns):
        w = (soff[s + 1] - soff[s]) // 32
        for lane in range(32):
            r = 32 * s + lane
            ks = [perm[soff[s] + 32 * k + lane] for k in range(w)]
            n_real = sum(1 for j in ks if j >= 0)
            assert all(j >= 0 for j in ks[:n_real]) and all(j < 0 for j in ks[n_real:])
            if r < m.n_rows:
                assert n_real == lens[r]
                assert ks[:n_real] == list(range(m.rowptr[r], m.rowptr[r + 1]))
                for j in ks[:n_real]:
                    dense[r, m.colind[j]] += m.val[j]
            else:
                assert n_real == 0
    want = np.zeros((m.n_rows, m.n_cols))
    for r in range(m.n_rows):
        for j in range(m.rowptr[r], m.rowptr[r + 1]):
            want[r, m.colind[j]] += m.val[j]
    assert np.array_equal(dense, want)
