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
