"""Pins of the oracle's SpMV (Fig. 1) and CSR validation against mathematics that does not
depend on the oracle: dense products, closed forms and exact permutations."""
import numpy as np
import pytest

import oracle
import synth


def _dense(m: synth.Csr) -> np.ndarray:
    a = np.zeros((m.n_rows, m.n_cols))
    for i in range(m.n_rows):
        for j in range(m.rowptr[i], m.rowptr[i + 1]):
            a[i, m.colind[j]] = m.val[j]
    return a


@pytest.mark.parametrize("shape,density,seed", [((1, 1), 1.0, 1), ((7, 5), 0.4, 2),
                                                ((64, 64), 0.1, 3), ((33, 64), 0.6, 4),
                                                ((64, 17), 0.0, 5)])
def test_spmv_matches_dense_integer_exact(shape, density, seed):
    m = synth.dense_random(shape[0], shape[1], density, seed, integer_values=True)
    x = np.random.default_rng(seed).integers(-5, 6, size=shape[1]).astype(np.float64)
    y, s = oracle.spmv(m.rowptr, m.colind, m.val, x)
    a = _dense(m)
    assert np.array_equal(y, a @ x)            # integer sums below 2^53 are exact
    assert np.array_equal(s, np.abs(a) @ np.abs(x))


def test_spmv_matches_dense_real_values():
    m = synth.dense_random(64, 64, 0.3, 11, integer_values=False)
    x = synth.uniform_vector(64, 12)
    y, s = oracle.spmv(m.rowptr, m.colind, m.val, x)
    ref = _dense(m) @ x
    assert np.all(np.abs(y - ref) <= 1e-14 * s + 1e-300)


def test_laplacian_of_quadratic_is_constant():
    """A u for u(ix, iy) = ix^2 + iy^2: -4 at interior points; on the boundary the missing
    neighbours' values (the quadratic extended to the ghost points) are added back."""
    n = 256
    m = synth.laplacian_2d(n)
    ix = np.arange(n * n) % n
    iy = np.arange(n * n) // n
    u = (ix ** 2 + iy ** 2).astype(np.float64)
    y, _ = oracle.spmv(m.rowptr, m.colind, m.val, u)
    expect = np.full(n * n, -4.0)
    ghost = lambda gx, gy: gx.astype(np.float64) ** 2 + gy.astype(np.float64) ** 2
    expect += np.where(ix == 0, ghost(ix - 1, iy), 0.0)
    expect += np.where(ix == n - 1, ghost(ix + 1, iy), 0.0)
    expect += np.where(iy == 0, ghost(ix, iy - 1), 0.0)
    expect += np.where(iy == n - 1, ghost(ix, iy + 1), 0.0)
    assert np.array_equal(y, expect)
    interior = (ix > 0) & (ix < n - 1) & (iy > 0) & (iy < n - 1)
    assert np.all(y[interior] == -4.0)


def test_identity_and_permutation_bit_exact():
    x = synth.uniform_vector(1000, 3)
    eye = synth.identity(1000)
    y, _ = oracle.spmv(eye.rowptr, eye.colind, eye.val, x)
    assert np.array_equal(y.view(np.uint64), x.view(np.uint64))
    p = synth.permutation(1000, 4)
    y, _ = oracle.spmv(p.rowptr, p.colind, p.val, x)
    assert np.array_equal(y, x[p.colind])


def test_empty_rows_and_empty_matrix():
    rp = np.array([0, 0, 2, 2], dtype=np.int32)
    ci = np.array([0, 2], dtype=np.int32)
    v = np.array([1.5, -2.0])
    y, s = oracle.spmv(rp, ci, v, np.array([2.0, 7.0, 1.0]))
    assert list(y) == [0.0, 1.0, 0.0] and list(s) == [0.0, 5.0, 0.0]
    y, s = oracle.spmv(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0), np.zeros(0))
    assert y.shape == (0,)


def test_sampled_rows_equal_full():
    m = synth.uniform_random(2000, 40, 5)
    x = synth.uniform_vector(2000, 6)
    y, s = oracle.spmv(m.rowptr, m.colind, m.val, x)
    rows = np.array([0, 5, 1999, 777], dtype=np.int64)
    ys, ss = oracle.spmv_rows(rows, m.rowptr, m.colind, m.val, x)
    assert np.array_equal(ys, y[rows]) and np.array_equal(ss, s[rows])


def test_spmm_matches_dense():
    m = synth.dense_random(40, 30, 0.3, 8, integer_values=True)
    X = np.random.default_rng(9).integers(-4, 5, size=(30, 4)).astype(np.float64)
    Y, S = oracle.spmm(m.rowptr, m.colind, m.val, X)
    assert np.array_equal(Y, _dense(m) @ X)
    assert np.array_equal(S, np.abs(_dense(m)) @ np.abs(X))


def test_validate_csr_codes():
    ok_rp = np.array([0, 2, 3], np.int32)
    ok_ci = np.array([0, 3, 1], np.int32)
    assert oracle.validate_csr(2, 4, ok_rp, ok_ci) == 0
    assert oracle.validate_csr(2, 4, np.array([1, 2, 3], np.int32), ok_ci) == 1
    assert oracle.validate_csr(2, 4, np.array([0, 3, 2], np.int32), ok_ci[:2]) == 2
    assert oracle.validate_csr(2, 4, np.array([0, 2, 2], np.int32), ok_ci) == 3
    assert oracle.validate_csr(2, 3, ok_rp, ok_ci) == 4
    assert oracle.validate_csr(2, 4, ok_rp, np.array([0, 3, -1], np.int32)) == 4
    assert oracle.validate_csr(2, 4, ok_rp, np.array([3, 0, 1], np.int32)) == 5
    assert oracle.validate_csr(2, 4, ok_rp, np.array([3, 3, 1], np.int32)) == 5


def test_generators_produce_valid_csr():
    for m in (synth.laplacian_2d(16), synth.stencil_27pt(6), synth.power_law(3000, seed=1),
              synth.scattered(3000, 8, seed=2), synth.banded(3000, 40, 0.3, 3),
              synth.uniform_random(3000, 64, 4)):
        assert oracle.validate_csr(m.n_rows, m.n_cols, m.rowptr, m.colind) == 0, m.name


def test_static_partition_baseline_equals_sequential_bit_for_bit():
    """The paper's static nnz-balanced baseline computes every row with the same sum."""
    mats = [synth.power_law(5000, seed=31, dtype=np.float64),
            synth.uniform_random(777, 9, seed=32, min_per_row=0),
            synth.identity(3)]
    for m in mats:
        x = synth.uniform_vector(m.n_cols, 33)
        y1, _ = oracle.spmv(m.rowptr, m.colind, m.val, x)
        for T in (1, 2, 5, 16):
            y, used = oracle.spmv_static(m.rowptr, m.colind, m.val, x, T)
            assert 1 <= used <= T
            assert np.array_equal(y.view(np.uint64), y1.view(np.uint64)), (m.name, T)
