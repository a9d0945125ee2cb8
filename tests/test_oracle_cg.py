"""Pins of the oracle's conjugate-gradient solver against properties of the method:
finite termination in as many steps as distinct eigenvalues, the exact solution, the
monotone A-norm error, and the residual recurrence."""
import numpy as np
import scipy.sparse as sp

import oracle
import synth


def _csr(A):
    A = sp.csr_matrix(A)
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)


def test_terminates_in_number_of_distinct_eigenvalues():
    # a diagonal SPD matrix with three distinct eigenvalues: the Krylov space has dimension 3
    d = np.tile([1.0, 2.0, 5.0], 10)
    rp, ci, v = _csr(np.diag(d))
    b = synth.uniform_vector(d.size, 3)
    x, k, conv, hist = oracle.cg(rp, ci, v, b, max_iters=3, rtol=0.0)
    assert k == 3
    assert hist[2] > 1e-3 * hist[0]                   # not done after two steps
    assert hist[3] <= 1e-13 * np.linalg.norm(b)      # done after three
    assert np.allclose(x, b / d, rtol=0, atol=1e-13)


def test_tridiagonal_exact_solution_in_n_steps():
    n = 12
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    rp, ci, v = _csr(T)
    b = synth.uniform_vector(n, 4)
    x, k, conv, hist = oracle.cg(rp, ci, v, b, max_iters=n, rtol=1e-14)
    assert k <= n
    assert np.max(np.abs(x - np.linalg.solve(T, b))) < 1e-12


def test_a_norm_error_is_monotone_and_recurrence_matches_true_residual():
    m = synth.laplacian_2d(12)
    A = sp.csr_matrix((m.val, m.colind, m.rowptr), shape=(m.n_rows, m.n_cols))
    xs = synth.uniform_vector(m.n_rows, 5)
    b = A @ xs
    x_star = np.linalg.solve(A.toarray(), b)
    errs = []
    for k in range(0, 31):
        x, kk, conv, hist = oracle.cg(m.rowptr, m.colind, m.val, b, max_iters=k, rtol=0.0)
        assert kk == k
        e = x - x_star
        errs.append(np.sqrt(e @ (A @ e)))
        true_res = np.linalg.norm(b - A @ x)
        assert abs(hist[-1] - true_res) <= 1e-10 * np.linalg.norm(b)
    errs = np.array(errs)
    assert np.all(errs[1:] <= errs[:-1] * (1 + 1e-12))
    assert errs[-1] < 1e-3 * errs[0]


def test_trivial_cases():
    m = synth.laplacian_2d(8)
    z = np.zeros(m.n_rows)
    x, k, conv, hist = oracle.cg(m.rowptr, m.colind, m.val, z, rtol=1e-12)
    assert k == 0 and conv and np.all(x == 0) and hist[0] == 0
    xs = synth.uniform_vector(m.n_rows, 6)
    b, _ = oracle.spmv(m.rowptr, m.colind, m.val, xs)
    x, k, conv, hist = oracle.cg(m.rowptr, m.colind, m.val, b, x0=xs, rtol=1e-12)
    assert k == 0 and conv and np.array_equal(x, xs)
