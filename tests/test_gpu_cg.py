"""GPU conjugate gradients against the oracle's textbook CG: the residual history, the
solution's true residual, iteration counts, determinism and argument errors."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def api(torch):
    from paper_1711_05487_gb300 import api as _api
    return _api


SYSTEMS = {
    "lap2d_64": lambda: synth.laplacian_2d(64),
    "lap27_16": lambda: synth.laplacian_27pt(16),
}
VARIANTS = [dict(vec=1, vs=1, index=1, tile_rows=32), dict(vec=1, vs=4),
            dict(partition=1), dict(vec=1, vs=1, tile_rows=128, tile_pipe=1, xpath=1)]


def _true_res(m, x, b):
    y, _ = oracle.spmv(m.rowptr, m.colind, m.val, x)
    return float(np.linalg.norm(b - y))


@pytest.mark.parametrize("name", list(SYSTEMS))
@pytest.mark.parametrize("precision", ["f64", "df64"])
def test_cg_follows_oracle(api, torch, name, precision):
    m = SYSTEMS[name]()
    b = synth.uniform_vector(m.n_rows, 41)
    xo, ko, co, ho = oracle.cg(m.rowptr, m.colind, m.val, b, max_iters=3000, rtol=1e-10)
    assert co
    A = api.SpmvMatrix.from_csr(m)
    if precision == "df64":
        A.set_precision("df64", "f64", "df64")
    bd = torch.from_numpy(b).cuda()
    for v in VARIANTS:
        A.set_variant(**v)
        x, rep, hist = A.cg(bd, max_iters=3000, rtol=1e-10, check_every=1, history=True)
        h = hist.cpu().numpy()
        assert rep["converged"] == 1, (v, rep)
        # the early residuals agree closely; rounding differences grow slowly with k
        k0 = min(30, len(h), len(ho))
        assert np.max(np.abs(h[:k0] - ho[:k0])) <= 1e-8 * ho[0], v
        assert abs(rep["iters"] - ko) <= max(3, ko // 50), (v, rep["iters"], ko)
        assert _true_res(m, x.cpu().numpy(), b) <= 2e-10 * np.linalg.norm(b), v
        assert abs(rep["b_norm"] - np.linalg.norm(b)) <= 1e-14 * np.linalg.norm(b)


def test_cg_is_deterministic_and_checks_in_chunks(api, torch):
    m = synth.laplacian_27pt(12)
    b = torch.from_numpy(synth.uniform_vector(m.n_rows, 42)).cuda()
    A = api.SpmvMatrix.from_csr(m)
    A.tune("profile")
    x1, r1 = A.cg(b, max_iters=500, rtol=1e-9, check_every=1)
    x2, r2 = A.cg(b, max_iters=500, rtol=1e-9, check_every=1)
    assert torch.equal(x1, x2) and r1["iters"] == r2["iters"]
    x3, r3 = A.cg(b, max_iters=500, rtol=1e-9, check_every=16)
    assert r1["iters"] <= r3["iters"] < r1["iters"] + 16
    assert r3["converged"] == 1


def test_cg_zero_iterations_and_initial_guess(api, torch):
    m = synth.laplacian_2d(32)
    xs = synth.uniform_vector(m.n_rows, 43)
    b = synth.uniform_vector(m.n_rows, 44)
    A = api.SpmvMatrix.from_csr(m)
    A.set_variant(vec=1, vs=1)
    x0 = torch.from_numpy(xs).cuda()
    x, rep, hist = A.cg(torch.from_numpy(b).cuda(), x0=x0, max_iters=0, rtol=0.0,
                        history=True)
    assert rep["iters"] == 0 and torch.equal(x, x0)
    want = _true_res(m, xs, b)
    assert abs(hist[0].item() - want) <= 1e-12 * want


def test_cg_argument_errors(api, torch):
    from paper_1711_05487_gb300._abi import SpmvError
    rect = synth.uniform_random(100, 5, seed=45, n_cols=120)
    A = api.SpmvMatrix.from_csr(rect)
    A.set_variant()
    b = torch.zeros(100, dtype=torch.float64, device="cuda")
    with pytest.raises(SpmvError) as e:
        A.cg(b)
    assert e.value.status == 7
    m = synth.laplacian_2d(8)
    B = api.SpmvMatrix.from_csr(m.astype(np.float32))
    B.set_variant()
    with pytest.raises(SpmvError) as e:
        B.cg(torch.zeros(m.n_rows, dtype=torch.float32, device="cuda"))
    assert e.value.status == 2
    C = api.SpmvMatrix.from_csr(m)
    with pytest.raises(SpmvError) as e:
        C.cg(torch.zeros(m.n_rows, dtype=torch.float64, device="cuda"))
    assert e.value.status == 4
