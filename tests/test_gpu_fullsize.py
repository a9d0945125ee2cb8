"""Parity at the full workload sizes, in the launch configuration the benchmark times (the
profile route's tuned variant): every output is computed on the GPU, and a sample of rows
(random rows, the first and last rows, the longest rows) is checked against the oracle row
by row."""
import concurrent.futures as cf
import os

import numpy as np
import pytest

import oracle
import synth
from gpu_util import TAU, check_rows, stored_values, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def api(torch):
    from paper_1711_05487_gb300 import api as _api
    return _api


def _sample_rows(m, n_random=20_000, n_long=64, seed=0):
    rng = np.random.default_rng(seed)
    lens = np.diff(m.rowptr)
    longest = np.argsort(lens)[-n_long:]
    rows = np.concatenate([rng.choice(m.n_rows, min(n_random, m.n_rows), replace=False),
                           [0, m.n_rows - 1], longest])
    return np.unique(rows).astype(np.int64)


def _check_sampled(m, x64, y, values, tau, what):
    rows = _sample_rows(m)
    ys, ss = oracle.spmv_rows(rows, m.rowptr, m.colind, values, x64)
    return check_rows(np.asarray(y, dtype=np.float64)[rows], ys, ss, tau, what)


@pytest.fixture(scope="module")
def stencil160():
    return synth.stencil_27pt(160)


@pytest.mark.parametrize("storage,vec,acc", [("f64", "f64", "f64"), ("df64", "f64", "df64"),
                                             ("f32", "f64", "f64"), ("f32", "f32", "f32"),
                                             ("bf16", "f32", "f32")])
def test_stencil_160_tuned_all_precisions(api, torch, stencil160, storage, vec, acc):
    m = stencil160
    A = api.SpmvMatrix.from_csr(m)
    if storage != "f64":
        A.set_precision(storage, vec, acc)
    rep = A.tune("profile")
    x64 = synth.uniform_vector(m.n_cols, synth.SEED_BASE + 12)
    if vec == "f32":
        x64 = x64.astype(np.float32).astype(np.float64)
    x = torch.from_numpy(x64).cuda()
    if vec == "f32":
        x = x.float()
    y = A.run(x).double().cpu().numpy()
    _check_sampled(m, x64, y, stored_values(m.val, storage), TAU[storage],
                   f"stencil 160^3 {storage}/{vec}/{acc} {rep.variant}")


# the pool the benchmark times on the full stencil (its variant sweep), plus the tuned
# geometry of the thread-per-row tile with 16-bit deltas
STENCIL_POOL = [dict(), dict(vec=1, vs=4), dict(vec=1, vs=1), dict(index=1, vec=1, vs=1),
                dict(vec=1, vs=1, xpath=1), dict(index=1, vec=1, vs=4), dict(partition=1),
                dict(xpath=2, vs=2), dict(partition=3, index=1),
                dict(index=1, vec=1, vs=1, xpath=1, tile_rows=32), dict(partition=2, index=1)]


def test_stencil_160_every_timed_variant(api, torch, stencil160):
    """Every variant the benchmark times on the 160^3 stencil (FP64), at full size, within
    the FP64 bound of the oracle on sampled rows."""
    m = stencil160
    A = api.SpmvMatrix.from_csr(m)
    x64 = synth.uniform_vector(m.n_cols, synth.SEED_BASE + 12)
    x = torch.from_numpy(x64).cuda()
    for v in STENCIL_POOL:
        A.set_variant(**v)
        y = A.run(x).cpu().numpy()
        _check_sampled(m, x64, y, m.val, TAU["f64"], f"stencil 160^3 {v}")


def test_powerlaw_4m_tuned(api, torch):
    m = synth.power_law(4_000_000)
    A = api.SpmvMatrix.from_csr(m)
    A.set_precision("f32", "f32", "f32")
    rep = A.tune("profile")
    x32 = synth.uniform_vector(m.n_cols, synth.SEED_BASE + 13).astype(np.float32)
    y = A.run(torch.from_numpy(x32).cuda()).double().cpu().numpy()
    # FP32 accumulation over merge-path tiles: products, per-thread runs of at most 7 and a
    # carry scan, each tile's part added in FP64 -- within the FP32-storage bound
    _check_sampled(m, x32.astype(np.float64), y, m.val.astype(np.float64), TAU["f32"],
                   f"powerlaw 4M {rep.variant}")
    # the decomposition the autotuner weighs against it, and thread-per-row short rows
    for v in (dict(partition=1), dict(partition=2, vs=1), dict(partition=2, vs=8, xpath=1)):
        A.set_variant(**v)
        y = A.run(torch.from_numpy(x32).cuda()).double().cpu().numpy()
        _check_sampled(m, x32.astype(np.float64), y, m.val.astype(np.float64), TAU["f32"],
                       f"powerlaw 4M {v}")


def test_scattered_16m_tuned(api, torch):
    m = synth.scattered(16_000_000, 8)
    A = api.SpmvMatrix.from_csr(m)
    rep = A.tune("profile")
    # x (128 MB) exceeds the L2: the ML class's column panels beat every single-pass variant
    assert rep.variant[2] >= 2, rep.variant
    x64 = synth.uniform_vector(m.n_cols, synth.SEED_BASE + 14)
    y = A.run(torch.from_numpy(x64).cuda()).cpu().numpy()
    _check_sampled(m, x64, y, m.val, TAU["f64"], f"scattered 16M {rep.variant}")
    # the panel copy of the full-size matrix equals the oracle's on a sample of rows
    prow, pcol, pval, w = (t.cpu().numpy() if hasattr(t, "cpu") else t for t in A.col_panels())
    P = rep.variant[2]
    assert w == oracle.panel_width(m.n_cols, P)
    for r in _sample_rows(m, n_random=2000, n_long=1, seed=5):
        s, e = m.rowptr[r], m.rowptr[r + 1]
        cols = m.colind[s:e]
        for p in range(P):
            inside = (cols >= p * w) & (cols < (p + 1) * w)
            a, b = prow[p, r], prow[p, r + 1]
            assert np.array_equal(pcol[a:b], cols[inside])
            assert np.array_equal(pval[a:b], m.val[s:e][inside])
    # the single-pass variant with x evict-last and the three-panel copy it competes with
    for v in (dict(vec=1, vs=4, xpath=1), dict(xpath=3, vs=1)):
        A.set_variant(**v)
        y = A.run(torch.from_numpy(x64).cuda()).cpu().numpy()
        _check_sampled(m, x64, y, m.val, TAU["f64"], f"scattered 16M {v}")


def test_batched_512_sampled(api, torch):
    specs = synth.batched_specs(512)
    with cf.ThreadPoolExecutor(max_workers=max(2, (os.cpu_count() or 4) - 2)) as ex:
        mats = list(ex.map(lambda sp: synth.make_from_spec(sp, dtype=np.float32), specs))
    # the benchmark's configuration: the learned selector picks each matrix's variant
    sel_path = os.path.join(os.path.dirname(api.__file__), "data", "selector_gb300.npz")
    sel = api.Selector.load(sel_path) if os.path.exists(sel_path) else None
    As, Xs, Ys, X32 = [], [], [], []
    for sp, m in zip(specs, mats):
        A = api.SpmvMatrix.from_csr(m)
        A.set_precision("f32", "f32", "f32")
        if sel is not None:
            A.tune("learned", selector=sel)
        else:
            A.set_variant()
        X = synth.uniform_vector(m.n_cols * sp["k"], sp["seed"], np.float32).reshape(m.n_cols, sp["k"])
        As.append(A)
        X32.append(X)
        Xs.append(torch.from_numpy(X).cuda())
        Ys.append(torch.full((m.n_rows, sp["k"]), float("nan"), dtype=torch.float32,
                             device="cuda"))
    b = api.Batch(As, Xs, Ys, [sp["k"] for sp in specs])
    b.run()
    torch.cuda.synchronize()
    for i, (sp, m, X, Y) in enumerate(zip(specs, mats, X32, Ys)):
        rows = _sample_rows(m, n_random=64, n_long=4, seed=i)
        Yg = Y.cpu().numpy().astype(np.float64)
        for q in range(sp["k"]):
            ys, ss = oracle.spmv_rows(rows, m.rowptr, m.colind, m.val.astype(np.float64),
                                      X[:, q].astype(np.float64))
            check_rows(Yg[rows, q], ys, ss, TAU["f32"], f"batched {i} {m.name} column {q}")
