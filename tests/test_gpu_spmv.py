"""GPU parity of every SpMV variant against the FP64 oracle (small and ragged matrices
spanning several tiles), value precisions, SpMM, host-buffer runs and edge cases."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TAU, check_rows, check_spmv, stored_values, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def api(torch):
    from paper_1711_05487_gb300 import api as _api
    return _api


def _matrices():
    return {
        "lap64": synth.laplacian_2d(64),
        "st27_12": synth.stencil_27pt(12),
        "powerlaw": synth.power_law(20_000, alpha=1.8, clip=20_000, seed=7, dtype=np.float64),
        "ragged_empty": synth.uniform_random(3001, 64, seed=8, min_per_row=0),
        "scattered": synth.scattered(60_000, 8, seed=9),
        "banded": synth.banded(5000, 300, 0.2, seed=10),
        "identity1": synth.identity(1),
        "one_long_row": synth.uniform_random(1, 9000, seed=11, min_per_row=9000, n_cols=20_000),
        "rect_wide": synth.uniform_random(700, 40, seed=12, n_cols=50_000),
        "rect_tall": synth.uniform_random(5000, 6, seed=13, n_cols=300),
        "lap2d_8bit": synth.laplacian_2d(150, 170),          # 8-bit deltas
        "banded_8bit": synth.banded(9000, 50, 0.4, seed=26),  # 8-bit deltas, ragged rows
    }


MATS = _matrices()

VARIANTS = (
    [dict()]                                                           # plain CSR-vector
    + [dict(vec=1, vs=w) for w in (2, 4, 8, 16, 32)]                   # CMP
    + [dict(index=1, vec=1, vs=w) for w in (2, 4, 8, 16, 32)]          # MB
    + [dict(xpath=1, vs=8), dict(vec=1, xpath=1, vs=4),
       dict(index=1, vec=1, xpath=1, vs=4)]                            # ML (+ joint)
    + [dict(partition=1), dict(partition=1, xpath=1)]                  # IMB
    + [dict(partition=2, vs=w) for w in (1, 2, 4, 8)] + [dict(partition=2, xpath=1)]
    + [dict(partition=2, index=1, vs=w) for w in (1, 2, 8)]             # MB + IMB
    + [dict(partition=2, index=1, xpath=1)]
    + [dict(vec=1, vs=1, tile_rows=r, tile_pipe=p) for r in (32, 64, 128) for p in (0, 1)]
    + [dict(index=1, vec=1, vs=1, tile_rows=r, tile_pipe=p, xpath=p) for r in (32, 128)
       for p in (0, 1)]                                                # width-1 tiles
    + [dict(xpath=p, vs=w, vec=c) for p, w, c in ((2, 1, 0), (2, 4, 1), (3, 2, 0), (5, 8, 1),
                                                  (16, 1, 1))]         # ML: column panels
    + [dict(partition=3), dict(partition=3, index=1), dict(partition=3, xpath=1),
       dict(partition=3, index=1, xpath=1)]                            # sliced rows
)


def _dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


@pytest.mark.parametrize("name", list(MATS))
def test_every_variant_fp64(api, torch, name):
    m = MATS[name]
    A = api.SpmvMatrix.from_csr(m)
    x64 = synth.uniform_vector(m.n_cols, 100)
    x = _dev(torch, x64)
    for v in VARIANTS:
        A.set_variant(**v)
        y = A.run(x)
        torch.cuda.synchronize()
        check_spmv(m, x64, y.cpu().numpy(), TAU["f64"], f"{name} {v}")


def test_laplacian_quadratic_closed_form_all_variants(api, torch):
    n = 256
    m = synth.laplacian_2d(n)
    ix = np.arange(n * n) % n
    iy = np.arange(n * n) // n
    u = (ix ** 2 + iy ** 2).astype(np.float64)
    A = api.SpmvMatrix.from_csr(m)
    interior = (ix > 0) & (ix < n - 1) & (iy > 0) & (iy < n - 1)
    for v in VARIANTS:
        A.set_variant(**v)
        y = A.run(_dev(torch, u)).cpu().numpy()
        assert np.all(y[interior] == -4.0), v          # integer sums are exact in any order


def test_identity_and_permutation_bit_exact(api, torch):
    x64 = synth.uniform_vector(100_000, 3)
    for m, want in ((synth.identity(100_000), x64),):
        A = api.SpmvMatrix.from_csr(m)
        for v in VARIANTS:
            A.set_variant(**v)
            y = A.run(_dev(torch, x64)).cpu().numpy()
            assert np.array_equal(y.view(np.uint64), want.view(np.uint64)), v
    p = synth.permutation(100_000, 4)
    A = api.SpmvMatrix.from_csr(p)
    for v in VARIANTS:
        A.set_variant(**v)
        y = A.run(_dev(torch, x64)).cpu().numpy()
        assert np.array_equal(y, x64[p.colind]), v


def test_empty_matrix_and_zero_rows(api, torch):
    m = synth.Csr(5, 7, np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0), "empty")
    A = api.SpmvMatrix.from_csr(m)
    for v in VARIANTS:
        A.set_variant(**v)
        y = torch.full((5,), 7.0, dtype=torch.float64, device="cuda")
        A.run(_dev(torch, np.ones(7)), y)
        assert torch.all(y == 0).item(), v


PRECISIONS = [("f32", "f64", "f64"), ("f32", "f32", "f64"), ("bf16", "f64", "f64"),
              ("bf16", "f32", "f64"), ("bf16", "f32", "f32"), ("f32", "f32", "f32"),
              ("df64", "f64", "df64"), ("f32", "f64", "df64"), ("f32", "f32", "df64"),
              ("bf16", "f64", "df64"), ("bf16", "f32", "df64")]


@pytest.mark.parametrize("storage,vec,acc", PRECISIONS)
@pytest.mark.parametrize("name", ["lap64", "st27_12", "powerlaw", "ragged_empty", "scattered"])
def test_precisions(api, torch, name, storage, vec, acc):
    m = MATS[name]
    A = api.SpmvMatrix.from_csr(m)
    A.set_precision(storage, vec, acc)
    x64 = synth.uniform_vector(m.n_cols, 101)
    if vec == "f32":
        x64 = x64.astype(np.float32).astype(np.float64)    # the x the GPU sees
    x = _dev(torch, x64, torch.float64 if vec == "f64" else torch.float32)
    variants = [dict(), dict(vec=1, vs=4), dict(index=1, vec=1, vs=4), dict(partition=1),
                dict(partition=2), dict(partition=2, index=1),
                dict(vec=1, xpath=1, vs=8), dict(vec=1, vs=1),
                dict(index=1, vec=1, vs=1, tile_rows=64, tile_pipe=1),
                dict(vec=1, vs=1, tile_rows=32, xpath=1),
                dict(xpath=2, vs=2), dict(xpath=3, vs=1, vec=1),
                dict(partition=3, index=1), dict(partition=3)]
    for v in variants:
        A.set_variant(**v)
        y = A.run(x).double().cpu().numpy()
        check_spmv(m, x64, y, TAU[storage], f"{name} {storage}/{vec}/{acc} {v}")
        if acc in ("f64", "df64") and vec == "f64":
            # the accumulation itself: FP64 bound against the values as stored
            check_spmv(m, x64, y, TAU["f64"], f"{name} {storage}/{vec}/{acc} {v} (stored)",
                       values=stored_values(m.val, storage))


SAME_SIGN_LENGTHS = ([0, 1, 15, 16, 17, 29, 30, 31, 33, 63, 64, 65, 127, 129, 500, 2047, 2049,
                      5000, 40_000] * 4)


def test_fp32_accumulation_bound_on_same_sign_long_rows(api, torch):
    """FP32 accumulation on rows whose products all have one sign and x > 0: the running sum
    grows with every product, so a plain FP32 chain's roundings add up (a sequential FP32 sum
    of a 40,000-product row errs by about 4e-6 of the row's sum, outside the 2e-6 bound;
    checked below with numpy). Every variant keeps every row within the FP32 bound, as do SpMM (k = 4, 16) and
    the batched launch (k = 1, 4, 16): long chains are summed in runs of 16 FP32 products."""
    m = synth.same_sign_rows(SAME_SIGN_LENGTHS, 60_000, seed=51, dtype=np.float32)
    x32 = np.random.default_rng(52).uniform(0.5, 1.0, m.n_cols).astype(np.float32)
    x64 = x32.astype(np.float64)
    # the plain FP32 chain this test guards against
    r = int(np.argmax(np.diff(m.rowptr)))
    s0, s1 = m.rowptr[r], m.rowptr[r + 1]
    prod = m.val[s0:s1] * x32[m.colind[s0:s1]]
    exact = float(np.sum(m.val[s0:s1].astype(np.float64) * x64[m.colind[s0:s1]]))
    seq = float(np.add.accumulate(prod, dtype=np.float32)[-1])
    assert abs(seq - exact) / exact > TAU["f32"]
    A = api.SpmvMatrix.from_csr(m)
    A.set_precision("f32", "f32", "f32")
    x = _dev(torch, x32)
    for v in VARIANTS:
        A.set_variant(**v)
        y = A.run(x).double().cpu().numpy()
        check_spmv(m, x64, y, TAU["f32"], f"same-sign rows {v}")
    for k in (4, 16):
        X32 = np.random.default_rng(53 + k).uniform(0.5, 1.0, (m.n_cols, k)).astype(np.float32)
        A.set_variant(vec=1, vs=4)
        Y = A.spmm(_dev(torch, X32)).double().cpu().numpy()
        Yr, Sr = oracle.spmm(m.rowptr, m.colind, m.val, X32.astype(np.float64))
        check_rows(Y.ravel(), Yr.ravel(), Sr.ravel(), TAU["f32"], f"same-sign spmm k={k}")
    As, Xs, Ys, X64 = [], [], [], []
    for k, vs in ((1, 1), (4, 2), (16, 4), (16, 32)):
        B = api.SpmvMatrix.from_csr(m)
        B.set_precision("f32", "f32", "f32")
        B.set_variant(vec=1, vs=vs)
        X = np.random.default_rng(60 + k + vs).uniform(0.5, 1.0, (m.n_cols, k)).astype(np.float32)
        As.append(B)
        Xs.append(_dev(torch, X))
        Ys.append(torch.full((m.n_rows, k), float("nan"), dtype=torch.float32, device="cuda"))
        X64.append(X.astype(np.float64))
    b = api.Batch(As, Xs, Ys, [1, 4, 16, 16])
    for plan in ((256, 512), (2048, 8192)):
        b.set_plan(*plan)
        b.run()
        torch.cuda.synchronize()
        for X, Y, k in zip(X64, Ys, (1, 4, 16, 16)):
            Yr, Sr = oracle.spmm(m.rowptr, m.colind, m.val, X)
            check_rows(Y.cpu().numpy().astype(np.float64).ravel(), Yr.ravel(), Sr.ravel(),
                       TAU["f32"], f"same-sign batched k={k} plan {plan}")
    b.close()


def test_unsupported_precision_rejected(api):
    from paper_1711_05487_gb300._abi import SpmvError
    A = api.SpmvMatrix.from_csr(MATS["lap64"])
    with pytest.raises(SpmvError):
        A.set_precision("f64", "f32", "f32")
    with pytest.raises(SpmvError):
        A.set_precision("f32", "f64", "f32")


@pytest.mark.parametrize("k", [1, 3, 4, 16])
@pytest.mark.parametrize("name", ["lap64", "powerlaw", "rect_wide"])
def test_spmm(api, torch, name, k):
    m = MATS[name]
    A = api.SpmvMatrix.from_csr(m)
    A.set_variant()
    X64 = np.random.default_rng(5).uniform(-1, 1, size=(m.n_cols, k))
    Y = A.spmm(_dev(torch, X64)).cpu().numpy()
    Yr, Sr = oracle.spmm(m.rowptr, m.colind, m.val, X64)
    check_rows(Y.ravel(), Yr.ravel(), Sr.ravel(), TAU["f64"], f"spmm {name} k={k}")
    A32 = api.SpmvMatrix.from_csr(m.astype(np.float32))
    A32.set_variant()
    X32 = X64.astype(np.float32)
    Y32 = A32.spmm(_dev(torch, X32)).double().cpu().numpy()
    Yr, Sr = oracle.spmm(m.rowptr, m.colind, m.val.astype(np.float32), X32)
    check_rows(Y32.ravel(), Yr.ravel(), Sr.ravel(), TAU["f32"], f"spmm32 {name} k={k}")


@pytest.mark.parametrize("gen", [lambda: synth.stencil_27pt(30),       # one launch
                                 lambda: synth.stencil_27pt(80),       # eight row chunks;
                                                                       # panels: slices, then
                                                                       # last-pass chunks
                                 lambda: synth.power_law(30_000, seed=14, dtype=np.float64)])
def test_run_host_equals_device_run(api, torch, gen):
    m = gen()
    A = api.SpmvMatrix.from_csr(m)
    x64 = synth.uniform_vector(m.n_cols, 7)
    xh = torch.from_numpy(x64).pin_memory()
    yh = torch.empty(m.n_rows, dtype=torch.float64).pin_memory()
    for v in (dict(index=1, vec=1), dict(vec=1, vs=1, tile_rows=64, tile_pipe=1),
              dict(vec=1, vs=4), dict(partition=1), dict(xpath=2, vs=4),
              dict(xpath=3, vs=1, vec=1), dict(partition=3, index=1)):
        A.set_variant(**v)
        yd = A.run(torch.from_numpy(x64).cuda()).cpu()
        yh.fill_(float("nan"))
        A.run_host(xh, yh)
        assert torch.equal(yd, yh), v


def test_not_tuned_and_bad_args(api, torch):
    from paper_1711_05487_gb300._abi import SpmvError
    A = api.SpmvMatrix.from_csr(MATS["lap64"])
    x = torch.zeros(A.n_cols, dtype=torch.float64, device="cuda")
    with pytest.raises(SpmvError) as e:
        A.run(x)
    assert e.value.status == 4
    with pytest.raises(SpmvError):
        A.set_variant(vs=3)


def test_runs_are_reproducible(api, torch):
    m = MATS["powerlaw"]
    A = api.SpmvMatrix.from_csr(m)
    x = _dev(torch, synth.uniform_vector(m.n_cols, 9))
    for v in VARIANTS:
        A.set_variant(**v)
        a = A.run(x).clone()
        b = A.run(x)
        assert torch.equal(a, b), v


def test_bounded_wait_expires_and_context_survives(api, torch):
    """A wait on an mbarrier phase nothing completes gives up after its limit, the error is
    reported to the host, and the next SpMV on the same context is correct."""
    from paper_1711_05487_gb300 import _abi
    m = MATS["st27_12"]
    A = api.SpmvMatrix.from_csr(m)
    assert _abi.spmv_selftest_wait_timeout(A.handle, 2_000_000) == 6     # 2 ms limit
    assert _abi.spmv_get_last_device_error(A.handle) == 0                  # cleared
    A.set_variant(vec=1, vs=1)
    x64 = synth.uniform_vector(m.n_cols, 15)
    check_spmv(m, x64, A.run(_dev(torch, x64)).cpu().numpy(), TAU["f64"], "after timeout")


def _df_runs(api, torch, m, x64, variants):
    """(double-float y, FP64 y) per width-1 variant on the same matrix and x."""
    A = api.SpmvMatrix.from_csr(m)
    D = api.SpmvMatrix.from_csr(m)
    D.set_precision("df64", "f64", "df64")
    x = _dev(torch, x64)
    out = []
    for v in variants:
        A.set_variant(**v)
        D.set_variant(**v)
        out.append((D.run(x).cpu().numpy(), A.run(x).cpu().numpy()))
    return out


DF_VARIANTS = [dict(vec=1, vs=1, tile_rows=r, xpath=xp) for r in (32, 128) for xp in (0, 1)] + \
              [dict(index=1, vec=1, vs=1, tile_rows=r) for r in (32, 64, 128)]


def test_df64_rows_that_do_not_split_fall_back_to_fp64(api, torch):
    """Rows that meet a value or x element outside [2^-40, 2^41) are recomputed with FP64
    FMAs, bit-identical to the FP64 tile kernel; zeros in x split exactly; every row stays
    within the FP64 bound of the oracle."""
    m = synth.uniform_random(20_000, 20, seed=21, min_per_row=0, n_cols=30_000)
    rng = np.random.default_rng(22)
    val = m.val.copy()
    bad_rows = rng.choice(m.n_rows, 300, replace=False)
    for r in bad_rows[:150]:                     # tiny and huge values
        s, e = m.rowptr[r], m.rowptr[r + 1]
        if e > s:
            val[s] = 1e-14 if r % 2 else 3e13
    m = synth.Csr(m.n_rows, m.n_cols, m.rowptr, m.colind, val, "df_edges")
    x64 = synth.uniform_vector(m.n_cols, 23)
    x64[rng.choice(m.n_cols, 200, replace=False)] = 0.0
    x64[rng.choice(m.n_cols, 50, replace=False)] = 1e-13
    x64[rng.choice(m.n_cols, 50, replace=False)] = -5e12
    xb = (x64 != 0) & ((np.abs(x64) < 2.0 ** -40) | (np.abs(x64) >= 2.0 ** 41))
    vb = (val != 0) & ((np.abs(val) < 2.0 ** -40) | (np.abs(val) >= 2.0 ** 41))
    bad = np.zeros(m.n_rows, bool)
    row_of = np.repeat(np.arange(m.n_rows), np.diff(m.rowptr))
    bad[row_of[vb | xb[m.colind]]] = True
    assert bad.sum() > 100
    for (yd, y64), v in zip(_df_runs(api, torch, m, x64, DF_VARIANTS), DF_VARIANTS):
        assert np.array_equal(yd[bad].view(np.uint64), y64[bad].view(np.uint64)), v
        check_spmv(m, x64, yd, TAU["df64"], f"df64 {v}")


def test_double_float_accumulation_on_fp32_storage_falls_back_like_fp64(api, torch):
    """FP32 storage with double-float accumulation: rows meeting a value or x element outside
    [2^-40, 2^41) are recomputed with FP64 FMAs, bit-identical to the FP64-accumulating tile
    kernel on the same FP32 values; every row is within the FP64 bound of the oracle on the
    stored values."""
    m = synth.uniform_random(20_000, 20, seed=24, min_per_row=0, n_cols=30_000)
    rng = np.random.default_rng(25)
    val = m.val.copy()
    for r in rng.choice(m.n_rows, 150, replace=False):
        s, e = m.rowptr[r], m.rowptr[r + 1]
        if e > s:
            val[s] = 1e-14 if r % 2 else 3e13
    m = synth.Csr(m.n_rows, m.n_cols, m.rowptr, m.colind, val, "df_f32_edges")
    x64 = synth.uniform_vector(m.n_cols, 26)
    x64[rng.choice(m.n_cols, 200, replace=False)] = 0.0
    x64[rng.choice(m.n_cols, 50, replace=False)] = 1e-13
    v32 = stored_values(val, "f32")
    xb = (x64 != 0) & ((np.abs(x64) < 2.0 ** -40) | (np.abs(x64) >= 2.0 ** 41))
    vb = (v32 != 0) & ((np.abs(v32) < 2.0 ** -40) | (np.abs(v32) >= 2.0 ** 41))
    bad = np.zeros(m.n_rows, bool)
    row_of = np.repeat(np.arange(m.n_rows), np.diff(m.rowptr))
    bad[row_of[vb | xb[m.colind]]] = True
    assert bad.sum() > 100
    D = api.SpmvMatrix.from_csr(m)
    D.set_precision("f32", "f64", "df64")
    F = api.SpmvMatrix.from_csr(m)
    F.set_precision("f32", "f64", "f64")
    x = _dev(torch, x64)
    for v in DF_VARIANTS:
        D.set_variant(**v)
        F.set_variant(**v)
        yd, yf = D.run(x).cpu().numpy(), F.run(x).cpu().numpy()
        assert np.array_equal(yd[bad].view(np.uint64), yf[bad].view(np.uint64)), v
        check_spmv(m, x64, yd, TAU["f64"], f"f32/df64 {v}", values=v32)


def test_df64_long_rows_and_ragged(api, torch):
    for m in (MATS["ragged_empty"], MATS["powerlaw"], MATS["one_long_row"], MATS["banded"]):
        x64 = synth.uniform_vector(m.n_cols, 24)
        long_rows = np.diff(m.rowptr) > 32
        for (yd, y64), v in zip(_df_runs(api, torch, m, x64, DF_VARIANTS), DF_VARIANTS):
            check_spmv(m, x64, yd, TAU["df64"], f"df64 {m.name} {v}")
            # rows above 32 nonzeros: FP64 FMAs in the FP64 tile kernel's order (oversize
            # tiles run the same warp-per-row code in both)
            assert np.array_equal(yd[long_rows], y64[long_rows]), (m.name, v)


def test_df64_run_host_equals_device_run(api, torch):
    m = synth.stencil_27pt(80)
    A = api.SpmvMatrix.from_csr(m)
    A.set_precision("df64", "f64", "df64")
    x64 = synth.uniform_vector(m.n_cols, 25)
    xh = torch.from_numpy(x64).pin_memory()
    yh = torch.empty(m.n_rows, dtype=torch.float64).pin_memory()
    for v in (dict(index=1, vec=1, vs=1), dict(vec=1, vs=1, tile_rows=64)):
        A.set_variant(**v)
        yd = A.run(torch.from_numpy(x64).cuda()).cpu()
        yh.fill_(float("nan"))
        A.run_host(xh, yh)
        assert torch.equal(yd, yh), v
        check_spmv(m, x64, yh.numpy(), TAU["df64"], f"df64 host {v}")


def test_df64_tune_and_reject_non_f64_input(api, torch):
    from paper_1711_05487_gb300._abi import SpmvError
    m = MATS["st27_12"]
    A = api.SpmvMatrix.from_csr(m)
    A.set_precision("df64", "f64", "df64")
    rep = A.tune("profile")
    x64 = synth.uniform_vector(m.n_cols, 26)
    check_spmv(m, x64, A.run(_dev(torch, x64)).cpu().numpy(), TAU["df64"], f"df64 tuned {rep.variant}")
    B = api.SpmvMatrix.from_csr(m.astype(np.float32))
    with pytest.raises(SpmvError):
        B.set_precision("df64", "f64", "df64")
    with pytest.raises(SpmvError):
        A.set_precision("df64", "f32", "df64")


def test_run_host_graph_replays_follow_buffers_and_variants(api, torch):
    """Page-locked buffers take the captured-graph path: a new buffer pair or a new variant
    is re-captured, and pageable buffers take the eager path; all equal the device run."""
    m = synth.stencil_27pt(80)          # x and y above 8 MB: the chunked pipeline
    A = api.SpmvMatrix.from_csr(m)
    xs = [synth.uniform_vector(m.n_cols, s) for s in (71, 72)]
    outs = {}
    for v in (dict(index=1, vec=1, vs=1, tile_rows=32), dict(vec=1, vs=4), dict(partition=1)):
        A.set_variant(**v)
        for pin in (True, False):
            for k, x64 in enumerate(xs):
                xh = torch.from_numpy(x64)
                yh = torch.full((m.n_rows,), float("nan"), dtype=torch.float64)
                if pin:
                    xh, yh = xh.pin_memory(), yh.pin_memory()
                for _ in range(2):                       # capture, then replay
                    A.run_host(xh, yh)
                    want = A.run(torch.from_numpy(x64).cuda()).cpu()
                    assert torch.equal(want, yh), (v, pin, k)
                outs[(str(v), pin, k)] = yh.clone()
        assert torch.equal(outs[(str(v), True, 0)], outs[(str(v), False, 0)])
