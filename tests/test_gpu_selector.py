"""GPU parity of the classification routes (profiling probes, features, learned MLP),
the MLP kernels against the oracle, and the batched persistent launch."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TAU, check_rows, check_spmv, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def api(torch):
    from paper_1711_05487_gb300 import api as _api
    return _api


@pytest.fixture(scope="module")
def abi(torch):
    from paper_1711_05487_gb300 import _abi
    return _abi


def _dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


ROUTE_MATS = {
    "st27_40": lambda: synth.stencil_27pt(40),
    "powerlaw": lambda: synth.power_law(200_000, seed=41, dtype=np.float64),
    "scattered": lambda: synth.scattered(400_000, 8, seed=42),
    "lap128": lambda: synth.laplacian_2d(128),
}


@pytest.mark.parametrize("name", list(ROUTE_MATS))
def test_profile_kernels_compute_the_modified_products(api, torch, name):
    """P_CSR / P_ML / P_CMP kernels (Section III-B): the baseline computes A x; the P_ML
    kernel uses colind'[j] = row(j) and the P_CMP kernel reads x[i] without colind, so both
    compute y_i = x_i * sum_j a_ij."""
    m = ROUTE_MATS[name]()
    A = api.SpmvMatrix.from_csr(m)
    x64 = synth.uniform_vector(m.n_cols, 5)
    x = _dev(torch, x64)
    y = torch.empty(m.n_rows, dtype=torch.float64, device="cuda")
    A.profile_kernel(0, x, y)
    check_spmv(m, x64, y.cpu().numpy(), TAU["f64"], "static baseline")
    rows = np.repeat(np.arange(m.n_rows, dtype=np.int32), np.diff(m.rowptr))
    yr, sr = oracle.spmv(m.rowptr, np.minimum(rows, m.n_cols - 1), m.val, x64)
    for which in (1, 2):
        A.profile_kernel(which, x, y)
        check_rows(y.cpu().numpy(), yr, sr, TAU["f64"], f"profile kernel {which}")


@pytest.mark.parametrize("name", list(ROUTE_MATS))
def test_profile_route_decision_and_result(api, torch, name):
    m = ROUTE_MATS[name]()
    A = api.SpmvMatrix.from_csr(m)
    r = A.tune("profile", reps=5)
    p = [r.p[k] for k in ("P_CSR", "P_MB", "P_ML", "P_IMB", "P_CMP", "P_peak")]
    assert all(v > 0 for v in p)
    assert r.classes == oracle.classify2(p, r.p2)
    lens = np.diff(m.rowptr)
    want = oracle.variant_for_classes(r.classes, lens.mean(), lens.max())
    if want[0] == 1:
        # IMB's decomposition: the autotuner keeps the faster of merge-path tiles (1) and
        # the row decomposition (2); the x path follows the classes either way
        assert r.variant[0] in (1, 2) and r.variant[2] == want[2]
    elif r.variant[0] == 3:
        # the autotuner may keep sliced rows, the same thread-per-row work in another
        # layout, with the classes' column and x paths
        assert want[0] == 0 and tuple(r.variant[1:3]) == want[1:3]
    else:
        assert tuple(r.variant[:4]) == want
    x64 = synth.uniform_vector(m.n_cols, 6)
    check_spmv(m, x64, A.run(_dev(torch, x64)).cpu().numpy(), TAU["f64"], f"{name} tuned")


@pytest.mark.parametrize("name", list(ROUTE_MATS))
def test_feature_route_decision_and_result(api, torch, name):
    m = ROUTE_MATS[name]()
    A = api.SpmvMatrix.from_csr(m)
    r = A.tune("features", autotune=0)
    f = np.array([r.features[k] for k in api.FEATURE_NAMES])
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    assert r.classes == oracle.feature_rules(f, m.n_cols, 8, l2)
    x64 = synth.uniform_vector(m.n_cols, 7)
    check_spmv(m, x64, A.run(_dev(torch, x64)).cpu().numpy(), TAU["f64"], f"{name} features")


def test_bandwidth_probe_is_plausible(abi):
    hbm, l2 = abi.spmv_probe_bandwidth()
    assert 1000 < hbm < 20000 and l2 > hbm


def test_gather_probe_is_plausible(abi):
    """Random gathers: an L2-resident x (16 MB) serves them faster than one far larger than
    the L2 (2 GB), where every gather misses to DRAM; the L2 rate is above 10 G gathers/s and
    each DRAM-bound gather moves at least a 32-byte sector within the HBM bound."""
    n = 1 << 26
    t_l2 = abi.spmv_probe_gather(4 << 20, 4, n, reps=3)
    t_dram = abi.spmv_probe_gather(1 << 29, 4, n, reps=3)
    assert 0 < t_l2 < t_dram
    assert n / (t_l2 * 1e-3) > 10e9
    assert 32 * n / (t_dram * 1e-3) / 1e9 < 20000
    with pytest.raises(abi.SpmvError):
        abi.spmv_probe_gather(1 << 32, 4, n)


def test_fma_probe_is_plausible(abi):
    """Register-only FMA chains: FP32 FMAs retire faster than FP64 ones, each rate stays
    below what the device's SMs could issue at 128 FMA lanes per clock at 2.5 GHz, and the
    FP64 rate with one chain and 16 warps per SM is within a third of the rate with four
    chains and 32 warps (the narrow FP64 pipe needs little parallelism to fill)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f64 = abi.spmv_probe_fma(8, 4, 32, reps=3)
    f64_1 = abi.spmv_probe_fma(8, 1, 16, reps=3)
    f32 = abi.spmv_probe_fma(4, 4, 32, reps=3)
    cap = sms * 128 * 2.5e9
    assert 1e9 < f64 < f32 < cap
    assert f64_1 > 0.67 * f64
    for bad in ((8, 3, 32), (8, 4, 0), (8, 4, 65), (8, 4, 33), (2, 4, 32)):
        with pytest.raises(abi.SpmvError):
            abi.spmv_probe_fma(*bad)


def test_profile_report_and_cta_times(api, torch):
    """spmv_profile: P_MB and P_peak equal the oracle's bounds at the reported B_max (the
    L2 rate for a cache-fitting working set, else HBM: the footnote's reading), the timed
    rates are 2 NNZ / t of their own timings, P_IMB follows t_imb, and every static-partition
    CTA of the CTA-time probe reports a plausible SM and a non-negative time."""
    m = synth.stencil_27pt(40)
    A = api.SpmvMatrix.from_csr(m)
    r = A.profile(reps=5)
    p = r["p"]
    ws = oracle.bounds(m.n_rows, m.n_cols, m.nnz, 4, 8, 8, 1.0)[2]
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    assert r["b_max_gbs"] == oracle.select_bmax(int(ws), l2, r["b_hbm_gbs"], r["b_l2_gbs"])
    p_mb, p_peak, _ = oracle.bounds(m.n_rows, m.n_cols, m.nnz, 4, 8, 8, r["b_max_gbs"])
    assert p["P_MB"] == pytest.approx(p_mb, rel=1e-12)
    assert p["P_peak"] == pytest.approx(p_peak, rel=1e-12)
    flops = 2.0 * m.nnz
    for key, t in (("P_CSR", "t_csr_ms"), ("P_ML", "t_ml_ms"), ("P_CMP", "t_cmp_ms"),
                   ("P_IMB", "t_imb_ms")):
        assert r[t] > 0 and p[key] == pytest.approx(flops / (r[t] * 1e-3) / 1e9, rel=1e-9)
    assert r["t_median_ms"] <= r["t_span_ms"] + 1e-9 and r["n_ctas"] > 0
    el, sm = A.profile_cta_times()
    assert el.shape == (r["n_ctas"],) and sm.shape == (r["n_ctas"],)
    assert np.all(el >= 0) and np.all((sm >= 0) & (sm < 1024)) and el.max() > 0


def test_device_bytes_follow_the_pool_data(api, torch):
    """The handle's device footprint: the CSR arrays at creation, more once a variant builds
    its data (delta index, sliced-row copy)."""
    m = synth.stencil_27pt(30)
    A = api.SpmvMatrix.from_csr(m)
    b0 = A.device_bytes()
    assert b0 >= 4 * (m.n_rows + 1) + 12 * m.nnz
    A.set_variant(index=1, vec=1)
    b1 = A.device_bytes()
    assert b1 >= b0 + 2 * m.nnz + 4 * m.n_rows
    A.set_variant(partition=3, index=1)
    assert A.device_bytes() >= b1 + 10 * m.nnz


# ------------------------------------------------------------------------ MLP --------
SIZES = np.array([12, 32, 32, 4], dtype=np.int32)


def _params(seed):
    return (np.random.default_rng(seed).standard_normal(oracle.mlp_nparams(SIZES)) * 0.3
            ).astype(np.float32)


def _features16(rng, n):
    f = np.zeros((n, 16))
    f[:, 0] = rng.integers(0, 2, n)
    f[:, 1] = rng.uniform(0, 1e-3, n)
    f[:, 2] = rng.integers(0, 5, n)
    f[:, 4] = rng.uniform(1, 60, n)
    f[:, 3] = f[:, 4] * rng.uniform(1, 500, n)
    f[:, 5] = f[:, 4] * rng.uniform(0, 3, n)
    f[:, 8] = rng.uniform(1, 1e6, n)
    f[:, 9] = f[:, 8] * rng.uniform(0, 2, n)
    f[:, 10] = rng.uniform(0, 1, n)
    f[:, 11] = rng.uniform(0, 0.5, n)
    f[:, 12] = rng.uniform(0, 1, n)
    f[:, 13] = f[:, 4] * rng.uniform(0, 1, n)
    f[:, 14] = rng.uniform(1e3, 1e7, n)
    f[:, 15] = f[:, 14] * f[:, 4]
    return f


def test_mlp_inputs_and_logits_bit_exact(abi, torch):
    rng = np.random.default_rng(1)
    f = _features16(rng, 500)
    mu = rng.standard_normal(12).astype(np.float32)
    inv = rng.uniform(0.1, 2, 12).astype(np.float32)
    X = torch.empty((500, 12), dtype=torch.float32, device="cuda")
    # device copies are kept alive until the kernels have read them
    fd, mud, invd = _dev(torch, f), _dev(torch, mu), _dev(torch, inv)
    abi.spmv_mlp_inputs(fd.data_ptr(), 500, mud.data_ptr(), invd.data_ptr(), X.data_ptr(), 0)
    torch.cuda.synchronize()
    Xo = oracle.mlp_inputs(f, mu, inv)
    assert np.array_equal(X.cpu().numpy().view(np.uint32), Xo.view(np.uint32))
    w = _params(2)
    wd = _dev(torch, w)
    L = torch.empty((500, 4), dtype=torch.float32, device="cuda")
    abi.spmv_mlp_logits(SIZES.ctypes.data, wd.data_ptr(), 500, X.data_ptr(), L.data_ptr(), 0)
    torch.cuda.synchronize()
    Lo = oracle.mlp_logits_f32(SIZES, w, Xo)
    assert np.array_equal(L.cpu().numpy().view(np.uint32), Lo.view(np.uint32))


def test_mlp_gradient_matches_fp64_oracle(abi, torch):
    rng = np.random.default_rng(3)
    B = 300
    X = rng.standard_normal((B, 12)).astype(np.float32)
    Y = (rng.random((B, 4)) < 0.4).astype(np.float32)
    w = _params(4)
    g = torch.empty(w.size, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    wd, Xd, Yd = _dev(torch, w), _dev(torch, X), _dev(torch, Y)
    abi.spmv_mlp_loss_grad(SIZES.ctypes.data, wd.data_ptr(), B, Xd.data_ptr(), Yd.data_ptr(),
                           g.data_ptr(), loss.data_ptr(), 0)
    l64, g64, _ = oracle.mlp_loss_grad(SIZES, w.astype(np.float64), X.astype(np.float64),
                                       Y.astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g64) <= 1e-4 * np.linalg.norm(g64)
    assert abs(loss.item() - l64) <= 1e-5 * abs(l64)


def test_mlp_training_reduces_loss(abi, torch):
    rng = np.random.default_rng(5)
    B = 512
    X = rng.standard_normal((B, 12)).astype(np.float32)
    Y = np.stack([X[:, 0] > 0, X[:, 1] > 0.5, X[:, 2] + X[:, 3] > 0, X[:, 4] < -0.2], 1
                 ).astype(np.float32)
    w = _dev(torch, _params(6) * 0.5)
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    hist = torch.empty(400, dtype=torch.float32, device="cuda")
    Xd, Yd = _dev(torch, X), _dev(torch, Y)
    abi.spmv_mlp_train(SIZES.ctypes.data, w.data_ptr(), m.data_ptr(), v.data_ptr(), B,
                       Xd.data_ptr(), Yd.data_ptr(), 400, 0, 1e-2, 0.9, 0.999, 1e-8,
                       hist.data_ptr(), 0)
    h = hist.cpu().numpy()
    assert h[-1] < 0.3 * h[0]
    _, _, probs = oracle.mlp_loss_grad(SIZES, w.cpu().numpy().astype(np.float64),
                                       X.astype(np.float64), Y.astype(np.float64), False)
    assert np.mean((probs > 0.5) == (Y > 0.5)) > 0.9


def test_selector_predict_matches_oracle_decision(api, torch):
    rng = np.random.default_rng(7)
    w = _params(8)
    mu = rng.standard_normal(12).astype(np.float32)
    inv = rng.uniform(0.1, 1, 12).astype(np.float32)
    sel = api.Selector(SIZES, w, mu, inv)
    f = _features16(rng, 200)
    Xo = oracle.mlp_inputs(f, mu, inv)
    Lo = oracle.mlp_logits_f32(SIZES, w, Xo)
    for i in range(200):
        cls, margin = sel.predict(f[i])
        want = sum(1 << o for o in range(4) if Lo[i, o] > 0)
        assert cls == want
        assert margin == pytest.approx(float(np.min(np.abs(Lo[i]))), rel=0, abs=0)


def test_learned_route_uses_selector_and_falls_back(api, torch):
    m = synth.stencil_27pt(30)
    A = api.SpmvMatrix.from_csr(m)
    w = np.zeros(oracle.mlp_nparams(SIZES), dtype=np.float32)
    w[-4:] = [1.0, -1.0, -1.0, -1.0]           # biases of the logits: always {MB}
    sel = api.Selector(SIZES, w)
    r = A.tune("learned", selector=sel, autotune=0)
    assert r.classes == 1 and r.mode_used == 2 and r.variant[1] == 1
    r = A.tune("learned", selector=sel, autotune=0, min_margin=2.0, reps=3)
    assert r.mode_used == 0                    # margin 1 < 2: profiling decided
    x64 = synth.uniform_vector(m.n_cols, 8)
    check_spmv(m, x64, A.run(_dev(torch, x64)).cpu().numpy(), TAU["f64"], "learned")


def test_learned_route_profiles_matrices_outside_the_training_range(api, torch):
    """With a training range set, a matrix whose standardized inputs leave it by more than
    the slack gets margin -1 and is classified by profiling; inside the range the MLP
    decides. The inputs are computed by the oracle to place the range around them."""
    m = synth.stencil_27pt(30)
    A = api.SpmvMatrix.from_csr(m)
    w = np.zeros(oracle.mlp_nparams(SIZES), dtype=np.float32)
    w[-4:] = [1.0, -1.0, -1.0, -1.0]           # biases of the logits: always {MB}
    f16 = np.zeros((1, 16))
    f16[0, :14] = A.features()[0]
    f16[0, 14], f16[0, 15] = m.n_rows, m.nnz
    x = oracle.mlp_inputs(f16, None, None)[0]
    inside = api.Selector(SIZES, w, in_lo=x - 0.1, in_hi=x + 0.1, slack=0.0)
    r = A.tune("learned", selector=inside, autotune=0)
    assert r.mode_used == 2 and r.margin == 1.0 and r.classes == 1
    lo, hi = x - 0.1, x + 0.1
    lo[0], hi[0] = x[0] + 0.5, x[0] + 1.0     # n_rows input below the range by 0.5
    outside = api.Selector(SIZES, w, in_lo=lo, in_hi=hi, slack=0.25)
    assert outside.predict(f16[0])[1] == -1.0
    r = A.tune("learned", selector=outside, autotune=0, reps=3)
    assert r.mode_used == 0 and r.margin == -1.0
    within_slack = api.Selector(SIZES, w, in_lo=lo, in_hi=hi, slack=0.6)
    assert within_slack.predict(f16[0])[1] == 1.0
    from paper_1711_05487_gb300._abi import SpmvError
    with pytest.raises(SpmvError):
        api.Selector(SIZES, w, in_lo=hi, in_hi=lo)


# -------------------------------------------------------------------- batched --------
def test_batched_persistent_matches_oracle(api, torch):
    specs = synth.batched_specs(24, n_lo=500, n_hi=30_000)
    specs.append({"family": "powerlaw", "n": 20_000, "alpha": 1.5, "seed": 99, "index": 99,
                  "k": 4})                                 # rows longer than one chunk
    mats, As, Xs, Ys, ks, X64 = [], [], [], [], [], []
    widths = [dict(), dict(vec=1, vs=1), dict(vec=1, vs=2), dict(vec=1, vs=8), dict(vec=1, vs=32)]
    for i, s in enumerate(specs):
        m = synth.make_from_spec(s, dtype=np.float32)
        A = api.SpmvMatrix.from_csr(m)
        w = widths[i % len(widths)]
        if w.get("vs") == 1 and np.diff(m.rowptr).max() > 64:
            w = dict()        # one lane per row only where rows are short (as the tuner picks)
        A.set_variant(**w)      # the batched kernel takes each handle's sub-warp width
        X = np.random.default_rng(s["seed"]).uniform(-1, 1, (m.n_cols, s["k"])).astype(np.float32)
        mats.append(m)
        As.append(A)
        Xs.append(_dev(torch, X))
        Ys.append(torch.full((m.n_rows, s["k"]), np.nan, dtype=torch.float32, device="cuda"))
        ks.append(s["k"])
        X64.append(X)
    assert max(np.diff(m.rowptr).max() for m in mats) > 4096
    b = api.Batch(As, Xs, Ys, ks)
    from paper_1711_05487_gb300._abi import SpmvError
    with pytest.raises(SpmvError):
        b.set_plan(16, 64)                        # item below the 32-nonzero minimum
    with pytest.raises(SpmvError):
        b.set_plan(1024, 512)                     # chunks shorter than items
    # the default plan, two explicit plans (small items with short chunks; large items with
    # long chunks) and the autotuner's pick all give the oracle's products
    plans = [None, (256, 512), (2048, 8192), "tune"]
    for rep, plan in enumerate(plans):
        if plan == "tune":
            item, chunk = b.tune(reps=2)
            assert item in (256, 512, 1024, 2048) and chunk in (2 * item, 4 * item)
        elif plan is not None:
            b.set_plan(*plan)
        for Y in Ys:
            Y.fill_(np.nan)
        b.run()
        torch.cuda.synchronize()
        for m, X, Y in zip(mats, X64, Ys):
            Yr, Sr = oracle.spmm(m.rowptr, m.colind, m.val, X)
            check_rows(Y.cpu().numpy().astype(np.float64).ravel(), Yr.ravel(), Sr.ravel(),
                       TAU["f32"], f"batched {m.name} plan {plan}")
    for Y in Ys:
        Y.fill_(np.nan)
    b.run_sequential()
    torch.cuda.synchronize()
    for m, X, Y in zip(mats, X64, Ys):
        Yr, Sr = oracle.spmm(m.rowptr, m.colind, m.val, X)
        check_rows(Y.cpu().numpy().astype(np.float64).ravel(), Yr.ravel(), Sr.ravel(),
                   TAU["f32"], f"sequential {m.name}")


def test_batch_refuses_handles_whose_precision_changed(api, torch):
    """The batch reads its handles' arrays in place: once a handle's precision changes (its
    value array reallocated) a batched run answers SPMV_ERR_ARG instead of reading freed
    memory; a handle whose variant change is refused keeps the variant it had."""
    from paper_1711_05487_gb300 import _abi
    mats = [synth.laplacian_2d(40), synth.uniform_random(3000, 12, seed=5)]
    As, Xs, Ys = [], [], []
    for m in mats:
        A = api.SpmvMatrix.from_csr(synth.Csr(m.n_rows, m.n_cols, m.rowptr, m.colind,
                                              m.val.astype(np.float32), m.name))
        A.set_variant()
        As.append(A)
        Xs.append(torch.ones((m.n_cols, 1), dtype=torch.float32, device="cuda"))
        Ys.append(torch.zeros((m.n_rows, 1), dtype=torch.float32, device="cuda"))
    b = api.Batch(As, Xs, Ys, [1, 1])
    b.run()
    torch.cuda.synchronize()
    As[1].set_precision("bf16", "f32", "f32")
    with pytest.raises(_abi.SpmvError) as ei:
        b.run()
    assert ei.value.status == _abi.SPMV_ERR_ARG
    b.close()
    # an invalid variant is refused before anything changes: the installed one still runs
    A = As[0]
    with pytest.raises(_abi.SpmvError):
        A.set_variant(partition=9)
    x = torch.ones(mats[0].n_cols, dtype=torch.float32, device="cuda")
    y = torch.zeros(mats[0].n_rows, dtype=torch.float32, device="cuda")
    A.run(x, y)
    torch.cuda.synchronize()
    yr, sr = oracle.spmv(mats[0].rowptr, mats[0].colind,
                         mats[0].val.astype(np.float32).astype(np.float64), np.ones(mats[0].n_cols))
    check_rows(y.cpu().numpy().astype(np.float64), yr, sr, TAU["f32"], "after refused variant")
