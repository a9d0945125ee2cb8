"""Bit-exact GPU parity of the integer and byte work: CSR validation, value rounding, the
16-bit delta index, merge-path table, Table I features and the selector's pure rules."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TAU, check_spmv, stored_values, torch_cuda

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


FORMAT_MATS = {
    "st27_14": lambda: synth.stencil_27pt(14),
    "lap2d_200": lambda: synth.laplacian_2d(200),                       # 8-bit deltas
    "banded_narrow": lambda: synth.banded(20_000, 60, 0.3, seed=25),     # 8-bit deltas
    "scattered_escape": lambda: synth.scattered(300_000, 4, seed=21),
    "powerlaw": lambda: synth.power_law(50_000, seed=22, dtype=np.float64),
    "ragged_empty": lambda: synth.uniform_random(7001, 80, seed=23, min_per_row=0),
    "banded_wide": lambda: synth.banded(200_000, 70_000, 0.0005, seed=24),
    "identity1": lambda: synth.identity(1),
}


@pytest.mark.parametrize("name", list(FORMAT_MATS))
def test_delta_index_bit_exact_and_round_trip(api, name):
    """The width (8 or 16 bits, one per matrix) and the index equal the oracle's; the CSR
    exported from the index equals the input."""
    m = FORMAT_MATS[name]()
    A = api.SpmvMatrix.from_csr(m)
    A.set_variant(index=1, vec=1)
    base, delta, esc, bits = A.delta()
    assert bits == oracle.delta_width(m.rowptr, m.colind)
    enc = oracle.delta8_encode if bits == 8 else oracle.delta16_encode
    ob, od, oe = enc(m.rowptr, m.colind)
    assert np.array_equal(base.cpu().numpy(), ob)
    assert np.array_equal(delta.cpu().numpy().view(np.uint8 if bits == 8 else np.uint16), od)
    assert np.array_equal(esc.cpu().numpy(), oe)
    rp, ci, v = A.export_csr()
    assert np.array_equal(rp.cpu().numpy(), m.rowptr)
    assert np.array_equal(ci.cpu().numpy(), m.colind)
    assert np.array_equal(v.cpu().numpy().view(np.uint64), m.val.view(np.uint64))


@pytest.mark.parametrize("index", [0, 1])
@pytest.mark.parametrize("name", ["st27_14", "lap2d_200", "scattered_escape", "ragged_empty",
                                  "identity1"])
def test_sell_bit_exact(api, name, index):
    """The sliced-row copy equals the oracle's layout: slice offsets, the stored values at
    their positions, the columns (index 0) or the delta index's deltas (index 1, 8 or 16
    bits, escape rows included), zero padding; FP32 storage keeps its own values."""
    m = FORMAT_MATS[name]()
    soff, perm = oracle.sell32(m.rowptr)
    pad = perm < 0
    src = np.where(pad, 0, perm)
    for storage in ("f64", "f32"):
        A = api.SpmvMatrix.from_csr(m)
        if storage == "f32":
            A.set_precision("f32", "f32", "f32")
        A.set_variant(partition=3, index=index)
        off, v, ix, bits = A.sell()
        assert np.array_equal(off.cpu().numpy(), soff)
        want_v = np.where(pad, 0.0, stored_values(m.val, storage)[src] if m.nnz else 0.0)
        assert np.array_equal(v.cpu().numpy().astype(np.float64), want_v)
        if index == 0:
            assert bits == 0
            want_i = np.where(pad, 0, m.colind[src] if m.nnz else 0)
            assert np.array_equal(ix.cpu().numpy(), want_i)
        else:
            assert bits == oracle.delta_width(m.rowptr, m.colind)
            enc = oracle.delta8_encode if bits == 8 else oracle.delta16_encode
            _, od, _ = enc(m.rowptr, m.colind)
            want_d = np.where(pad, 0, od[src] if m.nnz else 0)
            got = ix.cpu().numpy().view(np.uint8 if bits == 8 else np.uint16)
            assert np.array_equal(got, want_d)


@pytest.mark.parametrize("name", list(FORMAT_MATS))
def test_merge_path_table_bit_exact(api, name):
    m = FORMAT_MATS[name]()
    A = api.SpmvMatrix.from_csr(m)
    A.set_variant(partition=1)
    c, items = A.merge_path()
    assert np.array_equal(c.cpu().numpy(), oracle.merge_path(m.rowptr, items))


def test_value_rounding_bit_exact(abi, torch):
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.standard_normal(200_000) * 2.0 ** rng.integers(-150, 130, 200_000),
                        [0.0, -0.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, (2 - 2 ** -8) * 2.0 ** 127,
                         2.0 ** -133, 2.0 ** -134, 3 * 2.0 ** -134, 1e-300, 3.5e38, 1e308,
                         np.inf, -np.inf, np.nan]])
    vin = torch.from_numpy(v).cuda()
    o32 = torch.empty(v.size, dtype=torch.float32, device="cuda")
    o16 = torch.empty(v.size, dtype=torch.int16, device="cuda")
    abi.spmv_round_values(vin.data_ptr(), o32.data_ptr(), v.size, abi.SPMV_F32, 0)
    abi.spmv_round_values(vin.data_ptr(), o16.data_ptr(), v.size, abi.SPMV_BF16, 0)
    torch.cuda.synchronize()
    with np.errstate(over="ignore"):
        assert np.array_equal(o32.cpu().numpy().view(np.uint32),
                              oracle.round_f32(v).view(np.uint32))
    assert np.array_equal(o16.cpu().numpy().view(np.uint16), oracle.round_bf16_bits(v))


def test_row_bins_bit_exact(api, torch):
    """The row decomposition tables equal the oracle's, for a matrix with short, medium and
    long rows and for one with none of the latter two."""
    for m in (synth.power_law(60_000, alpha=1.4, clip=60_000, seed=19, dtype=np.float64),
              synth.laplacian_2d(40)):
        A = api.SpmvMatrix.from_csr(m)
        A.set_variant(partition=2, index=1)
        med, lng, first, ch = (t.cpu().numpy() for t in A.row_bins())
        om, ol, of, oc = oracle.row_bins(m.rowptr, m.colind, l_med=64, chunk=4096)
        assert np.array_equal(med, om) and np.array_equal(lng, ol)
        assert np.array_equal(first, of) and np.array_equal(ch, oc)


def test_row_bins_long_rows_repeatable(api, torch):
    """Long rows split into many chunks (up to 67): their partials are added in chunk order,
    so ten SpMVs in a row, on two handles, give the same bits, within the FP64 bound of the
    oracle."""
    m = synth.power_law(20_000, alpha=1.5, clip=20_000, seed=22, dtype=np.float64)
    x = torch.from_numpy(synth.uniform_vector(m.n_cols, 23)).cuda()
    ys = []
    for _ in range(2):
        A = api.SpmvMatrix.from_csr(m)
        A.set_variant(partition=2, bin_med=16, bin_chunk=300)
        for _ in range(10):
            ys.append(A.run(x).cpu().numpy())
    assert all(np.array_equal(y.view(np.uint64), ys[0].view(np.uint64)) for y in ys)
    check_spmv(m, x.cpu().numpy(), ys[0], TAU["f64"], "bins repeat")
    _, lng, first, _ = (t.cpu().numpy() for t in A.row_bins())
    assert lng.size > 50 and np.diff(first).max() > 20   # many long rows, some of many chunks


@pytest.mark.parametrize("l_med,chunk", [(2, 2), (32, 2048), (128, 8192), (64, 300),
                                         (1000, 1000)])
def test_row_bins_at_other_limits(api, torch, l_med, chunk):
    """A variant's own row decomposition limits: the tables equal the oracle's at those
    limits bit for bit (rebuilt when the limits change), and the SpMV stays within the FP64
    bound (FP32 too, for FP32 storage)."""
    m = synth.power_law(30_000, alpha=1.5, clip=30_000, seed=20, dtype=np.float64)
    x64 = synth.uniform_vector(m.n_cols, 21)
    A = api.SpmvMatrix.from_csr(m)
    for index in (0, 1):
        A.set_variant(partition=2, index=index, bin_med=l_med, bin_chunk=chunk)
        med, lng, first, ch = (t.cpu().numpy() for t in A.row_bins())
        om, ol, of, oc = oracle.row_bins(m.rowptr, m.colind, l_med=l_med, chunk=chunk)
        assert np.array_equal(med, om) and np.array_equal(lng, ol)
        assert np.array_equal(first, of) and np.array_equal(ch, oc)
        y = A.run(torch.from_numpy(x64).cuda()).cpu().numpy()
        check_spmv(m, x64, y, TAU["f64"], f"bins {l_med}/{chunk} index {index}")
    A32 = api.SpmvMatrix.from_csr(m.astype(np.float32))
    A32.set_variant(partition=2, bin_med=l_med, bin_chunk=chunk)
    x32 = x64.astype(np.float32)
    y = A32.run(torch.from_numpy(x32).cuda()).double().cpu().numpy()
    check_spmv(m.astype(np.float32), x32.astype(np.float64), y, TAU["f32"],
               f"bins f32 {l_med}/{chunk}")


def test_row_bin_limits_rejected(api):
    from paper_1711_05487_gb300._abi import SpmvError
    A = api.SpmvMatrix.from_csr(synth.laplacian_2d(20))
    for med, chunk in ((1, 0), (100, 50), (0, 1 << 21), (-3, 0)):
        with pytest.raises(SpmvError):
            A.set_variant(partition=2, bin_med=med, bin_chunk=chunk)


@pytest.mark.parametrize("n_panels", [2, 3, 7, 16])
def test_col_panels_bit_exact(api, torch, n_panels):
    """The column-panel copy (row pointers, columns, values in the storage dtype) equals the
    oracle's panel-major copy bit for bit: rows with and without nonzeros in a panel, empty
    rows, a row longer than a warp, empty trailing panels (16 panels of 32 columns over a
    100-column matrix), and FP32 storage."""
    mats = [synth.uniform_random(5000, 90, seed=27, min_per_row=0, n_cols=70_000),
            synth.scattered(20_000, 8, seed=28),
            synth.uniform_random(300, 12, seed=29, min_per_row=0, n_cols=100)]
    for m in mats:
        for storage in ("f64", "f32", "df64"):
            A = api.SpmvMatrix.from_csr(m)
            if storage != "f64":
                A.set_precision(storage, "f64" if storage == "df64" else "f32",
                                "df64" if storage == "df64" else "f32")
            A.set_variant(xpath=n_panels, vs=2)
            rp, ci, v, w = A.col_panels()
            prow, perm, ow = oracle.col_panels(m.rowptr, m.colind, m.n_cols, n_panels)
            assert w == ow
            assert np.array_equal(rp.cpu().numpy(), prow)
            assert np.array_equal(ci.cpu().numpy(), m.colind[perm])
            want = stored_values(m.val, "f64" if storage == "df64" else storage)[perm]
            got = v.cpu().numpy() if storage != "f32" else v.cpu().numpy().astype(np.float64)
            assert np.array_equal(got, want)


def test_df_split_bit_exact(abi, torch):
    """Double-float value pairs (DF64 storage) equal the oracle's split bit for bit."""
    rng = np.random.default_rng(31)
    v = np.concatenate([rng.standard_normal(200_000) * 2.0 ** rng.integers(-48, 48, 200_000),
                        [0.0, -0.0, 1.0, 1 + 2 ** -30, 1 + 2 ** -52, -3.75, 2.0 ** -40,
                         2.0 ** 41, 2.0 ** 41 - 2.0 ** -12, 2.0 ** -41, 1e-310, 1e308,
                         np.inf, -np.inf, np.nan, -(1 + 2 ** -46)]])
    vin = torch.from_numpy(v).cuda()
    out = torch.empty((v.size, 2), dtype=torch.int32, device="cuda")
    abi.spmv_round_values(vin.data_ptr(), out.data_ptr(), v.size, abi.SPMV_DF64, 0)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy().view(np.uint32), oracle.df_split_bits(v))


def test_validation_codes_match_oracle(abi, torch):
    cases = [
        (2, 4, [0, 2, 3], [0, 3, 1]),
        (2, 4, [1, 2, 3], [0, 3, 1]),
        (2, 4, [0, 3, 2], [0, 3]),
        (2, 4, [0, 2, 2], [0, 3, 1]),
        (2, 3, [0, 2, 3], [0, 3, 1]),
        (2, 4, [0, 2, 3], [0, 3, -1]),
        (2, 4, [0, 2, 3], [3, 0, 1]),
        (2, 4, [0, 2, 3], [3, 3, 1]),
        (3, 9, [0, 3, 3, 6], [0, 4, 2, 5, 8, 9]),
        (3, 9, [0, 3, 3, 6], [0, 4, 9, 5, 5, 8]),
    ]
    for n_rows, n_cols, rp, ci in cases:
        rp_d = torch.tensor(rp, dtype=torch.int32, device="cuda")
        ci_d = torch.tensor(ci + [0], dtype=torch.int32, device="cuda")
        code = abi.spmv_validate_csr(n_rows, n_cols, len(ci), rp_d.data_ptr(), ci_d.data_ptr(), 0)
        want = oracle.validate_csr(n_rows, n_cols, np.array(rp, np.int32), np.array(ci, np.int32))
        assert code == want, (rp, ci, code, want)


def test_create_rejects_invalid_csr(api):
    from paper_1711_05487_gb300._abi import SpmvError
    with pytest.raises(SpmvError) as e:
        api.SpmvMatrix(2, 4, np.array([0, 2, 3], np.int32), np.array([3, 0, 1], np.int32),
                       np.ones(3))
    assert e.value.status == 1


FEATURE_MATS = {
    "lap256": lambda: synth.laplacian_2d(256),
    "st27_20": lambda: synth.stencil_27pt(20),
    "powerlaw": lambda: synth.power_law(100_000, seed=31, dtype=np.float64),
    "scattered": lambda: synth.scattered(200_000, 8, seed=32),
    "ragged_empty": lambda: synth.uniform_random(9001, 100, seed=33, min_per_row=0),
    "banded": lambda: synth.banded(50_000, 2000, 0.05, seed=34),
}


@pytest.mark.parametrize("name", list(FEATURE_MATS))
@pytest.mark.parametrize("vec", ["f64", "f32"])
def test_features_bit_exact(api, torch, name, vec):
    m = FEATURE_MATS[name]()
    A = api.SpmvMatrix.from_csr(m)
    if vec == "f32":
        A.set_precision("f32", "f32", "f32")
    f, isum = A.features(line_bytes=128)
    vb = 8 if vec == "f64" else 4
    sb = 8 if vec == "f64" else 4
    ws = 4 * (m.n_rows + 1) + (4 + sb) * m.nnz + vb * (m.n_rows + m.n_cols)
    l2 = torch.cuda.get_device_properties(0).L2_cache_size
    of, oi = oracle.features(m.n_rows, m.n_cols, m.rowptr, m.colind, line_elems=128 // vb,
                             ws_bytes=ws, llc_bytes=l2)
    assert np.array_equal(f.view(np.uint64), of.view(np.uint64)), (f, of)
    assert np.array_equal(isum, oi)


def test_delta_widths_cover_both_cases():
    """The matrices above exercise both widths: 8 bits where every gap is at most 255 (the
    14^3 stencil's plane gap is 196), 16 bits where the plane gap is larger."""
    widths = {name: oracle.delta_width(m.rowptr, m.colind)
              for name, m in ((n, g()) for n, g in FORMAT_MATS.items())}
    assert widths["lap2d_200"] == 8 and widths["st27_14"] == 8
    assert widths["banded_wide"] == 16 and widths["scattered_escape"] == 16
