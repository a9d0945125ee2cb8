"""CPU oracle for the bottleneck-adaptive CSR SpMV method (arXiv 1711.05487).

TEST INFRASTRUCTURE ONLY. This package is the plain, slow reference that the GPU library
is checked against: a C file (``spmv_oracle.c``, FP64, no blocking or reordering beyond
the paper's own loops) plus thin numpy wrappers. Only ``tests/``, the package entry
point's ``smoke()`` and ``bench.py``'s CPU-baseline leg may import it. It imports nothing
from the GPU package and the GPU package imports nothing from it.

Functions whose results are tied to the paper or to mathematics by a test are "pinned";
the per-class bounds that are measurements (P_ML, P_CMP, P_IMB) have no value to pin:
only their construction is checked (parity unpinned for those three measurements).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spmv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

CLASS_MB, CLASS_ML, CLASS_IMB, CLASS_CMP = 1, 2, 4, 8
FEATURE_NAMES = ("size", "density", "nnz_min", "nnz_max", "nnz_avg", "nnz_sd", "bw_min",
                 "bw_max", "bw_avg", "bw_sd", "scatter_avg", "scatter_sd",
                 "clustering_avg", "misses_avg")


# Compiler flags. -ffp-contract=off keeps every FP64 operation rounded as written (no fused
# multiply-adds), which the fixed-order MLP inference and the exact pins rely on; -O3 is the
# optimisation level of the timed CPU baseline. No -march=native: the same flags build the
# same arithmetic on the x86 and Arm hosts.
BUILD_FLAGS = ("-O3", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    stamp = os.path.join(_BUILD, "flags.txt")
    flags = " ".join(BUILD_FLAGS)
    if (not force and os.path.exists(_LIB_PATH) and os.path.exists(stamp)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)
            and open(stamp).read() == flags):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", *BUILD_FLAGS, "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    # OpenMP only serves the static-partition baseline; without it that runs on one thread
    if subprocess.run(cmd, capture_output=True).returncode != 0:
        subprocess.run([c for c in cmd if c != "-fopenmp"], check=True)
    os.replace(tmp, _LIB_PATH)
    with open(stamp, "w") as fh:
        fh.write(flags)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double


def _declare(L):
    L.oracle_validate_csr.argtypes = [_I64, _I64, _I64, _P, _P]
    L.oracle_validate_csr.restype = ctypes.c_int
    L.oracle_spmv_f64.argtypes = [_I64, _P, _P, _P, _P, _P, _P]
    L.oracle_spmv_f64.restype = None
    L.oracle_spmv_rows_f64.argtypes = [_P, _I64, _P, _P, _P, _P, _P, _P]
    L.oracle_spmv_rows_f64.restype = None
    L.oracle_spmm_f64.argtypes = [_I64, _P, _P, _P, _P, _I64, _P, _P]
    L.oracle_spmm_f64.restype = None
    L.oracle_round_f32.argtypes = [_P, _P, _I64]
    L.oracle_round_f32.restype = None
    L.oracle_round_bf16.argtypes = [_P, _P, _I64]
    L.oracle_round_bf16.restype = None
    L.oracle_df_split.argtypes = [_P, _P, _I64]
    L.oracle_df_split.restype = None
    L.oracle_spmv_f64_static.argtypes = [_I64, _P, _P, _P, _P, _P, ctypes.c_int32]
    L.oracle_spmv_f64_static.restype = ctypes.c_int32
    L.oracle_row_bins.argtypes = [_I64, _P, _P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P, _P,
                                  _P]
    L.oracle_row_bins.restype = None
    L.oracle_cg.argtypes = [_I64, _P, _P, _P, _P, _P, _I64, _D, _P, _P]
    L.oracle_cg.restype = _I64
    L.oracle_delta16_encode.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.oracle_delta16_encode.restype = _I64
    L.oracle_delta16_decode.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.oracle_delta16_decode.restype = None
    L.oracle_delta8_encode.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.oracle_delta8_encode.restype = _I64
    L.oracle_delta8_decode.argtypes = [_I64, _P, _P, _P, _P, _P]
    L.oracle_delta8_decode.restype = None
    L.oracle_delta_width.argtypes = [_I64, _P, _P]
    L.oracle_delta_width.restype = ctypes.c_int32
    L.oracle_sell32.argtypes = [_I64, _P, _P, _P]
    L.oracle_sell32.restype = _I64
    L.oracle_panel_width.argtypes = [_I64, ctypes.c_int32]
    L.oracle_panel_width.restype = ctypes.c_int32
    L.oracle_col_panels.argtypes = [_I64, _I64, _P, _P, ctypes.c_int32, _P, _P]
    L.oracle_col_panels.restype = None
    L.oracle_merge_path.argtypes = [_I64, _I64, _P, _I64, _P]
    L.oracle_merge_path.restype = None
    L.oracle_features.argtypes = [_I64, _I64, _P, _P, _I64, _I64, _I64, _P, _P]
    L.oracle_features.restype = None
    L.oracle_bounds.argtypes = [_I64, _I64, _I64, _I64, _I64, _I64, _D, _P]
    L.oracle_bounds.restype = None
    L.oracle_select_bmax.argtypes = [_I64, _I64, _D, _D]
    L.oracle_select_bmax.restype = _D
    L.oracle_classify.argtypes = [_P, _D, _D, _D]
    L.oracle_classify.restype = ctypes.c_uint32
    L.oracle_classify2.argtypes = [_P, _P, _D, _D, _D]
    L.oracle_classify2.restype = ctypes.c_uint32
    L.oracle_variant_for_classes.argtypes = [ctypes.c_uint32, _D, _D, _D, _P]
    L.oracle_variant_for_classes.restype = None
    L.oracle_amortization_iters.argtypes = [_D, _D, _D]
    L.oracle_amortization_iters.restype = _D
    L.oracle_mlp_nparams.argtypes = [_P]
    L.oracle_mlp_nparams.restype = _I64
    L.oracle_mlp_loss_grad_f64.argtypes = [_P, _P, _I64, _P, _P, _P, _P]
    L.oracle_mlp_loss_grad_f64.restype = _D
    L.oracle_mlp_logits_f32.argtypes = [_P, _P, _I64, _P, _P]
    L.oracle_mlp_logits_f32.restype = None
    L.oracle_log2p1_f32.argtypes = [ctypes.c_float]
    L.oracle_log2p1_f32.restype = ctypes.c_float
    L.oracle_log2p1_f32_array.argtypes = [_P, _P, _I64]
    L.oracle_log2p1_f32_array.restype = None
    L.oracle_feature_rules.argtypes = [_P, _I64, _I64, _I64, _D]
    L.oracle_feature_rules.restype = ctypes.c_uint32
    L.oracle_mlp_inputs.argtypes = [_P, _I64, _P, _P, _P]
    L.oracle_mlp_inputs.restype = None


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ------------------------------------------------------------------------------ CSR
def validate_csr(n_rows, n_cols, rowptr, colind) -> int:
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    return int(lib().oracle_validate_csr(n_rows, n_cols, ci.shape[0], _p(rp), _p(ci)))


def spmv(rowptr, colind, val, x):
    """FP64 y = A x and s = sum |a_ij x_j| (Fig. 1). Values and x are widened to FP64
    exactly (FP32 and BF16 storage values are exact in FP64)."""
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    v, xx = _c(val, np.float64), _c(x, np.float64)
    n = rp.shape[0] - 1
    y, s = np.empty(n), np.empty(n)
    lib().oracle_spmv_f64(n, _p(rp), _p(ci), _p(v), _p(xx), _p(y), _p(s))
    return y, s


def spmv_rows(rows, rowptr, colind, val, x):
    r = _c(rows, np.int64)
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    v, xx = _c(val, np.float64), _c(x, np.float64)
    y, s = np.empty(r.shape[0]), np.empty(r.shape[0])
    lib().oracle_spmv_rows_f64(_p(r), r.shape[0], _p(rp), _p(ci), _p(v), _p(xx), _p(y), _p(s))
    return y, s


def spmm(rowptr, colind, val, X):
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    v, XX = _c(val, np.float64), _c(X, np.float64)
    n, k = rp.shape[0] - 1, XX.shape[1]
    Y, S = np.empty((n, k)), np.empty((n, k))
    lib().oracle_spmm_f64(n, _p(rp), _p(ci), _p(v), _p(XX), k, _p(Y), _p(S))
    return Y, S


# ------------------------------------------------------------------------ precision
def round_f32(v) -> np.ndarray:
    a = _c(v, np.float64)
    out = np.empty(a.shape[0], dtype=np.float32)
    lib().oracle_round_f32(_p(a), _p(out), a.shape[0])
    return out


def round_bf16_bits(v) -> np.ndarray:
    a = _c(v, np.float64)
    out = np.empty(a.shape[0], dtype=np.uint16)
    lib().oracle_round_bf16(_p(a), _p(out), a.shape[0])
    return out


def df_split_bits(v) -> np.ndarray:
    """Double-float split: uint32 array (n, 2) of FP32 bit patterns (hi, lo)."""
    a = _c(v, np.float64)
    out = np.empty((a.shape[0], 2), dtype=np.uint32)
    lib().oracle_df_split(_p(a), _p(out), a.shape[0])
    return out


def row_bins(rowptr, colind, l_med=64, chunk=4096):
    """(med_rows, long_rows, long_first, chunks (n, 4)) of the row decomposition."""
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    n = rp.shape[0] - 1
    lens = np.diff(rp.astype(np.int64))
    max_ch = int(np.sum((lens + chunk - 1) // chunk)) + 1
    med = np.empty(max(n, 1), np.int32)
    lng = np.empty(max(n, 1), np.int32)
    first = np.empty(n + 1, np.int32)
    ch = np.empty((max_ch, 4), np.int32)
    counts = np.zeros(3, np.int64)
    lib().oracle_row_bins(n, _p(rp), _p(ci), l_med, chunk, _p(med), _p(lng), _p(first), _p(ch),
                          _p(counts))
    a, b, c = (int(v) for v in counts)
    return med[:a], lng[:b], first[:b + 1], ch[:c]


def sell32(rowptr):
    """(soff, perm) of the sliced-row layout: slice s spans positions [soff[s], soff[s+1]),
    element k of row 32 s + l at soff[s] + 32 k + l; perm = CSR position or -1 (padding)."""
    rp = _c(rowptr, np.int32)
    n = rp.shape[0] - 1
    ns = (n + 31) // 32
    lens = np.diff(rp.astype(np.int64))
    bound = 0
    for s in range(0, n, 32):
        bound += 32 * int(lens[s:s + 32].max()) if lens[s:s + 32].size else 0
    soff = np.empty(ns + 1, np.int64)
    perm = np.empty(max(bound, 1), np.int32)
    tot = lib().oracle_sell32(n, _p(rp), _p(soff), _p(perm))
    return soff, perm[:tot]


def panel_width(n_cols: int, n_panels: int) -> int:
    """Columns per panel: ceil(n_cols / n_panels) rounded up to a multiple of 32."""
    return int(lib().oracle_panel_width(int(n_cols), int(n_panels)))


def col_panels(rowptr, colind, n_cols: int, n_panels: int):
    """(prow (n_panels, n_rows + 1), perm, width) of the column-panel copy: panel p's rows
    are prow[p] into the copy, whose columns are colind[perm] and values val[perm]."""
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    n = rp.shape[0] - 1
    prow = np.empty((n_panels, n + 1), np.int32)
    perm = np.empty(max(ci.shape[0], 1), np.int32)
    lib().oracle_col_panels(n, int(n_cols), _p(rp), _p(ci), int(n_panels), _p(prow), _p(perm))
    return prow, perm[:ci.shape[0]], panel_width(n_cols, n_panels)


def spmv_static(rowptr, colind, val, x, n_threads: int):
    """The paper's static nnz-balanced baseline on n_threads OpenMP threads; returns
    (y, threads used). y equals spmv()'s bit for bit."""
    rp, ci, v, xx = (_c(rowptr, np.int32), _c(colind, np.int32), _c(val, np.float64),
                     _c(x, np.float64))
    n = rp.shape[0] - 1
    y = np.empty(n, dtype=np.float64)
    used = lib().oracle_spmv_f64_static(n, _p(rp), _p(ci), _p(v), _p(xx), _p(y), int(n_threads))
    return y, int(used)


def cg(rowptr, colind, val, b, x0=None, max_iters=1000, rtol=1e-10):
    """Conjugate gradients; returns (x, iterations, converged, ||r_k|| for k = 0..iterations)."""
    rp, ci, v = _c(rowptr, np.int32), _c(colind, np.int32), _c(val, np.float64)
    bb = _c(b, np.float64)
    n = bb.shape[0]
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    hist = np.zeros(max_iters + 1)
    conv = np.zeros(1, dtype=np.int32)
    k = lib().oracle_cg(n, _p(rp), _p(ci), _p(v), _p(bb), _p(x), max_iters, float(rtol),
                        _p(hist), _p(conv))
    return x, int(k), bool(conv[0]), hist[:k + 1]


def bf16_bits_to_f64(bits) -> np.ndarray:
    b = _c(bits, np.uint16).astype(np.uint32) << 16
    return b.view(np.float32).astype(np.float64)


# ------------------------------------------------------------------------- formats
def delta16_encode(rowptr, colind):
    """Returns (base int32[N], delta uint16[NNZ], esc_col int32[n_esc])."""
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    n = rp.shape[0] - 1
    base = np.empty(n, dtype=np.int32)
    delta = np.empty(ci.shape[0], dtype=np.uint16)
    esc = np.empty(max(1, ci.shape[0]), dtype=np.int32)
    n_esc = lib().oracle_delta16_encode(n, _p(rp), _p(ci), _p(base), _p(delta), _p(esc))
    return base, delta, esc[:n_esc].copy()


def delta8_encode(rowptr, colind):
    """Returns (base int32[N], delta uint8[NNZ], esc_col int32[n_esc])."""
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    n = rp.shape[0] - 1
    base = np.empty(n, dtype=np.int32)
    delta = np.empty(ci.shape[0], dtype=np.uint8)
    esc = np.empty(max(1, ci.shape[0]), dtype=np.int32)
    n_esc = lib().oracle_delta8_encode(n, _p(rp), _p(ci), _p(base), _p(delta), _p(esc))
    return base, delta, esc[:n_esc].copy()


def delta8_decode(rowptr, base, delta, esc_col):
    rp = _c(rowptr, np.int32)
    b, d = _c(base, np.int32), _c(delta, np.uint8)
    e = _c(esc_col if len(esc_col) else np.zeros(1, np.int32), np.int32)
    out = np.empty(d.shape[0], dtype=np.int32)
    lib().oracle_delta8_decode(rp.shape[0] - 1, _p(rp), _p(b), _p(d), _p(e), _p(out))
    return out


def delta_width(rowptr, colind) -> int:
    """8 or 16: the per-matrix width of the delta index."""
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    return int(lib().oracle_delta_width(rp.shape[0] - 1, _p(rp), _p(ci)))


def delta16_decode(rowptr, base, delta, esc_col):
    rp = _c(rowptr, np.int32)
    b, d = _c(base, np.int32), _c(delta, np.uint16)
    e = _c(esc_col if len(esc_col) else np.zeros(1, np.int32), np.int32)
    out = np.empty(d.shape[0], dtype=np.int32)
    lib().oracle_delta16_decode(rp.shape[0] - 1, _p(rp), _p(b), _p(d), _p(e), _p(out))
    return out


def merge_path(rowptr, items_per_tile: int) -> np.ndarray:
    """(rows ended, nonzeros consumed) at every tile boundary: int32[n_tiles + 1, 2]."""
    rp = _c(rowptr, np.int32)
    n = rp.shape[0] - 1
    nnz = int(rp[-1])
    n_tiles = -(-(n + nnz) // items_per_tile)
    out = np.zeros((n_tiles + 1, 2), dtype=np.int32)
    lib().oracle_merge_path(n, nnz, _p(rp), items_per_tile, _p(out))
    return out


# ------------------------------------------------------------------------ features
def features(n_rows, n_cols, rowptr, colind, line_elems=16, ws_bytes=0, llc_bytes=0):
    """Table I features (14 doubles, FEATURE_NAMES order) and 12 exact integer sums."""
    rp, ci = _c(rowptr, np.int32), _c(colind, np.int32)
    out = np.empty(14)
    isum = np.empty(12, dtype=np.uint64)
    lib().oracle_features(n_rows, n_cols, _p(rp), _p(ci), line_elems, ws_bytes, llc_bytes,
                          _p(out), _p(isum))
    return out, isum


# ------------------------------------------------------------- bounds and classify
def bounds(n_rows, n_cols, nnz, idx_bytes, val_bytes, vec_bytes, b_max_gbs):
    out = np.empty(3)
    lib().oracle_bounds(n_rows, n_cols, nnz, idx_bytes, val_bytes, vec_bytes, b_max_gbs,
                        _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def select_bmax(ws_bytes, llc_bytes, b_main, b_llc) -> float:
    return float(lib().oracle_select_bmax(int(ws_bytes), int(llc_bytes), b_main, b_llc))


def classify(p_csr, p_mb, p_ml, p_imb, p_cmp, p_peak, t_imb=1.24, t_ml=1.25, t_mb=0.75):
    p = np.array([p_csr, p_mb, p_ml, p_imb, p_cmp, p_peak], dtype=np.float64)
    return int(lib().oracle_classify(_p(p), t_imb, t_ml, t_mb))


def classify2(p6, p2=None, t_imb=1.24, t_ml=1.25, t_mb=0.75):
    p = np.ascontiguousarray(p6, dtype=np.float64)
    q = None if p2 is None else np.ascontiguousarray(p2, dtype=np.float64)
    return int(lib().oracle_classify2(_p(p), None if q is None else _p(q), t_imb, t_ml, t_mb))


def variant_for_classes(cls, nnz_avg, nnz_max, long_ratio=32.0):
    out = np.zeros(4, dtype=np.int32)
    lib().oracle_variant_for_classes(int(cls), float(nnz_avg), float(nnz_max),
                                     float(long_ratio), _p(out))
    return tuple(int(v) for v in out)


def amortization_iters(t_pre, t_base, t_opt) -> float:
    return float(lib().oracle_amortization_iters(t_pre, t_base, t_opt))


def feature_rules(features14, n_cols, vec_bytes, llc_bytes, long_ratio=32.0) -> int:
    f = _c(features14, np.float64)
    return int(lib().oracle_feature_rules(_p(f), int(n_cols), int(vec_bytes), int(llc_bytes),
                                          float(long_ratio)))


# ------------------------------------------------------------------------------ MLP
MLP_INPUTS = 12


def mlp_inputs(feat16, mu=None, inv_sigma=None) -> np.ndarray:
    """FP32 selector inputs from rows of 16 doubles (14 features, n_rows, nnz)."""
    f = _c(np.atleast_2d(feat16), np.float64)
    out = np.empty((f.shape[0], MLP_INPUTS), dtype=np.float32)
    m = None if mu is None else _c(mu, np.float32)
    s = None if inv_sigma is None else _c(inv_sigma, np.float32)
    lib().oracle_mlp_inputs(_p(f), f.shape[0], None if m is None else _p(m),
                            None if s is None else _p(s), _p(out))
    return out


def mlp_nparams(sizes) -> int:
    s = _c(sizes, np.int32)
    return int(lib().oracle_mlp_nparams(_p(s)))


def mlp_loss_grad(sizes, params, X, Y, want_grad=True):
    s = _c(sizes, np.int32)
    prm = _c(params, np.float64)
    XX, YY = _c(X, np.float64), _c(Y, np.float64)
    g = np.empty_like(prm) if want_grad else None
    probs = np.empty((XX.shape[0], int(s[3])))
    loss = lib().oracle_mlp_loss_grad_f64(_p(s), _p(prm), XX.shape[0], _p(XX), _p(YY),
                                          _p(g) if g is not None else None, _p(probs))
    return float(loss), g, probs


def mlp_logits_f32(sizes, params, X):
    s = _c(sizes, np.int32)
    prm = _c(params, np.float32)
    XX = _c(X, np.float32)
    out = np.empty((XX.shape[0], int(s[3])), dtype=np.float32)
    lib().oracle_mlp_logits_f32(_p(s), _p(prm), XX.shape[0], _p(XX), _p(out))
    return out


def log2p1_f32(v) -> np.ndarray:
    a = _c(np.atleast_1d(v), np.float32)
    out = np.empty_like(a)
    lib().oracle_log2p1_f32_array(_p(a), _p(out), a.shape[0])
    return out


# ---------------------------------------------------------------- selector metrics
def exact_match_ratio(pred_masks, true_masks) -> float:
    """Section IV-B: share of samples whose predicted class set equals the label set."""
    p, t = np.asarray(pred_masks), np.asarray(true_masks)
    return float(np.mean(p == t)) if p.size else 0.0


def partial_match_ratio(pred_masks, true_masks) -> float:
    """Section IV-B: share of samples whose prediction contains at least one correct
    class. A sample whose label set is empty counts as matched when the prediction is
    empty too (the dummy class of Section III-D)."""
    p, t = np.asarray(pred_masks), np.asarray(true_masks)
    if not p.size:
        return 0.0
    hit = ((p & t) != 0) | ((p == 0) & (t == 0))
    return float(np.mean(hit))


def harmonic_mean(rates) -> float:
    """Section IV-A: rates are summarised over runs with the harmonic mean."""
    r = np.asarray(rates, dtype=np.float64)
    return float(r.size / np.sum(1.0 / r))
