"""ctypes binding of include/spmv_gb300.h: the same entry points, argument marshalling only.

Every function here forwards to the CUDA library and raises SpmvError on a non-zero status.
Pointers are plain integers (device addresses from torch tensors' data_ptr(), or host
addresses); streams are cudaStream_t integers (torch.cuda.Stream.cuda_stream). Nothing is
computed on the host: when the library is missing the import fails loudly.
"""
from __future__ import annotations

import ctypes
import os

from . import buildlib as _build

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_D = ctypes.c_double
_F = ctypes.c_float

SPMV_F64, SPMV_F32, SPMV_BF16, SPMV_DF64 = 0, 1, 2, 3
TUNE_PROFILE, TUNE_FEATURES, TUNE_LEARNED, TUNE_FIXED = 0, 1, 2, 3
CLASS_MB, CLASS_ML, CLASS_IMB, CLASS_CMP = 1, 2, 4, 8
NUM_FEATURES = 14
MLP_INPUTS = 12

STATUS = {0: "SPMV_OK", 1: "SPMV_ERR_INVALID_CSR", 2: "SPMV_ERR_UNSUPPORTED_DTYPE",
          3: "SPMV_ERR_OOM", 4: "SPMV_ERR_NOT_TUNED", 5: "SPMV_ERR_CUDA",
          6: "SPMV_ERR_TIMEOUT", 7: "SPMV_ERR_ARG", 8: "SPMV_ERR_NO_SELECTOR",
          9: "SPMV_ERR_TOO_LARGE"}
(SPMV_OK, SPMV_ERR_INVALID_CSR, SPMV_ERR_UNSUPPORTED_DTYPE, SPMV_ERR_OOM, SPMV_ERR_NOT_TUNED,
 SPMV_ERR_CUDA, SPMV_ERR_TIMEOUT, SPMV_ERR_ARG, SPMV_ERR_NO_SELECTOR, SPMV_ERR_TOO_LARGE) = range(10)


class SpmvError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class spmv_variant(ctypes.Structure):
    _fields_ = [("partition", _I32), ("index", _I32), ("xpath", _I32), ("vec", _I32),
                ("vs", _I32), ("tile_rows", _I32), ("tile_pipe", _I32), ("bin_med", _I32),
                ("bin_chunk", _I32)]

    def as_tuple(self):
        return (self.partition, self.index, self.xpath, self.vec, self.vs, self.tile_rows,
                self.tile_pipe, self.bin_med, self.bin_chunk)

    def __repr__(self):
        return (f"spmv_variant(partition={self.partition}, index={self.index}, "
                f"xpath={self.xpath}, vec={self.vec}, vs={self.vs}, "
                f"tile_rows={self.tile_rows}, tile_pipe={self.tile_pipe}, "
                f"bin_med={self.bin_med}, bin_chunk={self.bin_chunk})")


class spmv_tune_opts(ctypes.Structure):
    _fields_ = [("t_imb", _D), ("t_ml", _D), ("t_mb", _D), ("long_row_ratio", _D),
                ("autotune", _I32), ("reps", _I32), ("fixed", spmv_variant),
                ("selector", _P), ("min_margin", _D), ("second_pass", _I32),
                ("bin_med", _I32), ("bin_chunk", _I32)]


class spmv_tune_report(ctypes.Structure):
    _fields_ = [("classes", _U32), ("mode_used", _I32), ("variant", spmv_variant),
                ("p", _D * 6), ("p2", _D * 2), ("b_max_gbs", _D),
                ("features", _D * NUM_FEATURES),
                ("margin", _D), ("t_pre_ms", _D), ("t_classify_ms", _D), ("t_prep_ms", _D),
                ("t_autotune_ms", _D)]


class spmv_profile_report(ctypes.Structure):
    _fields_ = [("p", _D * 6), ("b_max_gbs", _D), ("b_hbm_gbs", _D), ("b_l2_gbs", _D),
                ("t_csr_ms", _D), ("t_ml_ms", _D), ("t_cmp_ms", _D), ("t_median_ms", _D),
                ("t_span_ms", _D), ("t_imb_ms", _D), ("n_ctas", _I32), ("vs", _I32),
                ("p2", _D * 2)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("p", "p2")}
        d["p"] = list(self.p)
        d["p2"] = list(self.p2)
        return d


class spmv_cg_report(ctypes.Structure):
    _fields_ = [("iters", _I32), ("converged", _I32), ("res_norm", _D), ("b_norm", _D),
                ("t_ms", _D)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

# name -> (restype, argtypes); status-returning entries raise on error
_DECL = {
    "spmv_tune_opts_default": (_I32, [ctypes.POINTER(spmv_tune_opts)]),
    "spmv_create": (_I32, [ctypes.POINTER(_P), _I64, _I64, _I64, _P, _P, _P, _I32, _I32, _P]),
    "spmv_destroy": (_I32, [_P]),
    "spmv_set_precision": (_I32, [_P, _I32, _I32, _I32, _P]),
    "spmv_tune": (_I32, [_P, _I32, ctypes.POINTER(spmv_tune_opts),
                         ctypes.POINTER(spmv_tune_report), _P]),
    "spmv_set_variant": (_I32, [_P, ctypes.POINTER(spmv_variant), _P]),
    "spmv_run": (_I32, [_P, _P, _P, _P]),
    "spmv_run_host": (_I32, [_P, _P, _P, _P]),
    "spmv_run_spmm": (_I32, [_P, _P, _P, _I32, _P]),
    "spmv_cg": (_I32, [_P, _P, _P, _I32, _D, _I32, _P, ctypes.POINTER(spmv_cg_report), _P]),
    "spmv_export_csr": (_I32, [_P, _P, _P, _P, _P]),
    "spmv_get_delta": (_I32, [_P, _P, _P, _P, ctypes.POINTER(_I64), ctypes.POINTER(_I32), _P]),
    "spmv_get_merge_path": (_I32, [_P, _P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P]),
    "spmv_get_row_bins": (_I32, [_P, _P, _P, _P, _P, _P, _P]),
    "spmv_get_col_panels": (_I32, [_P, _P, _P, _P, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                   _P]),
    "spmv_get_sell": (_I32, [_P, _P, _P, _P, ctypes.POINTER(_I64), ctypes.POINTER(_I32), _P]),
    "spmv_features": (_I32, [_P, _I32, _P, _P, _P]),
    "spmv_profile": (_I32, [_P, _I32, ctypes.POINTER(spmv_profile_report), _P]),
    "spmv_profile_cta_times": (_I32, [_P, _P, _P, ctypes.POINTER(_I32), _P]),
    "spmv_profile_kernel": (_I32, [_P, _I32, _P, _P, _P]),
    "spmv_probe_bandwidth": (_I32, [ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "spmv_probe_gather": (_I32, [_I64, _I32, _I64, _I32, ctypes.POINTER(_D), _P]),
    "spmv_probe_fma": (_I32, [_I32, _I32, _I32, _I32, ctypes.POINTER(_D), _P]),
    "spmv_classify": (_U32, [_P, _D, _D, _D]),
    "spmv_classify2": (_U32, [_P, _P, _D, _D, _D]),
    "spmv_variant_for_classes": (None, [_U32, _D, _D, _D, ctypes.POINTER(spmv_variant)]),
    "spmv_bounds": (None, [_I64, _I64, _I64, _I32, _I32, _I32, _D, _P]),
    "spmv_feature_rules": (_U32, [_P, _I64, _I32, _I64, _D]),
    "spmv_validate_csr": (_I32, [_I64, _I64, _I64, _P, _P, ctypes.POINTER(_I32), _P]),
    "spmv_round_values": (_I32, [_P, _P, _I64, _I32, _P]),
    "spmv_get_last_device_error": (_I32, [_P, ctypes.POINTER(_I32)]),
    "spmv_get_device_bytes": (_I32, [_P, ctypes.POINTER(_I64)]),
    "spmv_selftest_wait_timeout": (_I32, [_P, _I64, _P]),
    "spmv_status_string": (ctypes.c_char_p, [_I32]),
    "spmv_mlp_inputs": (_I32, [_P, _I64, _P, _P, _P, _P]),
    "spmv_mlp_logits": (_I32, [_P, _P, _I64, _P, _P, _P]),
    "spmv_mlp_loss_grad": (_I32, [_P, _P, _I64, _P, _P, _P, _P, _P]),
    "spmv_mlp_train": (_I32, [_P, _P, _P, _P, _I64, _P, _P, _I32, _I32, _F, _F, _F, _F, _P,
                              _P]),
    "spmv_selector_create": (_I32, [ctypes.POINTER(_P), _P, _P, _P, _P]),
    "spmv_selector_destroy": (_I32, [_P]),
    "spmv_selector_predict": (_I32, [_P, _P, ctypes.POINTER(_U32), ctypes.POINTER(_D), _P]),
    "spmv_selector_set_range": (_I32, [_P, _P, _P, ctypes.c_float]),
    "spmv_batch_create": (_I32, [ctypes.POINTER(_P), _P, _I32, _P, _P, _P, _P]),
    "spmv_run_batched": (_I32, [_P, _P]),
    "spmv_batch_set_plan": (_I32, [_P, _I32, _I32, _P]),
    "spmv_batch_tune": (_I32, [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32), _P]),
    "spmv_run_batched_sequential": (_I32, [_P, _P]),
    "spmv_batch_destroy": (_I32, [_P]),
    "spmv_run_noalloc": (_I32, [_I64, _I64, _I64, _P, _P, _P, _P, _P, _P]),
}

DECLARED = tuple(_DECL)


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load the CUDA library (building it first when it is missing and nvcc is here)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path} is missing")
        path = _build.build()
    L = ctypes.CDLL(path)
    for name, (res, args) in _DECL.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status: int, where: str) -> None:
    if status != 0:
        raise SpmvError(status, where)


def _call(name, *args):
    st = getattr(lib(), name)(*args)
    check(st, name)


# ------------------------------------------------------------------- entry points ----
def spmv_tune_opts_default() -> spmv_tune_opts:
    o = spmv_tune_opts()
    _call("spmv_tune_opts_default", ctypes.byref(o))
    return o


def spmv_create(n_rows, n_cols, nnz, row_ptr, col_ind, val, val_type, device_ptrs, stream=0):
    h = _P()
    _call("spmv_create", ctypes.byref(h), n_rows, n_cols, nnz, row_ptr, col_ind, val,
          val_type, device_ptrs, stream)
    return h.value


def spmv_destroy(h):
    _call("spmv_destroy", h)


def spmv_set_precision(h, storage, vec_type, acc_type, stream=0):
    _call("spmv_set_precision", h, storage, vec_type, acc_type, stream)


def spmv_tune(h, mode, opts=None, stream=0) -> spmv_tune_report:
    rep = spmv_tune_report()
    _call("spmv_tune", h, mode, ctypes.byref(opts) if opts is not None else None,
          ctypes.byref(rep), stream)
    return rep


def spmv_set_variant(h, variant: spmv_variant, stream=0):
    _call("spmv_set_variant", h, ctypes.byref(variant), stream)


def spmv_run(h, x, y, stream=0):
    _call("spmv_run", h, x, y, stream)


def spmv_run_host(h, x_host, y_host, stream=0):
    _call("spmv_run_host", h, x_host, y_host, stream)


def spmv_run_spmm(h, X, Y, k, stream=0):
    _call("spmv_run_spmm", h, X, Y, k, stream)


def spmv_cg(h, b, x, max_iters, rtol, check_every=1, res_hist=None, stream=0) -> dict:
    rep = spmv_cg_report()
    _call("spmv_cg", h, b, x, max_iters, rtol, check_every, res_hist, ctypes.byref(rep), stream)
    return rep.as_dict()


def spmv_export_csr(h, row_ptr, col_ind, val, stream=0):
    _call("spmv_export_csr", h, row_ptr, col_ind, val, stream)


def spmv_get_delta(h, base=None, delta=None, esc_col=None, stream=0) -> tuple[int, int]:
    """Returns (n_esc, bits); copies the index when the pointers are given."""
    n, bits = _I64(), _I32()
    _call("spmv_get_delta", h, base, delta, esc_col, ctypes.byref(n), ctypes.byref(bits), stream)
    return n.value, bits.value


def spmv_get_row_bins(h, med_rows=None, long_rows=None, long_first=None, chunks=None,
                      stream=0):
    """Returns (n_med, n_long, n_chunks); copies the lists when the pointers are given."""
    counts = (_I64 * 3)()
    _call("spmv_get_row_bins", h, med_rows, long_rows, long_first, chunks,
          ctypes.cast(counts, _P), stream)
    return int(counts[0]), int(counts[1]), int(counts[2])


def spmv_get_sell(h, slice_off=None, val=None, idx=None, stream=0):
    """Returns (n_positions, idx_bits); copies the sliced rows when the pointers are given."""
    n, b = _I64(), _I32()
    _call("spmv_get_sell", h, slice_off, val, idx, ctypes.byref(n), ctypes.byref(b), stream)
    return n.value, b.value


def spmv_get_col_panels(h, panel_rowptr=None, panel_col=None, panel_val=None, stream=0):
    """Returns (n_panels, panel_cols); copies the panel copy when the pointers are given."""
    n, w = _I32(), _I32()
    _call("spmv_get_col_panels", h, panel_rowptr, panel_col, panel_val, ctypes.byref(n),
          ctypes.byref(w), stream)
    return n.value, w.value


def spmv_get_merge_path(h, coord=None, stream=0):
    n, d = _I64(), _I64()
    _call("spmv_get_merge_path", h, coord, ctypes.byref(n), ctypes.byref(d), stream)
    return n.value, d.value


def spmv_features(h, line_bytes, features_host, isum_host=None, stream=0):
    _call("spmv_features", h, line_bytes, features_host, isum_host, stream)


def spmv_profile(h, reps, stream=0) -> spmv_profile_report:
    r = spmv_profile_report()
    _call("spmv_profile", h, reps, ctypes.byref(r), stream)
    return r


def spmv_profile_cta_times(h, elapsed_host=None, smid_host=None, n=0, stream=0) -> int:
    c = _I32(n)
    _call("spmv_profile_cta_times", h, elapsed_host, smid_host, ctypes.byref(c), stream)
    return c.value


def spmv_profile_kernel(h, which, x, y, stream=0):
    _call("spmv_profile_kernel", h, which, x, y, stream)


def spmv_probe_bandwidth():
    a, b = _D(), _D()
    _call("spmv_probe_bandwidth", ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def spmv_probe_gather(n_x, elem_bytes, count, reps=5, stream=0):
    """Milliseconds of `count` random gathers from an n_x-element array (the ceiling of an
    SpMV with uniform random columns)."""
    ms = _D()
    _call("spmv_probe_gather", n_x, elem_bytes, count, reps, ctypes.byref(ms), stream)
    return ms.value


def spmv_probe_fma(elem_bytes, chains, warps_per_sm, reps=5, stream=0):
    """Fused multiply-adds per second of a register-only kernel with `chains` independent
    chains per thread and warps_per_sm warps per SM (elem_bytes 8: FP64, 4: FP32)."""
    r = _D()
    _call("spmv_probe_fma", elem_bytes, chains, warps_per_sm, reps, ctypes.byref(r), stream)
    return r.value


def spmv_classify(p_host, t_imb=1.24, t_ml=1.25, t_mb=0.75) -> int:
    return int(lib().spmv_classify(p_host, t_imb, t_ml, t_mb))


def spmv_classify2(p_host, p2_host=None, t_imb=1.24, t_ml=1.25, t_mb=0.75) -> int:
    return int(lib().spmv_classify2(p_host, p2_host, t_imb, t_ml, t_mb))


def spmv_variant_for_classes(classes, nnz_avg, nnz_max, long_row_ratio=32.0) -> spmv_variant:
    v = spmv_variant()
    lib().spmv_variant_for_classes(classes, nnz_avg, nnz_max, long_row_ratio, ctypes.byref(v))
    return v


def spmv_bounds(n_rows, n_cols, nnz, idx_bytes, val_bytes, vec_bytes, b_max, out_host):
    lib().spmv_bounds(n_rows, n_cols, nnz, idx_bytes, val_bytes, vec_bytes, b_max, out_host)


def spmv_feature_rules(features_host, n_cols, vec_bytes, l2_bytes, long_row_ratio=32.0) -> int:
    return int(lib().spmv_feature_rules(features_host, n_cols, vec_bytes, l2_bytes,
                                        long_row_ratio))


def spmv_validate_csr(n_rows, n_cols, nnz, row_ptr, col_ind, stream=0) -> int:
    c = _I32()
    _call("spmv_validate_csr", n_rows, n_cols, nnz, row_ptr, col_ind, ctypes.byref(c), stream)
    return c.value


def spmv_round_values(inp, out, n, to, stream=0):
    _call("spmv_round_values", inp, out, n, to, stream)


def spmv_get_last_device_error(h) -> int:
    c = _I32()
    _call("spmv_get_last_device_error", h, ctypes.byref(c))
    return c.value


def spmv_selftest_wait_timeout(h, limit_ns, stream=0) -> int:
    """Returns the raw status: SPMV_ERR_TIMEOUT (6) when the bounded wait expired."""
    return int(lib().spmv_selftest_wait_timeout(h, limit_ns, stream))


def spmv_get_device_bytes(h) -> int:
    b = _I64()
    _call("spmv_get_device_bytes", h, ctypes.byref(b))
    return b.value


def spmv_status_string(s) -> str:
    return lib().spmv_status_string(s).decode()


def spmv_mlp_inputs(feat, batch, mu, inv_sigma, X, stream=0):
    _call("spmv_mlp_inputs", feat, batch, mu, inv_sigma, X, stream)


def spmv_mlp_logits(sizes_host, params, batch, X, logits, stream=0):
    _call("spmv_mlp_logits", sizes_host, params, batch, X, logits, stream)


def spmv_mlp_loss_grad(sizes_host, params, batch, X, Y, grad, loss, stream=0):
    _call("spmv_mlp_loss_grad", sizes_host, params, batch, X, Y, grad, loss, stream)


def spmv_mlp_train(sizes_host, params, m, v, batch, X, Y, steps, t0, lr, beta1, beta2, eps,
                   loss_hist, stream=0):
    _call("spmv_mlp_train", sizes_host, params, m, v, batch, X, Y, steps, t0, lr, beta1,
          beta2, eps, loss_hist, stream)


def spmv_selector_create(sizes_host, params_host, mu_host, inv_sigma_host):
    s = _P()
    _call("spmv_selector_create", ctypes.byref(s), sizes_host, params_host, mu_host,
          inv_sigma_host)
    return s.value


def spmv_selector_destroy(s):
    _call("spmv_selector_destroy", s)


def spmv_selector_set_range(s, lo_host, hi_host, slack):
    _call("spmv_selector_set_range", s, lo_host, hi_host, float(slack))


def spmv_selector_predict(s, feat16_host, stream=0):
    c, m = _U32(), _D()
    _call("spmv_selector_predict", s, feat16_host, ctypes.byref(c), ctypes.byref(m), stream)
    return c.value, m.value


def spmv_batch_create(handles, X, Y, k, stream=0):
    n = len(handles)
    H = (_P * n)(*handles)
    XX = (_P * n)(*X)
    YY = (_P * n)(*Y)
    KK = (_I32 * n)(*k)
    b = _P()
    _call("spmv_batch_create", ctypes.byref(b), H, n, XX, YY, KK, stream)
    return b.value


def spmv_batch_set_plan(b, item_nnz, chunk_nnz, stream=0):
    _call("spmv_batch_set_plan", b, int(item_nnz), int(chunk_nnz), stream)


def spmv_batch_tune(b, reps=5, stream=0):
    """Returns the (item_nnz, chunk_nnz) plan the autotuner kept."""
    i, c = _I32(), _I32()
    _call("spmv_batch_tune", b, int(reps), ctypes.byref(i), ctypes.byref(c), stream)
    return i.value, c.value


def spmv_run_batched(b, stream=0):
    _call("spmv_run_batched", b, stream)


def spmv_run_batched_sequential(b, stream=0):
    _call("spmv_run_batched_sequential", b, stream)


def spmv_batch_destroy(b):
    _call("spmv_batch_destroy", b)


def spmv_run_noalloc(n_rows, n_cols, nnz, row_ptr, col_ind, val, x, y, stream=0):
    """y = A x (FP64) without any device allocation; see the header for the scratch limit."""
    _call("spmv_run_noalloc", n_rows, n_cols, nnz, row_ptr, col_ind, val, x, y, stream)
