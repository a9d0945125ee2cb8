"""Python convenience layer over the C ABI: torch tensors for device memory and streams.

The classes below only marshal arguments (data_ptr(), dtypes, streams) into the C entry
points of _abi; every step of the SpMV path runs in the CUDA library.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np
import torch

from . import _abi
from ._abi import (SPMV_BF16, SPMV_DF64, SPMV_F32, SPMV_F64, TUNE_FEATURES, TUNE_FIXED, TUNE_LEARNED,
                   TUNE_PROFILE, spmv_variant)

DTYPE_CODE = {torch.float64: SPMV_F64, torch.float32: SPMV_F32, torch.bfloat16: SPMV_BF16,
              "f64": SPMV_F64, "f32": SPMV_F32, "bf16": SPMV_BF16, "df64": SPMV_DF64}
# DF64 handles keep and export their FP64 values; x and y are FP64
TORCH_DTYPE = {SPMV_F64: torch.float64, SPMV_F32: torch.float32, SPMV_BF16: torch.bfloat16,
               SPMV_DF64: torch.float64}
MODES = {"profile": TUNE_PROFILE, "features": TUNE_FEATURES, "learned": TUNE_LEARNED,
         "fixed": TUNE_FIXED}
CLASS_NAMES = ((1, "MB"), (2, "ML"), (4, "IMB"), (8, "CMP"))
P_NAMES = ("P_CSR", "P_MB", "P_ML", "P_IMB", "P_CMP", "P_peak")
FEATURE_NAMES = ("size", "density", "nnz_min", "nnz_max", "nnz_avg", "nnz_sd", "bw_min",
                 "bw_max", "bw_avg", "bw_sd", "scatter_avg", "scatter_sd",
                 "clustering_avg", "misses_avg")


def class_names(mask: int) -> list[str]:
    """Names of the bottleneck classes (Fig. 3: MB, ML, IMB, CMP) set in a class mask."""
    return [n for b, n in CLASS_NAMES if mask & b]


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def variant(partition=0, index=0, xpath=0, vec=0, vs=0, tile_rows=0, tile_pipe=0,
            bin_med=0, bin_chunk=0) -> spmv_variant:
    """A pool variant (Table II knobs): partition 0 rows, 1 merge-path tiles, 2 row
    decomposition, 3 sliced rows; index 1 delta columns; xpath 1 x evict-last in the L2,
    P >= 2 P column panels; vec vector loads; vs sub-warp width (1: thread per row);
    tile_rows / tile_pipe the width-1 tile geometry (0: chosen by the library); bin_med /
    bin_chunk the row decomposition's limits (0: 64 and 4096)."""
    return spmv_variant(partition, index, xpath, vec, vs, tile_rows, tile_pipe, bin_med,
                        bin_chunk)


CSR_VECTOR = dict(partition=0, index=0, xpath=0, vec=0, vs=0, tile_rows=0, tile_pipe=0,
                  bin_med=0, bin_chunk=0)


def _as_torch(a, dtype=None) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a if dtype is None else a.to(dtype)
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t if dtype is None else t.to(dtype)


@dataclasses.dataclass
class TuneResult:
    classes: int
    mode_used: int
    variant: tuple
    p: dict
    p2: list
    b_max_gbs: float
    features: dict
    margin: float
    t_pre_ms: float
    t_classify_ms: float
    t_prep_ms: float
    t_autotune_ms: float

    @property
    def class_names(self):
        """Names of the classes the route found."""
        return class_names(self.classes)

    @staticmethod
    def from_report(r: _abi.spmv_tune_report) -> "TuneResult":
        """Converts the C tune report."""
        return TuneResult(int(r.classes), int(r.mode_used), r.variant.as_tuple(),
                          dict(zip(P_NAMES, list(r.p))), list(r.p2), float(r.b_max_gbs),
                          dict(zip(FEATURE_NAMES, list(r.features))), float(r.margin),
                          float(r.t_pre_ms), float(r.t_classify_ms), float(r.t_prep_ms),
                          float(r.t_autotune_ms))


class SpmvMatrix:
    """A CSR matrix owned by the library on the current CUDA device."""

    def __init__(self, n_rows, n_cols, rowptr, colind, val, stream=None):
        rp = _as_torch(rowptr, torch.int32).contiguous()
        ci = _as_torch(colind, torch.int32).contiguous()
        v = _as_torch(val).contiguous()
        if v.dtype not in DTYPE_CODE:
            raise TypeError(f"unsupported value dtype {v.dtype}")
        dev = rp.is_cuda
        if dev != ci.is_cuda or dev != v.is_cuda:
            raise ValueError("rowptr, colind and val must all be host or all be device tensors")
        self.n_rows, self.n_cols, self.nnz = int(n_rows), int(n_cols), int(ci.numel())
        self._h = None
        self._h = _abi.spmv_create(self.n_rows, self.n_cols, self.nnz, rp.data_ptr(),
                                   ci.data_ptr() if self.nnz else None,
                                   v.data_ptr() if self.nnz else None, DTYPE_CODE[v.dtype],
                                   1 if dev else 0, _stream(stream))
        self.in_type = DTYPE_CODE[v.dtype]
        self.storage = self.in_type
        self.vec = SPMV_F64 if self.in_type == SPMV_F64 else SPMV_F32
        self.acc = self.vec
        self.report: TuneResult | None = None

    @classmethod
    def from_csr(cls, m, stream=None) -> "SpmvMatrix":
        """Copies a CSR matrix (n_rows, n_cols, rowptr, colind, val) into the library."""
        return cls(m.n_rows, m.n_cols, m.rowptr, m.colind, m.val, stream)

    @property
    def handle(self) -> int:
        """The C handle, for calls through the ctypes binding."""
        return self._h

    def close(self):
        """Destroys the C handle and frees its device memory."""
        if self._h:
            _abi.spmv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ----------------------------------------------------------------- configuration
    def set_precision(self, storage="f64", vec="f64", acc="f64", stream=None):
        """Value storage ('f64', 'f32', 'bf16', 'df64'), x / y dtype and accumulation;
        the handle must be tuned again afterwards."""
        s, v, a = DTYPE_CODE[storage], DTYPE_CODE[vec], DTYPE_CODE[acc]
        try:
            _abi.spmv_set_precision(self._h, s, v, a, _stream(stream))
        except _abi.SpmvError as e:
            if e.status not in (_abi.SPMV_ERR_ARG, _abi.SPMV_ERR_UNSUPPORTED_DTYPE):
                # a failure while converting leaves the handle at the input dtype's defaults
                self.storage = self.in_type
                self.vec = SPMV_F64 if self.in_type == SPMV_F64 else SPMV_F32
                self.acc = self.vec
            raise
        self.storage, self.vec, self.acc = s, v, a

    @property
    def vec_dtype(self) -> torch.dtype:
        """torch dtype of x and y."""
        return TORCH_DTYPE[self.vec]

    def tune(self, mode="profile", stream=None, selector=None, fixed=None, **kw) -> TuneResult:
        """Section III: classify with `mode` ('profile', 'features', 'learned' with a
        `selector`, or 'fixed' with a `fixed` variant), then build and autotune the variant;
        other keywords set fields of the tune options. Synchronizes."""
        opts = _abi.spmv_tune_opts_default()
        for k, val in kw.items():
            setattr(opts, k, val)
        if selector is not None:
            opts.selector = selector.handle if hasattr(selector, "handle") else selector
        if fixed is not None:
            opts.fixed = fixed if isinstance(fixed, spmv_variant) else variant(**fixed)
        rep = _abi.spmv_tune(self._h, MODES[mode] if isinstance(mode, str) else mode, opts,
                             _stream(stream))
        self.report = TuneResult.from_report(rep)
        return self.report

    def set_variant(self, stream=None, **knobs):
        """Installs a variant by hand (the knobs of `variant`; none: plain CSR-vector)."""
        v = variant(**{**CSR_VECTOR, **knobs})
        _abi.spmv_set_variant(self._h, v, _stream(stream))

    # ----------------------------------------------------------------------- running
    def run(self, x: torch.Tensor, y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """y = A x (Fig. 1) on device tensors, asynchronous on `stream`; allocates y when
        it is not given."""
        if y is None:
            y = torch.empty(self.n_rows, dtype=self.vec_dtype, device=x.device)
        _abi.spmv_run(self._h, x.data_ptr(), y.data_ptr(), _stream(stream))
        return y

    def run_host(self, x: torch.Tensor, y: torch.Tensor, stream=None) -> torch.Tensor:
        """y = A x with host tensors (page-locked ones replay a captured pipeline of
        uploads, chunk kernels and downloads); returns when y is on the host."""
        _abi.spmv_run_host(self._h, x.data_ptr(), y.data_ptr(), _stream(stream))
        return y

    def spmm(self, X: torch.Tensor, Y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Y = A X for row-major X of shape (n_cols, k)."""
        k = X.shape[1]
        if Y is None:
            Y = torch.empty((self.n_rows, k), dtype=self.vec_dtype, device=X.device)
        _abi.spmv_run_spmm(self._h, X.data_ptr(), Y.data_ptr(), k, _stream(stream))
        return Y

    # ---------------------------------------------------------------- inspection
    def features(self, line_bytes=128, stream=None):
        """Table I features computed on the GPU (14, FEATURE_NAMES order) and their 12 exact
        integer sums."""
        f = np.zeros(14)
        isum = np.zeros(12, dtype=np.uint64)
        _abi.spmv_features(self._h, line_bytes, f.ctypes.data, isum.ctypes.data, _stream(stream))
        return f, isum

    def profile(self, reps=20, stream=None) -> dict:
        """Section III-B profile: P-vector, bandwidths and the timings behind them."""
        r = _abi.spmv_profile(self._h, reps, _stream(stream)).as_dict()
        r["p"] = dict(zip(P_NAMES, r["p"]))
        return r

    def profile_cta_times(self, stream=None):
        """Per-CTA elapsed ms and SM id of one static-partition baseline launch."""
        n = _abi.spmv_profile_cta_times(self._h, None, None, 0, _stream(stream))
        el = np.zeros(n)
        sm = np.zeros(n, dtype=np.int32)
        _abi.spmv_profile_cta_times(self._h, el.ctypes.data, sm.ctypes.data, n, _stream(stream))
        return el, sm

    def profile_kernel(self, which: int, x: torch.Tensor, y: torch.Tensor, stream=None):
        """Runs one profiling kernel once into y: 0 the static-partition baseline, 1 the
        P_ML kernel, 2 the P_CMP kernel."""
        _abi.spmv_profile_kernel(self._h, which, x.data_ptr(), y.data_ptr(), _stream(stream))
        return y

    def cg(self, b: torch.Tensor, x0: torch.Tensor | None = None, max_iters: int = 1000,
           rtol: float = 1e-10, check_every: int = 10, history: bool = False, stream=None):
        """Conjugate gradients on the tuned handle (SPD matrix, FP64 vectors). Returns
        (x, report dict[, ||r_k|| history as a device tensor])."""
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        hist = torch.zeros(max_iters + 1, dtype=torch.float64, device=b.device) if history else None
        rep = _abi.spmv_cg(self._h, b.data_ptr(), x.data_ptr(), max_iters, rtol, check_every,
                           None if hist is None else hist.data_ptr(), _stream(stream))
        if history:
            return x, rep, hist[:rep["iters"] + 1]
        return x, rep

    def export_csr(self, device="cuda", stream=None):
        """The matrix as CSR with its stored values (columns decoded from the delta index
        when the installed variant uses one)."""
        rp = torch.empty(self.n_rows + 1, dtype=torch.int32, device=device)
        ci = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=device)
        v = torch.empty(max(self.nnz, 1), dtype=TORCH_DTYPE[self.storage], device=device)
        _abi.spmv_export_csr(self._h, rp.data_ptr(), ci.data_ptr(), v.data_ptr(), _stream(stream))
        return rp, ci[:self.nnz], v[:self.nnz]

    def delta(self, device="cuda", stream=None):
        """The delta column index: (base, delta as uint8/int16 bits, escape columns, width)."""
        n_esc, bits = _abi.spmv_get_delta(self._h)
        base = torch.empty(max(self.n_rows, 1), dtype=torch.int32, device=device)
        delta = torch.empty(max(self.nnz, 1), dtype=torch.uint8 if bits == 8 else torch.int16,
                            device=device)
        esc = torch.empty(max(n_esc, 1), dtype=torch.int32, device=device)
        _abi.spmv_get_delta(self._h, base.data_ptr(), delta.data_ptr(), esc.data_ptr(),
                            _stream(stream))
        return base[:self.n_rows], delta[:self.nnz], esc[:n_esc], bits

    def row_bins(self, device="cuda", stream=None):
        """The row decomposition (partition 2): medium rows, long rows, each long row's first
        chunk, and the chunk table (row, first nonzero, end nonzero, the column a delta
        decode of the chunk starts from)."""
        n_med, n_long, n_ch = _abi.spmv_get_row_bins(self._h)
        med = torch.empty(max(n_med, 1), dtype=torch.int32, device=device)
        lng = torch.empty(max(n_long, 1), dtype=torch.int32, device=device)
        first = torch.empty(n_long + 1, dtype=torch.int32, device=device)
        ch = torch.empty((max(n_ch, 1), 4), dtype=torch.int32, device=device)
        _abi.spmv_get_row_bins(self._h, med.data_ptr(), lng.data_ptr(), first.data_ptr(),
                               ch.data_ptr(), _stream(stream))
        return med[:n_med], lng[:n_long], first, ch[:n_ch]

    def sell(self, device="cuda", stream=None):
        """The sliced-row copy (partition 3): (slice offsets, values, columns or deltas,
        delta bits or 0)."""
        n, bits = _abi.spmv_get_sell(self._h)
        ns = (self.n_rows + 31) // 32
        off = torch.empty(ns + 1, dtype=torch.int64, device=device)
        v = torch.empty(max(n, 1), dtype=TORCH_DTYPE[self.storage], device=device)
        it = {0: torch.int32, 16: torch.int16, 8: torch.uint8}[bits]
        ix = torch.empty(max(n, 1), dtype=it, device=device)
        _abi.spmv_get_sell(self._h, off.data_ptr(), v.data_ptr(), ix.data_ptr(), _stream(stream))
        return off, v[:n], ix[:n], bits

    def col_panels(self, device="cuda", stream=None):
        """The column-panel copy (variant xpath = P >= 2): (row pointers (P, n_rows + 1),
        columns, values, panel width)."""
        n_p, w = _abi.spmv_get_col_panels(self._h)
        rp = torch.empty((n_p, self.n_rows + 1), dtype=torch.int32, device=device)
        ci = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=device)
        v = torch.empty(max(self.nnz, 1), dtype=TORCH_DTYPE[self.storage], device=device)
        _abi.spmv_get_col_panels(self._h, rp.data_ptr(), ci.data_ptr(), v.data_ptr(),
                                 _stream(stream))
        return rp, ci[:self.nnz], v[:self.nnz], w

    def merge_path(self, device="cuda", stream=None):
        """The merge-path table (rows ended, nonzeros consumed) at every tile boundary, and
        the merge items per tile."""
        n_tiles, items = _abi.spmv_get_merge_path(self._h)
        c = torch.empty((n_tiles + 1, 2), dtype=torch.int32, device=device)
        _abi.spmv_get_merge_path(self._h, c.data_ptr(), _stream(stream))
        return c, items

    def device_bytes(self) -> int:
        """Device memory held by the handle, in bytes."""
        return _abi.spmv_get_device_bytes(self._h)


class Selector:
    """A learned selector (MLP weights + input standardization) on the current device, with
    the training range of its standardized inputs when known: a matrix whose inputs leave
    that range by more than `slack` gets margin -1, and the learned route profiles it."""

    def __init__(self, sizes, params, mu=None, inv_sigma=None, in_lo=None, in_hi=None,
                 slack=0.5):
        self.sizes = np.ascontiguousarray(sizes, dtype=np.int32)
        self.params = np.ascontiguousarray(params, dtype=np.float32)
        self.mu = None if mu is None else np.ascontiguousarray(mu, dtype=np.float32)
        self.inv_sigma = None if inv_sigma is None else np.ascontiguousarray(inv_sigma,
                                                                             dtype=np.float32)
        self.in_lo = None if in_lo is None else np.ascontiguousarray(in_lo, dtype=np.float32)
        self.in_hi = None if in_hi is None else np.ascontiguousarray(in_hi, dtype=np.float32)
        self.slack = float(slack)
        self.handle = _abi.spmv_selector_create(
            self.sizes.ctypes.data, self.params.ctypes.data,
            None if self.mu is None else self.mu.ctypes.data,
            None if self.inv_sigma is None else self.inv_sigma.ctypes.data)
        if self.in_lo is not None and self.in_hi is not None:
            _abi.spmv_selector_set_range(self.handle, self.in_lo.ctypes.data,
                                         self.in_hi.ctypes.data, self.slack)

    def predict(self, feat16, stream=None):
        """(class mask, margin) for 16 feature values; margin -1 outside the training range."""
        f = np.ascontiguousarray(feat16, dtype=np.float64)
        return _abi.spmv_selector_predict(self.handle, f.ctypes.data, _stream(stream))

    def close(self):
        """Frees the selector's device buffers."""
        if self.handle:
            _abi.spmv_selector_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def save(self, path: str):
        """Writes the weights, standardization and training range to an .npz file."""
        empty = np.zeros(0, np.float32)
        np.savez(path, sizes=self.sizes, params=self.params,
                 mu=self.mu if self.mu is not None else empty,
                 inv_sigma=self.inv_sigma if self.inv_sigma is not None else empty,
                 in_lo=self.in_lo if self.in_lo is not None else empty,
                 in_hi=self.in_hi if self.in_hi is not None else empty,
                 slack=np.array([self.slack], np.float32), version=np.array([2]))

    @classmethod
    def load(cls, path: str) -> "Selector":
        """Reads a selector written by `save`."""
        z = np.load(path)
        opt = {k: (z[k] if k in z.files and z[k].size else None)
               for k in ("mu", "inv_sigma", "in_lo", "in_hi")}
        slack = float(z["slack"][0]) if "slack" in z.files else 0.5
        return cls(z["sizes"], z["params"], opt["mu"], opt["inv_sigma"], opt["in_lo"],
                   opt["in_hi"], slack)


class Batch:
    """Many FP32 matrices with k in {1, 4, 16} right-hand sides, one persistent launch."""

    def __init__(self, mats, Xs, Ys, ks, stream=None):
        self.mats = list(mats)
        self.Xs, self.Ys = list(Xs), list(Ys)
        self.handle = _abi.spmv_batch_create([m.handle for m in self.mats],
                                             [x.data_ptr() for x in self.Xs],
                                             [y.data_ptr() for y in self.Ys], list(ks),
                                             _stream(stream))

    def run(self, stream=None):
        """All products of the batch: one persistent launch replayed from a CUDA graph."""
        _abi.spmv_run_batched(self.handle, _stream(stream))

    def set_plan(self, item_nnz, chunk_nnz, stream=None):
        """Sets the work plan: nonzeros per warp item and the chunk length of split rows."""
        _abi.spmv_batch_set_plan(self.handle, item_nnz, chunk_nnz, _stream(stream))

    def tune(self, reps=5, stream=None):
        """Times the candidate work plans and keeps the fastest: (item_nnz, chunk_nnz)."""
        return _abi.spmv_batch_tune(self.handle, reps, _stream(stream))

    def run_sequential(self, stream=None):
        """The same products launched matrix by matrix, for comparison."""
        _abi.spmv_run_batched_sequential(self.handle, _stream(stream))

    def close(self):
        """Frees the batch (its plan, graph and buffers; not the handles)."""
        if self.handle:
            _abi.spmv_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
