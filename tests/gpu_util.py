"""Helpers for the GPU parity tests (imported by tests/test_gpu_*.py only)."""
import numpy as np
import pytest

import oracle

# Tolerances on |y_gpu - y_oracle| <= tau * sum_j |a_ij x_j| per row, by value storage
TAU = {"f64": 1e-12, "df64": 1e-12, "f32": 2e-6, "bf16": 8e-3}


def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def stored_values(val64: np.ndarray, storage: str) -> np.ndarray:
    """The values the GPU multiplies with, widened exactly to FP64 (oracle rounding)."""
    if storage in ("f64", "df64"):
        return val64.astype(np.float64)
    if storage == "f32":
        return oracle.round_f32(val64).astype(np.float64)
    return oracle.bf16_bits_to_f64(oracle.round_bf16_bits(val64))


def check_rows(y_gpu, y_ref, s_ref, tau, what=""):
    y_gpu = np.asarray(y_gpu, dtype=np.float64)
    err = np.abs(y_gpu - y_ref)
    zero = s_ref == 0
    assert np.all(y_gpu[zero] == 0.0), f"{what}: rows with s = 0 must be exactly 0"
    nz = ~zero
    ratio = err[nz] / s_ref[nz] if nz.any() else np.zeros(1)
    worst = float(ratio.max()) if ratio.size else 0.0
    assert worst <= tau, f"{what}: max |err|/s = {worst:.3e} > {tau:.1e}"
    return worst


def check_spmv(m, x64, y_gpu, tau, what="", values=None):
    """Full comparison against the oracle's FP64 y = A x with the original values (the
    error bound includes the rounding of the stored values)."""
    val = m.val if values is None else values
    y, s = oracle.spmv(m.rowptr, m.colind, val, x64)
    return check_rows(y_gpu, y, s, tau, what)
