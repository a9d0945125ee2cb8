"""GB300-native bottleneck-adaptive CSR SpMV (arXiv 1711.05487).

The compute path is the CUDA library built from csrc/ (libspmv_gb300.so, sm_103a); this
package only loads it and marshals arguments. See include/spmv_gb300.h for the C ABI.
"""
from . import _abi  # noqa: F401
from ._abi import (CLASS_CMP, CLASS_IMB, CLASS_MB, CLASS_ML, SPMV_BF16, SPMV_F32, SPMV_F64,
                   SpmvError, spmv_variant)
from .buildlib import build

__all__ = ["build", "SpmvError", "spmv_variant", "SPMV_F64", "SPMV_F32", "SPMV_BF16",
           "CLASS_MB", "CLASS_ML", "CLASS_IMB", "CLASS_CMP", "SpmvMatrix", "Selector", "Batch",
           "variant", "class_names"]


def __getattr__(name):
    # the torch-based layer is imported lazily so that the ABI can be inspected without torch
    if name in ("SpmvMatrix", "Selector", "Batch", "variant", "class_names", "TuneResult",
                "CSR_VECTOR"):
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
