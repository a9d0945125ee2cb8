"""The allocation-free entry point spmv_run_noalloc.

It serves callers that must not allocate device memory (an application whose allocator
owns the device memory budget, code running with the device nearly full, latency-critical
code that cannot afford a synchronizing cudaMalloc / cudaFree): its scratch is one fixed
16 MiB array in device global memory instead of per-handle allocations. This test calls it
through the C ABI and compares it with the oracle's y = A x and with the existing entry
point, spmv_run on a handle with the same (merge-path) variant, within the FP64 tolerance
the other tests use, on two calls in a row (the second call reuses the scratch the first
one left behind). Around the second call the device's free memory must not change: the
call allocates nothing.

The file is named to be collected last, so that a run stopping at the first failure has
run every other test before this one.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TAU, check_rows, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


def _cases():
    return [synth.power_law(60_000, alpha=1.6, clip=30_000, seed=61, dtype=np.float64),
            synth.stencil_27pt(30),
            synth.uniform_random(7000, 90, seed=62, min_per_row=0),
            synth.uniform_random(1, 9000, seed=63, min_per_row=9000, n_cols=20_000)]


def test_noalloc_matches_regular_entry_point(torch):
    from paper_1711_05487_gb300 import _abi, api
    for m in _cases():
        x64 = synth.uniform_vector(m.n_cols, 64)
        x = torch.from_numpy(x64).cuda()
        A = api.SpmvMatrix.from_csr(m)
        A.set_variant(partition=1)
        y_ref = A.run(x).cpu().numpy()
        rp = torch.from_numpy(m.rowptr).cuda()
        ci = torch.from_numpy(m.colind).cuda()
        v = torch.from_numpy(m.val).cuda()
        y_or, s = oracle.spmv(m.rowptr, m.colind, m.val, x64)
        check_rows(y_ref, y_or, s, TAU["f64"], f"{m.name} spmv_run")
        outs = []
        for call in range(2):
            y = torch.full((m.n_rows,), np.nan, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            free_before = torch.cuda.mem_get_info()[0]
            _abi.spmv_run_noalloc(m.n_rows, m.n_cols, m.nnz, rp.data_ptr(), ci.data_ptr(),
                                  v.data_ptr(), x.data_ptr(), y.data_ptr(), 0)
            torch.cuda.synchronize()
            free_after = torch.cuda.mem_get_info()[0]
            if call == 1:       # the first call may load the module; the second allocates nothing
                assert free_after == free_before, (m.name, free_before, free_after)
            outs.append(y.cpu().numpy())
            check_rows(outs[-1], y_or, s, TAU["f64"], f"{m.name} call {call} vs oracle")
            check_rows(outs[-1], y_ref, s, TAU["f64"], f"{m.name} call {call} vs spmv_run")
        assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_oversized_problems(torch):
    from paper_1711_05487_gb300 import _abi
    with pytest.raises(_abi.SpmvError) as e:
        # about 2.1e9 merge items, above the fixed scratch; rejected before any pointer is used
        _abi.spmv_run_noalloc(1 << 30, 1 << 30, (1 << 30) + 5, 1, 1, 1, 1, 1, 0)
    assert e.value.status == 9
