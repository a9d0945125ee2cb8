"""The largest matrix a handle accepts (nnz just under 2^31 - 2^21 - 1, row offsets near the
top of int32), built on the device from synth's closed form: every variant whose index
arithmetic reaches those offsets (the plain CSR-vector, the thread-per-row tile with int32
columns and with 16-bit deltas and escape rows, merge-path tiles, the row decomposition
with and without deltas) gives rows within the FP64 bound of the oracle, on a sample that
includes the last rows (the long ones, chunked) and the rows around the band of shorter
rows and the escape rows."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TAU, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def api(torch):
    from paper_1711_05487_gb300 import api as _api
    return _api

VARIANTS = [dict(), dict(vec=1, vs=1), dict(index=1, vec=1, vs=1), dict(partition=1),
            dict(partition=2), dict(partition=2, index=1)]


def _sample_rows():
    n = synth.MAX_NNZ_ROWS
    lens = synth.max_nnz_lengths()
    rng = np.random.default_rng(synth.SEED_BASE + 90)
    band = np.flatnonzero(lens == 32)
    picks = [rng.integers(0, n, 3000), np.arange(8), np.arange(n - 40, n),
             np.flatnonzero(lens == 16), band[:4], band[-4:], band[-1] + np.arange(1, 5)]
    return np.unique(np.concatenate(picks))


def test_max_nnz_every_offset_path(api, torch):
    free, _ = torch.cuda.mem_get_info()
    if free < 100e9:
        pytest.skip(f"needs about 100 GB of free device memory, {free / 1e9:.0f} GB free")
    rp, ci, v = synth.max_nnz_device(torch)
    nnz = ci.numel()
    assert synth.MAX_NNZ - 1024 < nnz <= synth.MAX_NNZ
    A = api.SpmvMatrix(synth.MAX_NNZ_ROWS, synth.MAX_NNZ_COLS, rp, ci, v)
    del rp, ci, v
    torch.cuda.empty_cache()
    x64 = synth.max_nnz_x()
    x = torch.from_numpy(x64).cuda()
    rows = _sample_rows()
    sub = synth.max_nnz_rows(rows)
    want, s = oracle.spmv(sub.rowptr, sub.colind, sub.val, x64)
    rows_t = torch.from_numpy(rows).cuda()
    for var in VARIANTS:
        A.set_variant(**var)
        y = A.run(x)
        got = y[rows_t].cpu().numpy()
        err = np.abs(got - want)
        bad = err > TAU["f64"] * s
        assert not bad.any(), (var, rows[bad][:5], err[bad][:5], s[bad][:5])
        del y
