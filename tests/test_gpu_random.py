"""GPU parity on randomly structured matrices (several tiles, ragged tails, empty rows, gaps
exactly at the 8- and 16-bit limits and past them): the delta index bit for bit against the
oracle, and every variant that reads it, or that re-partitions the rows or the columns,
within the FP64 bound of the oracle's y = A x."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TAU, check_spmv, torch_cuda

pytestmark = pytest.mark.gpu

CASES = [(3001, 4_000, 40, 30.0, 1), (9000, 70_000, 24, 3000.0, 2),
         (20_011, 400_000, 40, 300.0, 3), (4096, 1_000_000, 12, 100_000.0, 4),
         (12_345, 300, 40, 1.0, 5), (777, 200_000, 40, 3000.0, 6)]

VARIANTS = [dict(index=1, vec=1), dict(index=1, vec=1, vs=1, tile_rows=32),
            dict(index=1, vec=1, vs=1, tile_rows=128, tile_pipe=1),
            dict(partition=3, index=1), dict(partition=2, index=1, vs=4),
            dict(partition=1), dict(xpath=2, vs=2), dict(xpath=3, vs=1)]


@pytest.fixture(scope="module")
def api():
    torch_cuda()
    from paper_1711_05487_gb300 import api as _api
    return _api


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}_s{c[4]}")
def test_random_structure(api, case):
    import torch
    n_rows, n_cols, max_len, gap_scale, seed = case
    m = synth.random_gaps(n_rows, n_cols, max_len, gap_scale, synth.SEED_BASE + 300 + seed)
    A = api.SpmvMatrix.from_csr(m)
    A.set_variant(index=1, vec=1)
    base, delta, esc, bits = A.delta()
    assert bits == oracle.delta_width(m.rowptr, m.colind)
    enc = oracle.delta8_encode if bits == 8 else oracle.delta16_encode
    ob, od, oe = enc(m.rowptr, m.colind)
    assert np.array_equal(base.cpu().numpy(), ob)
    assert np.array_equal(delta.cpu().numpy().view(np.uint8 if bits == 8 else np.uint16), od)
    assert np.array_equal(esc.cpu().numpy(), oe)
    x64 = synth.uniform_vector(n_cols, synth.SEED_BASE + 400 + seed)
    x = torch.from_numpy(x64).cuda()
    for v in VARIANTS:
        A.set_variant(**v)
        y = A.run(x)
        torch.cuda.synchronize()
        check_spmv(m, x64, y.cpu().numpy(), TAU["f64"], f"{m.name} {v}")
