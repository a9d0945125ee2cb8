"""CPU-side checks of the C ABI: the library builds, loads, exports every entry point that
include/spmv_gb300.h declares, and its pure host functions (classifier, class map,
bounds, feature rules) agree with the oracle. No CUDA computation runs here."""
import itertools
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(spmv_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def abi():
    from paper_1711_05487_gb300 import _abi
    _abi.lib()
    return _abi


def test_library_exports_every_declared_symbol(abi):
    declared = _declared_functions()
    assert len(declared) >= 30
    out = subprocess.run(["nm", "-D", "--defined-only", abi.library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared - exported
    assert not missing, missing
    # the Python binding names every declared function too
    assert declared == set(abi.DECLARED)


def test_binding_has_one_function_per_declared_call():
    """The Python binding is argument marshalling with the header's names: one function per
    declared entry point, and nothing else named like one."""
    src = open(os.path.join(ROOT, "paper_1711_05487_gb300", "_abi.py")).read()
    bound = set(re.findall(r"^def (spmv_[a-z0-9_]+)\(", src, flags=re.M))
    assert bound == _declared_functions()


def test_status_strings(abi):
    for s in range(10):
        assert abi.spmv_status_string(s)
    assert "invalid argument" in abi.spmv_status_string(7)


def test_create_rejects_nnz_past_the_int32_headroom(abi):
    """spmv_create takes at most SPMV_MAX_NNZ = 2^31 - 2^21 - 1 nonzeros (int32 offsets with
    room for the kernels' widest stride through a row, a 2^20-nonzero chunk) and refuses one
    more with SPMV_ERR_ARG before it reads any array or touches the GPU."""
    import ctypes
    hdr = open(os.path.join(ROOT, "include", "spmv_gb300.h")).read()
    lim = int(re.search(r"#define SPMV_MAX_NNZ (\d+)LL", hdr).group(1))
    assert lim == 2 ** 31 - 2 ** 21 - 1
    dummy = ctypes.c_int64(0)
    p = ctypes.addressof(dummy)
    for n_rows, n_cols, nnz in ((10, 10, lim + 1), (10, 10, 2 ** 31 - 1), (2 ** 31 - 1, 10, 0),
                                (10, 2 ** 31 - 1, 0), (-1, 10, 0)):
        with pytest.raises(abi.SpmvError) as e:
            abi.spmv_create(n_rows, n_cols, nnz, p, p, p, abi.SPMV_F64, 0)
        assert e.value.status == 7


def _p_vector(bits):
    imb, ml, mb, cmp_ = bits
    p_imb = 200.0 if imb else 110.0
    p_ml = 200.0 if ml else 110.0
    if mb:
        rest = (110.0, 150.0, 300.0)
    elif cmp_:
        rest = (150.0, 110.0, 300.0)
    else:
        rest = (400.0, 450.0, 500.0)
    return [100.0, rest[0], p_ml, p_imb, rest[1], rest[2]]


def test_classify_matches_oracle(abi):
    rng = np.random.default_rng(0)
    vectors = [_p_vector(b) for b in itertools.product([0, 1], repeat=4)]
    vectors += list(rng.uniform(10, 1000, size=(2000, 6)))
    vectors += [[100, 500, 125, 124, 550, 600], [100, 133.3, 100, 100, 150, 600]]
    for v in vectors:
        p = np.ascontiguousarray(v, dtype=np.float64)
        for t in [(1.24, 1.25, 0.75), (1.1, 1.5, 0.9)]:
            assert abi.spmv_classify(p.ctypes.data, *t) == oracle.classify(*p, *t)


def test_classify2_matches_oracle(abi):
    rng = np.random.default_rng(2)
    for _ in range(3000):
        p = np.ascontiguousarray(rng.uniform(10, 1000, 6))
        p2 = np.ascontiguousarray(rng.uniform(10, 1500, 2))
        for q in (p2, None):
            got = abi.spmv_classify2(p.ctypes.data, None if q is None else q.ctypes.data)
            assert got == oracle.classify2(p, q)


def test_variant_map_matches_oracle(abi):
    for cls in range(16):
        for avg, mx in [(10, 1000), (10, 100), (1, 33), (0, 0)]:
            v = abi.spmv_variant_for_classes(cls, avg, mx, 32.0)
            assert v.as_tuple()[:4] == oracle.variant_for_classes(cls, avg, mx, 32.0)


def test_bounds_match_oracle(abi):
    out = np.zeros(3)
    for args in [(4, 4, 10, 4, 8, 8, 100.0), (4096000, 4096000, 109215352, 4, 8, 8, 6793.4),
                 (16_000_000, 16_000_000, 128_000_000, 2, 2, 4, 7000.0)]:
        abi.spmv_bounds(*args, out.ctypes.data)
        assert tuple(out) == oracle.bounds(*args)


def test_feature_rules_match_oracle(abi):
    rng = np.random.default_rng(1)
    for _ in range(3000):
        f = np.zeros(14)
        f[0] = float(rng.integers(0, 2))
        f[4] = float(rng.choice([0.0, 2.0, 5.0, 30.0]))
        f[3] = f[4] * float(rng.choice([1.0, 20.0, 40.0]))
        f[13] = f[4] * float(rng.choice([0.2, 0.5, 0.9]))
        n_cols = int(rng.choice([10 ** 5, 10 ** 7, 10 ** 8]))
        vb = int(rng.choice([4, 8]))
        l2 = 126 << 20
        assert abi.spmv_feature_rules(f.ctypes.data, n_cols, vb, l2, 32.0) == \
            oracle.feature_rules(f, n_cols, vb, l2, 32.0)


def test_product_path_has_no_oracle_or_fallback():
    """The package must not import the oracle nor compute anything on the host."""
    pkg = os.path.join(ROOT, "paper_1711_05487_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "spmv_oracle" not in text, f
