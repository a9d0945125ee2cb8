"""The learned selector end to end at a small scale: dataset labelled by the profile route,
GPU training, decisions bit-exact against the oracle's FP32 inference, the learned tuning
route reproducing them, and what the network gains over the method without it (the profile
route): the same variant choices at a fraction of the tuning time."""
import numpy as np
import pytest

import oracle
from gpu_util import torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return torch_cuda()


@pytest.fixture(scope="module")
def trained(torch):
    from paper_1711_05487_gb300 import selector_train as st
    ds = st.build_dataset(72, seed=424242, n_lo=3000, n_hi=60_000, reps=3, workers=4, log=None)
    tr, te = np.arange(56), np.arange(56, 72)
    params, mu, inv, hist = st.train(ds["feat16"][tr], ds["classes"][tr], steps=1500, lr=5e-3)
    return st, ds, tr, te, params, mu, inv, hist


def test_training_fits_profile_labels(trained):
    st, ds, tr, te, params, mu, inv, hist = trained
    assert hist[-1] < 0.5 * hist[0]
    pred, _ = st.predict(params, mu, inv, ds["feat16"][tr])
    ev = st.evaluate(ds, tr, pred)
    assert ev["partial_match_ratio"] >= 0.9, ev
    assert ev["exact_match_ratio"] >= 0.75, ev


def test_decisions_bit_exact_vs_oracle(trained):
    st, ds, tr, te, params, mu, inv, hist = trained
    pred, lg = st.predict(params, mu, inv, ds["feat16"])
    X = oracle.mlp_inputs(ds["feat16"], mu, inv)
    Lo = oracle.mlp_logits_f32(np.array(st.SIZES, np.int32), params, X)
    assert np.array_equal(lg.view(np.uint32), Lo.view(np.uint32))
    want = np.zeros(len(pred), dtype=np.int32)
    for b in range(4):
        want |= (Lo[:, b] > 0).astype(np.int32) << b
    assert np.array_equal(pred, want)


def test_learned_route_gains_over_profiling(trained, torch):
    import synth
    from paper_1711_05487_gb300 import api
    st, ds, tr, te, params, mu, inv, hist = trained
    sel = api.Selector(st.SIZES, params, mu, inv)
    pred, _ = st.predict(params, mu, inv, ds["feat16"][te])
    t_learned, t_profile = [], []
    for k, i in enumerate(te[:8]):
        m = synth.make_from_spec(synth.mixed_spec(int(i), seed=424242, n_lo=3000, n_hi=60_000))
        A = api.SpmvMatrix.from_csr(m)
        r = A.tune("learned", selector=sel, autotune=0)
        assert r.mode_used == 2 and r.classes == pred[k]
        t_learned.append(r.t_pre_ms)
        t_profile.append(A.tune("profile", autotune=0).t_pre_ms)
    # the trained network replaces the micro-benchmarks: tuning is several times cheaper
    assert np.median(t_learned) * 3 < np.median(t_profile), (t_learned, t_profile)
