"""EAPruned with 16 or 8 lanes per pair (several pairs per warp): the same
results as a warp per pair, bit for bit, for 1-NN, explicit pairs with
cut-offs and prune-only matrices, every distance, ragged lengths."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import KINDS, WORKLOAD_PARAMS, check_nn, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


def _with_env(env, fn):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return fn()
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


def _kw(kind):
    kw = dict(WORKLOAD_PARAMS[kind])
    if kind in ("cdtw", "erp"):
        kw["window_ratio"] = 0.3
    return kw


@pytest.mark.parametrize("kind", KINDS)
def test_groups_match_warp_per_pair(kind):
    from paper_2102_05221_gb300 import eap
    rng = np.random.default_rng(700 + KINDS.index(kind))
    qlen = list(rng.integers(1, 400, size=14)) + [1, 2, 63, 64, 65, 129]
    rlen = list(rng.integers(1, 400, size=40)) + [1, 64, 128, 257, 400]
    Qp = synth.ragged_walks(len(qlen), qlen, 81 + KINDS.index(kind), n_classes=3)
    Rp = synth.ragged_walks(len(rlen), rlen, 82 + KINDS.index(kind), n_classes=3)
    Q, R = eap.SeriesSet.from_packed(Qp), eap.SeriesSet.from_packed(Rp)
    p = gpu_params(eap, kind, **_kw(kind))
    nq, nr = len(qlen), len(rlen)
    ia = np.repeat(np.arange(nq), nr).astype(np.int32)
    ib = np.tile(np.arange(nr), nq).astype(np.int32)

    def run():
        i, d = eap.eap_nn1(p, Q, R)
        base = eap.eap_pairs(gpu_params(eap, kind, prune=0, **_kw(kind)), Q, R, ia, ib).cpu().numpy()
        cut = np.where(np.isfinite(base), base * np.float32(0.999), base).astype(np.float32)
        cut[::2] = base[::2]
        pr = eap.eap_pairs(p, Q, R, ia, ib, cut).cpu().numpy()
        return i.cpu().numpy(), d.cpu().numpy(), pr

    ref = _with_env({"EAP_G": "32", "EAP_W": "4"}, run)
    for g, w in (("16", "4"), ("16", "5"), ("16", "8"), ("8", "4"), ("8", "8")):
        got = _with_env({"EAP_G": g, "EAP_W": w}, run)
        for a, b in zip(ref, got):
            assert np.array_equal(a, b), (kind, g, w)
    D = O.cross(oracle_params(kind, **_kw(kind)), Qp, Rp)
    check_nn(ref[0], ref[1], D)


def test_groups_prune_only_matrix_and_subseq():
    from paper_2102_05221_gb300 import eap
    Sp = synth.ragged_walks(24, list(np.random.default_rng(5).integers(30, 300, size=24)), 83)
    (S,) = [eap.SeriesSet.from_packed(Sp)]
    p = eap.params("msm")
    m32 = _with_env({"EAP_G": "32", "EAP_W": "4"}, lambda: eap.eap_pairwise(p, S, eap.EAP_PRUNE_ONLY).cpu().numpy())
    m16 = _with_env({"EAP_G": "16", "EAP_W": "4"}, lambda: eap.eap_pairwise(p, S, eap.EAP_PRUNE_ONLY).cpu().numpy())
    assert np.array_equal(m32, m16)
    T = synth.long_series(20000, 84)
    Qp, _ = synth.subseq_queries(T, [64, 200], 85)
    Q = eap.SeriesSet.from_packed(Qp)
    pc = eap.params("cdtw", window_ratio=0.1)
    a = _with_env({"EAP_G": "32"}, lambda: [x.cpu().numpy() for x in eap.eap_subseq(pc, T, Q)])
    b = _with_env({"EAP_G": "8"}, lambda: [x.cpu().numpy() for x in eap.eap_subseq(pc, T, Q)])
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
