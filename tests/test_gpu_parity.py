"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Element by element on seeded inputs: 1-NN indices exact except flagged
near-ties, distances within 1e-4 relative; all-pairs matrices element-wise;
the EAPruned +inf contract bit-exact on the GPU's own float32 distances.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import KINDS, REL_TOL, WORKLOAD_PARAMS, check_nn, close, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eap():
    from paper_2102_05221_gb300 import eap as E
    E.load()
    return E


def _sets(eap, *packed):
    return [eap.SeriesSet.from_packed(p) for p in packed]


def test_small_dtw_unpruned_1nn(eap):
    """64 train x 32 test, length 128, plain (unpruned) DTW 1-NN."""
    ds = synth.workload_small_dtw()
    tr, te = synth.pack(ds.train), synth.pack(ds.test)
    R, Q = _sets(eap, tr, te)
    idx, dist = eap.eap_nn1(eap.params("dtw", prune=0), Q, R)
    D = O.cross(O.make_params("dtw"), te, tr)
    check_nn(idx.cpu().numpy(), dist.cpu().numpy(), D)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prune", [1, 0])
def test_nn1_ragged_all_distances(eap, kind, prune):
    """Uneven lengths (1..300, several tiles and a ragged tail) for every distance."""
    rng = np.random.default_rng(100 + KINDS.index(kind))
    qlen = list(rng.integers(1, 300, size=12)) + [1, 2, 31, 32, 33, 257]
    rlen = list(rng.integers(1, 300, size=40)) + [1, 64, 128, 129, 300]
    Qp = synth.ragged_walks(len(qlen), qlen, 7 + KINDS.index(kind), n_classes=3)
    Rp = synth.ragged_walks(len(rlen), rlen, 8 + KINDS.index(kind), n_classes=3)
    kw = dict(WORKLOAD_PARAMS[kind])
    if kind in ("cdtw", "erp"):
        kw["window_ratio"] = 0.3
    Q, R = _sets(eap, Qp, Rp)
    idx, dist = eap.eap_nn1(gpu_params(eap, kind, prune=prune, **kw), Q, R)
    D = O.cross(oracle_params(kind, **kw), Qp, Rp)
    check_nn(idx.cpu().numpy(), dist.cpu().numpy(), D)


@pytest.mark.parametrize("kind", KINDS)
def test_pairs_inf_contract_is_exact(eap, kind):
    """EAPruned returns D exactly when D <= cut-off and +inf otherwise
    (Section 2.2), on the GPU's own float32 D: cut-offs D, the next float
    below D, 0, +inf and D*(1 +- 1e-3)."""
    rng = np.random.default_rng(5)
    lens = list(rng.integers(20, 400, size=16))
    Ap = synth.ragged_walks(16, lens, 31, n_classes=2)
    Bp = synth.ragged_walks(16, list(rng.integers(20, 400, size=16)), 32, n_classes=2)
    kw = dict(WORKLOAD_PARAMS[kind])
    if kind in ("cdtw", "erp"):
        kw["window_ratio"] = 0.5
    A, B = _sets(eap, Ap, Bp)
    ia = np.repeat(np.arange(16), 16).astype(np.int32)
    ib = np.tile(np.arange(16), 16).astype(np.int32)
    base = eap.eap_pairs(gpu_params(eap, kind, prune=0, **kw), A, B, ia, ib).cpu().numpy()
    D = O.cross(oracle_params(kind, **kw), Ap, Bp)
    for k in range(len(ia)):
        assert close(float(base[k]), float(D[ia[k], ib[k]])), (kind, k, base[k], D[ia[k], ib[k]])
    p1 = gpu_params(eap, kind, prune=1, **kw)
    fin = np.isfinite(base)
    cases = {
        "eq": base.copy(),
        "below": np.where(fin, np.nextafter(base, np.float32(0)), base).astype(np.float32),
        "zero": np.zeros_like(base),
        "inf": np.full_like(base, np.inf),
        "up": (base * np.float32(1.001)).astype(np.float32),
        "down": (base * np.float32(0.999)).astype(np.float32),
    }
    for name, cut in cases.items():
        got = eap.eap_pairs(p1, A, B, ia, ib, cut).cpu().numpy()
        want = np.where(base <= cut, base, np.float32(np.inf))
        assert np.array_equal(got, want), (kind, name, np.flatnonzero(got != want)[:5])


@pytest.mark.parametrize("kind", KINDS)
def test_pairwise_prune_only_equals_base_and_oracle(eap, kind):
    """Prune-only mode (cut-off = each pair's diagonal-path cost) is exact:
    bit-identical to Base on the GPU, and within tolerance of the oracle."""
    rng = np.random.default_rng(9)
    Sp = synth.ragged_walks(20, list(rng.integers(40, 300, size=20)), 41)
    kw = dict(WORKLOAD_PARAMS[kind])
    if kind in ("cdtw", "erp"):
        kw["window_ratio"] = 0.9
    (S,) = _sets(eap, Sp)
    m_pr = eap.eap_pairwise(gpu_params(eap, kind, **kw), S, eap.EAP_PRUNE_ONLY).cpu().numpy()
    m_base = eap.eap_pairwise(gpu_params(eap, kind, **kw), S, eap.EAP_BASE).cpu().numpy()
    assert np.array_equal(m_pr, m_base)
    M = O.pairwise(oracle_params(kind, **kw), Sp)
    for i in range(20):
        assert m_pr[i, i] == 0.0
        for j in range(20):
            if i < j:
                assert close(float(m_pr[i, j]), float(M[i, j])), (kind, i, j, m_pr[i, j], M[i, j])
            assert m_pr[i, j] == m_pr[j, i]


def test_edge_cases(eap):
    """Empty sets, length-1 series, and windows too small for any alignment."""
    one = synth.pack([np.array([0.5], np.float32)])
    Q, R = _sets(eap, one, one)
    idx, dist = eap.eap_nn1(eap.params("dtw"), Q, R)
    assert idx.item() == 0 and dist.item() == 0.0
    # No candidates: -1 / +inf.
    empty = eap.SeriesSet(np.zeros(0, np.float32), np.zeros(0, np.int64), np.zeros(0, np.int32))
    idx, dist = eap.eap_nn1(eap.params("dtw"), Q, empty)
    assert idx.item() == -1 and math.isinf(dist.item())
    # No queries: nothing to do.
    idx, dist = eap.eap_nn1(eap.params("dtw"), empty, R)
    assert idx.numel() == 0
    # CDTW window 1 between lengths 6 and 8 (Fig. CDTW): no alignment.
    a = synth.pack([np.array([3, 1, 4, 4, 1, 1], np.float32)])
    b = synth.pack([np.array([1, 3, 2, 1, 2, 2, 0, 5], np.float32), np.array([1, 3, 2, 1, 2, 2, 0], np.float32)])
    A, B = _sets(eap, a, b)
    idx, dist = eap.eap_nn1(eap.params("cdtw", window=1, window_ratio=-1.0), A, B)
    assert idx.item() == 1 and math.isfinite(dist.item())
    b2 = synth.pack([np.array([1, 3, 2, 1, 2, 2, 0, 5], np.float32)])
    (B2,) = _sets(eap, b2)
    idx, dist = eap.eap_nn1(eap.params("cdtw", window=1, window_ratio=-1.0), A, B2)
    assert idx.item() == -1 and math.isinf(dist.item())
    # Worked example: DTW(S,T) = 9.
    t = synth.pack([np.array([1, 3, 2, 1, 2, 2], np.float32)])
    (T,) = _sets(eap, t)
    idx, dist = eap.eap_nn1(eap.params("dtw"), A, T)
    assert dist.item() == 9.0
    out = eap.eap_pairs(eap.params("dtw"), A, T, [0], [0], [6.0]).cpu().numpy()
    assert math.isinf(out[0])
    out = eap.eap_pairs(eap.params("dtw"), A, T, [0], [0], [9.0]).cpu().numpy()
    assert out[0] == 9.0
    # Negative cut-off: everything is above it.
    out = eap.eap_pairs(eap.params("dtw"), A, T, [0], [0], [-1.0]).cpu().numpy()
    assert math.isinf(out[0])


def test_invalid_arguments_are_rejected(eap):
    one = synth.pack([np.array([0.5, 1.0], np.float32)])
    Q, R = _sets(eap, one, one)
    with pytest.raises(eap.EapError) as e:
        eap.eap_nn1(eap.params("msm", msm_c=-1.0), Q, R)
    assert e.value.code == eap.EAP_EINVAL
    bad_kind = eap.params("dtw")
    bad_kind.kind = 9
    with pytest.raises(eap.EapError):
        eap.eap_nn1(bad_kind, Q, R)
    bad = eap.SeriesSet(np.zeros(4, np.float32), np.array([0, 3], np.int64), np.array([2, 2], np.int32))
    with pytest.raises(eap.EapError):
        eap.eap_nn1(eap.params("dtw"), bad, R)
    zero_len = eap.SeriesSet(np.zeros(4, np.float32), np.array([0], np.int64), np.array([0], np.int32))
    with pytest.raises(eap.EapError):
        eap.eap_nn1(eap.params("dtw"), zero_len, R)


def test_lb_keogh_matches_oracle_and_bounds_cdtw(eap):
    x = synth.ragged_walks(10, [200] * 10, 55)
    (X,) = _sets(eap, x)
    ia = np.repeat(np.arange(10), 10).astype(np.int32)
    ib = np.tile(np.arange(10), 10).astype(np.int32)
    for w in (0, 5, 20):
        lb = eap.eap_lb_keogh(eap.params("cdtw", window=w, window_ratio=-1.0), X, X, ia, ib).cpu().numpy()
        dd = eap.eap_pairs(eap.params("cdtw", window=w, window_ratio=-1.0, prune=0), X, X, ia, ib).cpu().numpy()
        for k in range(len(ia)):
            ref = O.lb_keogh(x.series(ia[k]), x.series(ib[k]), w)
            assert close(float(lb[k]), ref) or (ref == 0 and lb[k] == 0)
            assert lb[k] <= dd[k] * (1 + 1e-5)


@pytest.mark.parametrize("kind", KINDS)
def test_nn1_full_workload_sampled(eap, kind):
    """1000 train x 1000 test, length 512, the launch the benchmark times;
    24 sampled queries checked against the oracle's full distance rows."""
    ds = synth.workload_nn1_512()
    tr, te = synth.pack(ds.train), synth.pack(ds.test)
    R, Q = _sets(eap, tr, te)
    kw = WORKLOAD_PARAMS[kind]
    idx, dist = eap.eap_nn1(gpu_params(eap, kind, **kw), Q, R)
    rows = list(np.random.default_rng(KINDS.index(kind)).choice(ds.test.shape[0], size=24, replace=False))
    sub = synth.pack([ds.test[r] for r in rows])
    D = O.cross(oracle_params(kind, **kw), sub, tr)
    check_nn(idx.cpu().numpy(), dist.cpu().numpy(), D, rows=rows)


@pytest.mark.parametrize("kind", ["dtw", "cdtw"])
@pytest.mark.parametrize("lb", [1, 2])
def test_nn1_with_lb_keogh_cascade(eap, kind, lb):
    """Alg. 2: LB_Keogh (and the two-way lb-keogh2 cascade) ahead of EAPruned
    changes no result, and skips pairs."""
    ds = synth.make_dataset(400, 60, 256, 5, 4242)
    tr, te = synth.pack(ds.train), synth.pack(ds.test)
    R, Q = _sets(eap, tr, te)
    kw = {"window_ratio": 0.1} if kind == "cdtw" else {}
    i0, d0, s0 = eap.eap_nn1(gpu_params(eap, kind, **kw), Q, R, with_stats=True)
    i1, d1, s1 = eap.eap_nn1(gpu_params(eap, kind, lb=lb, **kw), Q, R, with_stats=True)
    assert np.array_equal(i0.cpu().numpy(), i1.cpu().numpy())
    assert np.array_equal(d0.cpu().numpy(), d1.cpu().numpy())
    assert s1["pairs_lb_pruned"] > 0 and s0["pairs_lb_pruned"] == 0
    D = O.cross(oracle_params(kind, **kw), te, tr)
    check_nn(i1.cpu().numpy(), d1.cpu().numpy(), D)


def test_validation_mode_rejects_non_finite_inputs(eap):
    """EAP_CHECK_INPUTS=1 scans the inputs for NaN / Inf first."""
    import os
    x = synth.ragged_walks(4, [50] * 4, 91)
    bad = synth.pack([x.series(0), np.where(np.arange(50) == 7, np.nan, x.series(1)).astype(np.float32)])
    Q, B = eap.SeriesSet.from_packed(x), eap.SeriesSet.from_packed(bad)
    T = np.concatenate([x.series(0), [np.inf], x.series(1)]).astype(np.float32)
    old = os.environ.get("EAP_CHECK_INPUTS")
    os.environ["EAP_CHECK_INPUTS"] = "1"
    try:
        for call in (lambda: eap.eap_nn1(eap.params("dtw"), Q, B),
                     lambda: eap.eap_pairs(eap.params("msm"), B, Q, [1], [0], [1.0]),
                     lambda: eap.eap_pairwise(eap.params("erp"), B),
                     lambda: eap.eap_subseq(eap.params("cdtw"), T, Q)):
            with pytest.raises(eap.EapError) as e:
                call()
            assert e.value.code == eap.EAP_EINVAL
        # Finite inputs pass the scan.
        idx, dist = eap.eap_nn1(eap.params("dtw"), Q, Q)
        assert np.array_equal(idx.cpu().numpy(), np.arange(4))
    finally:
        if old is None:
            del os.environ["EAP_CHECK_INPUTS"]
        else:
            os.environ["EAP_CHECK_INPUTS"] = old
