"""Derivative variants (DDTW, DCDTW, DWDTW, DERP, DMSM, DTWE; Section 2.3):
every entry point with derivative = 1 against the FP64 oracle's derivative
distances, element by element on seeded ragged inputs."""
import math
import time

import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import KINDS, WORKLOAD_PARAMS, check_nn, close, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eap():
    from paper_2102_05221_gb300 import eap as E
    E.load()
    return E


def _kw(kind, ratio=0.3):
    kw = dict(WORKLOAD_PARAMS[kind])
    if kind in ("cdtw", "erp"):
        kw["window_ratio"] = ratio
    kw["derivative"] = 1
    return kw


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("prune", [1, 0])
def test_derivative_nn1_ragged(eap, kind, prune):
    """Ragged lengths 1..300 (one- and two-point series have zero derivative)."""
    rng = np.random.default_rng(300 + KINDS.index(kind))
    qlen = list(rng.integers(3, 300, size=10)) + [1, 2, 3, 33, 257]
    rlen = list(rng.integers(3, 300, size=36)) + [1, 2, 64, 129, 300]
    Qp = synth.ragged_walks(len(qlen), qlen, 61 + KINDS.index(kind), n_classes=3)
    Rp = synth.ragged_walks(len(rlen), rlen, 62 + KINDS.index(kind), n_classes=3)
    kw = _kw(kind)
    Q, R = eap.SeriesSet.from_packed(Qp), eap.SeriesSet.from_packed(Rp)
    idx, dist = eap.eap_nn1(gpu_params(eap, kind, prune=prune, **kw), Q, R)
    D = O.cross(oracle_params(kind, **kw), Qp, Rp)
    check_nn(idx.cpu().numpy(), dist.cpu().numpy(), D)
    # The derivative changes the answer: the plain distance ranks differently somewhere.
    D0 = O.cross(oracle_params(kind, **dict(kw, derivative=0)), Qp, Rp)
    assert not np.allclose(D, D0)


@pytest.mark.parametrize("kind", KINDS)
def test_derivative_pairwise_and_pairs(eap, kind):
    rng = np.random.default_rng(7 + KINDS.index(kind))
    Sp = synth.ragged_walks(18, list(rng.integers(20, 260, size=18)), 91)
    kw = _kw(kind, 0.9)
    (S,) = [eap.SeriesSet.from_packed(Sp)]
    m_pr = eap.eap_pairwise(gpu_params(eap, kind, **kw), S, eap.EAP_PRUNE_ONLY).cpu().numpy()
    m_base = eap.eap_pairwise(gpu_params(eap, kind, **kw), S, eap.EAP_BASE).cpu().numpy()
    assert np.array_equal(m_pr, m_base)
    M = O.pairwise(oracle_params(kind, **kw), Sp)
    for i in range(18):
        for j in range(i + 1, 18):
            assert close(float(m_pr[i, j]), float(M[i, j])), (kind, i, j, m_pr[i, j], M[i, j])
    # Raw EAPruned pairs: D exactly at cut-off D, +inf just below it.
    ia = np.repeat(np.arange(18), 18).astype(np.int32)
    ib = np.tile(np.arange(18), 18).astype(np.int32)
    base = eap.eap_pairs(gpu_params(eap, kind, prune=0, **kw), S, S, ia, ib).cpu().numpy()
    for k in range(len(ia)):
        assert close(float(base[k]), float(M[ia[k], ib[k]])), (kind, k)
    p1 = gpu_params(eap, kind, prune=1, **kw)
    assert np.array_equal(eap.eap_pairs(p1, S, S, ia, ib, base).cpu().numpy(), base)
    below = np.where(np.isfinite(base) & (base > 0), np.nextafter(base, np.float32(0)), base).astype(np.float32)
    got = eap.eap_pairs(p1, S, S, ia, ib, below).cpu().numpy()
    want = np.where(base <= below, base, np.float32(np.inf))
    assert np.array_equal(got, want)
    # The allocation-free variant derives into its fixed scratch and agrees bit for bit.
    assert np.array_equal(eap.eap_pairs_noalloc(p1, S, S, ia, ib, below).cpu().numpy(), want)


def test_derivative_offsets_do_not_matter(eap):
    """A series and the same series shifted by a constant are at distance 0."""
    x = (np.random.default_rng(3).integers(-64, 64, size=(6, 200)) / 16.0).astype(np.float32)
    A = eap.SeriesSet.from_packed(synth.pack(list(x)))
    B = eap.SeriesSet.from_packed(synth.pack(list(x + np.float32(2.5))))
    for kind in KINDS:
        idx, dist = eap.eap_nn1(eap.params(kind, derivative=1), A, B)
        assert np.array_equal(idx.cpu().numpy(), np.arange(6)), kind
        assert np.all(dist.cpu().numpy() == 0.0), kind


def test_derivative_lb_keogh_bounds_dcdtw(eap):
    x = synth.ragged_walks(8, [160] * 8, 57)
    (X,) = [eap.SeriesSet.from_packed(x)]
    ia = np.repeat(np.arange(8), 8).astype(np.int32)
    ib = np.tile(np.arange(8), 8).astype(np.int32)
    p = eap.params("cdtw", window=8, window_ratio=-1.0, derivative=1)
    lb = eap.eap_lb_keogh(p, X, X, ia, ib).cpu().numpy()
    dd = eap.eap_pairs(eap.params("cdtw", window=8, window_ratio=-1.0, prune=0, derivative=1), X, X, ia, ib).cpu().numpy()
    assert np.all(lb <= dd * (1 + 1e-5))
    assert lb[ia != ib].sum() > 0
    # LB_Keogh-accelerated DCDTW 1-NN equals the oracle.
    idx, dist = eap.eap_nn1(eap.params("cdtw", window=8, window_ratio=-1.0, derivative=1, lb=2), X, X)
    D = O.cross(O.make_params("cdtw", window=8, derivative=1), x, x)
    check_nn(idx.cpu().numpy(), dist.cpu().numpy(), D)


def test_derivative_in_batch_and_serving(eap):
    import torch
    tasks, refs = [], []
    for d, kind in enumerate(KINDS):
        ds = synth.make_dataset(60, 12, 96 + 40 * d, 3, 7100 + d)
        tr, te = synth.pack(ds.train), synth.pack(ds.test)
        kw = _kw(kind, 0.2) if d % 2 == 0 else dict(WORKLOAD_PARAMS[kind])
        tasks.append((kind, kw, tr, te, eap.Nn1Task(gpu_params(eap, kind, **kw), eap.SeriesSet.from_packed(te),
                                                    eap.SeriesSet.from_packed(tr))))
    eap.eap_nn1_batch([t for *_, t in tasks])
    torch.cuda.synchronize()
    for kind, kw, tr, te, t in tasks:
        i1, d1 = eap.eap_nn1(t.p, t.queries, t.refs)
        assert np.array_equal(t.out_idx.cpu().numpy(), i1.cpu().numpy()), kind
        assert np.array_equal(t.out_dist.cpu().numpy(), d1.cpu().numpy()), kind
        D = O.cross(oracle_params(kind, **kw), te, tr)
        check_nn(t.out_idx.cpu().numpy(), t.out_dist.cpu().numpy(), D)
    # Serving: derivative queries against a resident set.
    refs = synth.ragged_walks(120, (64, 300), 81)
    qs = synth.ragged_walks(12, (64, 300), 82)
    with eap.Server(max_inflight=32) as srv:
        sid = srv.add_refset(refs)
        jobs = []
        for i in range(12):
            kind = KINDS[i % 6]
            kw = _kw(kind, 0.5)
            while True:
                t = srv.submit(sid, gpu_params(eap, kind, **kw), qs.series(i))
                if t is not None:
                    break
                time.sleep(0.001)
            jobs.append((t, kind, kw, qs.series(i)))
        srv.drain(60000)
        for t, kind, kw, q in jobs:
            idx, dist = srv.poll(t)
            D = O.cross(oracle_params(kind, **kw), synth.pack([q]), refs)
            check_nn(np.array([idx]), np.array([dist]), D)


def test_derivative_flag_is_validated(eap):
    one = synth.pack([np.array([0.5, 1.0, 2.0], np.float32)])
    Q = eap.SeriesSet.from_packed(one)
    with pytest.raises(eap.EapError) as e:
        eap.eap_nn1(eap.params("dtw", derivative=2), Q, Q)
    assert e.value.code == eap.EAP_EINVAL
    idx, dist = eap.eap_nn1(eap.params("dtw", derivative=1), Q, Q)
    assert idx.item() == 0 and dist.item() == 0.0 and not math.isnan(dist.item())


def test_near_zero_distance_between_short_series(eap):
    """ERP (squared cost) with derivative series, 7 queries against 39
    candidates of 2 to 561 points (a seeded random configuration).  Query 2
    and its nearest candidate have 3 points each, so both derivative series
    are constant and the distance, 1.13e-5, is 3 (a - b)^2 with |a - b| far
    below the values' size.  Per-step float rounding of the estimate missed
    the 1e-4 relative tolerance here (1.1e-4); one rounding of an estimate
    evaluated in double keeps it inside."""
    from tests.test_gpu_random_configs import EDGE_LENGTHS, _config
    seed = 50179
    rng = np.random.default_rng(seed)
    cfg = _config(rng)
    assert cfg["kind"] == "erp" and cfg["gpu"]["derivative"] == 1
    nq, nr = int(rng.integers(1, 12)), int(rng.integers(1, 40))
    pool = EDGE_LENGTHS + list(rng.integers(1, 600, size=8))
    qlen = [int(rng.choice(pool)) for _ in range(nq)]
    rlen = [int(rng.choice(pool)) for _ in range(nr)]
    Qp = synth.ragged_walks(nq, qlen, seed + 7, n_classes=3)
    Rp = synth.ragged_walks(nr, rlen, seed + 11, n_classes=3)
    Q, R = eap.SeriesSet.from_packed(Qp), eap.SeriesSet.from_packed(Rp)
    idx, dist = eap.eap_nn1(eap.params("erp", **cfg["gpu"]), Q, R)
    D = O.cross(O.make_params("erp", **cfg["orc"]), Qp, Rp)
    assert qlen[2] == 3 and 0 < D[2].min() < 1e-4
    check_nn(idx.cpu().numpy(), dist.cpu().numpy(), D)
