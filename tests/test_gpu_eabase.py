"""EABase (Alg. 4: every cell until the computation is abandoned) on the GPU,
through the C ABI: exact distances below the cut-off, D or +inf above it,
1-NN identical to Base and to the FP64 oracle."""
import math

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
    return kw


@pytest.mark.parametrize("kind", KINDS)
def test_eabase_nn1_equals_base_and_oracle(eap, kind):
    rng = np.random.default_rng(500 + KINDS.index(kind))
    qlen = list(rng.integers(1, 300, size=12)) + [1, 2, 31, 33, 257]
    rlen = list(rng.integers(1, 300, size=40)) + [1, 64, 129, 300]
    Qp = synth.ragged_walks(len(qlen), qlen, 17 + KINDS.index(kind), n_classes=3)
    Rp = synth.ragged_walks(len(rlen), rlen, 18 + KINDS.index(kind), n_classes=3)
    Q, R = eap.SeriesSet.from_packed(Qp), eap.SeriesSet.from_packed(Rp)
    kw = _kw(kind)
    i0, d0 = eap.eap_nn1(gpu_params(eap, kind, prune=0, **kw), Q, R)
    i2, d2, st = eap.eap_nn1(gpu_params(eap, kind, prune=2, **kw), Q, R, with_stats=True)
    assert np.array_equal(i2.cpu().numpy(), i0.cpu().numpy())
    assert np.array_equal(d2.cpu().numpy(), d0.cpu().numpy())
    D = O.cross(oracle_params(kind, **kw), Qp, Rp)
    check_nn(i2.cpu().numpy(), d2.cpu().numpy(), D)
    assert st["pairs"] == len(qlen) * len(rlen)
    assert st["cells_computed"] <= st["cells_effective"]


@pytest.mark.parametrize("kind", KINDS)
def test_eabase_pairs_contract(eap, kind):
    """D exactly when D <= cut-off (bit-identical to Base); D or +inf above."""
    rng = np.random.default_rng(41)
    Ap = synth.ragged_walks(14, list(rng.integers(20, 420, size=14)), 71, n_classes=2)
    Bp = synth.ragged_walks(14, list(rng.integers(20, 420, size=14)), 72, n_classes=2)
    A, B = eap.SeriesSet.from_packed(Ap), eap.SeriesSet.from_packed(Bp)
    kw = _kw(kind, 0.6)
    ia = np.repeat(np.arange(14), 14).astype(np.int32)
    ib = np.tile(np.arange(14), 14).astype(np.int32)
    base = eap.eap_pairs(gpu_params(eap, kind, prune=0, **kw), A, B, ia, ib).cpu().numpy()
    D = O.cross(oracle_params(kind, **kw), Ap, Bp)
    for k in range(len(ia)):
        assert close(float(base[k]), float(D[ia[k], ib[k]]))
    p2 = gpu_params(eap, kind, prune=2, **kw)
    fin = np.isfinite(base)
    cases = {
        "eq": base.copy(),
        "below": np.where(fin, np.nextafter(base, np.float32(0)), base).astype(np.float32),
        "half": (base * np.float32(0.5)).astype(np.float32),
        "zero": np.zeros_like(base),
        "inf": np.full_like(base, np.inf),
        "up": (base * np.float32(1.5)).astype(np.float32),
    }
    abandoned_somewhere = False
    for name, cut in cases.items():
        got, st = eap.eap_pairs(p2, A, B, ia, ib, cut, with_stats=True)
        got = got.cpu().numpy()
        below = base <= cut
        assert np.array_equal(got[below], base[below]), (kind, name)
        above = ~below
        ok = (got[above] == base[above]) | np.isinf(got[above])
        assert ok.all(), (kind, name, np.flatnonzero(~ok)[:5])
        if name in ("zero", "half") and fin.any():
            abandoned_somewhere |= st["pairs_abandoned"] > 0
    assert abandoned_somewhere, kind


def test_eabase_erp_live_vertical_border(eap):
    """ERP = 0 through a path down the vertical border, while the first row's
    only interior cell costs 5: neither EABase nor EAPruned may abandon at 4."""
    a = synth.pack([np.array([0, 0, 0, 5], np.float32)])
    b = synth.pack([np.array([5], np.float32)])
    A, B = eap.SeriesSet.from_packed(a), eap.SeriesSet.from_packed(b)
    for prune in (1, 2):
        p = eap.params("erp", erp_gap=0.0, window_ratio=-1.0, prune=prune)
        assert eap.eap_pairs(p, A, B, [0], [0], [4.0]).cpu().numpy()[0] == 0.0
        assert eap.eap_pairs(p, B, A, [0], [0], [4.0]).cpu().numpy()[0] == 0.0
        idx, dist = eap.eap_nn1(p, B, A)
        assert idx.item() == 0 and dist.item() == 0.0


def test_eabase_full_workload_sampled(eap):
    """1000 x 1000 x 512 (MSM and DTW): EABase 1-NN equals EAPruned's and the
    oracle on sampled queries, and abandons pairs."""
    ds = synth.workload_nn1_512()
    tr, te = synth.pack(ds.train), synth.pack(ds.test)
    R, Q = eap.SeriesSet.from_packed(tr), eap.SeriesSet.from_packed(te)
    for kind in ("dtw", "msm"):
        kw = WORKLOAD_PARAMS[kind]
        i1, d1 = eap.eap_nn1(gpu_params(eap, kind, prune=1, **kw), Q, R)
        i2, d2, st = eap.eap_nn1(gpu_params(eap, kind, prune=2, **kw), Q, R, with_stats=True)
        assert np.array_equal(i1.cpu().numpy(), i2.cpu().numpy())
        assert np.array_equal(d1.cpu().numpy(), d2.cpu().numpy())
        assert st["pairs_abandoned"] > 0
        rows = list(np.random.default_rng(3).choice(ds.test.shape[0], size=8, replace=False))
        sub = synth.pack([ds.test[r] for r in rows])
        D = O.cross(oracle_params(kind, **kw), sub, tr)
        check_nn(i2.cpu().numpy(), d2.cpu().numpy(), D, rows=rows)


def test_prune_mode_is_validated(eap):
    one = synth.pack([np.array([0.5, 1.0], np.float32)])
    Q = eap.SeriesSet.from_packed(one)
    with pytest.raises(eap.EapError) as e:
        eap.eap_nn1(eap.params("dtw", prune=4), Q, Q)
    assert e.value.code == eap.EAP_EINVAL
    # The batched entry point runs EAPruned only.
    t = eap.Nn1Task(eap.params("dtw", prune=2), Q, Q)
    with pytest.raises(eap.EapError):
        eap.eap_nn1_batch([t])
    assert not math.isnan(float(eap.eap_nn1(eap.params("dtw", prune=2), Q, Q)[1].item()))


@pytest.mark.parametrize("kind", KINDS)
def test_prune_only_nn1_equals_base(eap, kind):
    """Prune (mode 3: each pair's own diagonal bound as cut-off) computes
    every distance exactly: the 1-NN equals Base bit for bit and nothing is
    abandoned."""
    rng = np.random.default_rng(900 + KINDS.index(kind))
    Qp = synth.ragged_walks(10, list(rng.integers(8, 300, size=10)), 27, n_classes=3)
    Rp = synth.ragged_walks(30, list(rng.integers(8, 300, size=30)), 28, n_classes=3)
    Q, R = eap.SeriesSet.from_packed(Qp), eap.SeriesSet.from_packed(Rp)
    kw = _kw(kind, 1.0)   # a full window: every pair has an alignment
    i0, d0 = eap.eap_nn1(gpu_params(eap, kind, prune=0, **kw), Q, R)
    i3, d3, st = eap.eap_nn1(gpu_params(eap, kind, prune=3, **kw), Q, R, with_stats=True)
    assert np.array_equal(i3.cpu().numpy(), i0.cpu().numpy())
    assert np.array_equal(d3.cpu().numpy(), d0.cpu().numpy())
    assert st["pairs_abandoned"] == 0 and st["pairs"] == 300
    with pytest.raises(eap.EapError):
        eap.eap_pairs(gpu_params(eap, kind, prune=3, **kw), Q, R, [0], [0], [1.0])
