"""Sub-sequence search (Section 5.3) through the C ABI against the FP64
oracle: every z-normalised window of a long series, DTW and CDTW."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import REL_TOL, TIE_REL, close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eap():
    from paper_2102_05221_gb300 import eap as E
    E.load()
    return E


def _check(eap, kind, kw, T, Qp, pos, dist):
    """Positions equal the oracle's unless the oracle's best two windows are a
    near-tie; distances within tolerance; the GPU's window re-evaluated by the
    oracle gives the GPU's distance."""
    p = O.make_params(kind, **kw)
    for k in range(Qp.lengths.shape[0]):
        q = Qp.series(k)
        opos, od = O.subseq(p, T, q)
        gpos, gd = int(pos[k]), float(dist[k])
        if opos < 0:
            assert gpos == -1 and math.isinf(gd)
            continue
        assert close(gd, od), (kind, k, gpos, opos, gd, od)
        if gpos != opos:
            # Allowed only when the two windows' oracle distances are within a near-tie.
            d_at = O.subseq(p, T[gpos:gpos + len(q)], q)[1]
            assert abs(d_at - od) <= TIE_REL * max(od, 1e-30), (kind, k, gpos, opos, d_at, od)


@pytest.mark.parametrize("kind,kw", [("dtw", {}), ("cdtw", {"window_ratio": 0.1}), ("cdtw", {"window": 0})])
def test_subseq_matches_oracle(eap, kind, kw):
    T = synth.long_series(6000, 901)
    lens = [1, 2, 16, 31, 64, 100, 257]
    Qp, planted = synth.subseq_queries(T, lens, 902, planted=True, noise=0.2)
    Qr, _ = synth.subseq_queries(T, [24, 80, 130], 903, planted=False)
    Q = eap.SeriesSet.from_packed(Qp)
    pos, dist, st = eap.eap_subseq(eap.params(kind, **dict(kw, **({"window_ratio": -1.0} if "window" in kw else {}))),
                                   T, Q, with_stats=True)
    _check(eap, kind, kw, T, Qp, pos.cpu().numpy(), dist.cpu().numpy())
    assert st["pairs"] == sum(6000 - m + 1 for m in lens)
    R = eap.SeriesSet.from_packed(Qr)
    pos, dist = eap.eap_subseq(eap.params(kind, **dict(kw, **({"window_ratio": -1.0} if "window" in kw else {}))),
                               T, R)
    _check(eap, kind, kw, T, Qr, pos.cpu().numpy(), dist.cpu().numpy())


def test_subseq_edge_cases(eap):
    T = synth.long_series(300, 904)
    Qp = synth.pack([T[:301].copy() if len(T) > 300 else np.concatenate([T, T[:1]]), T.copy(), T[50:90].copy()])
    pos, dist = eap.eap_subseq(eap.params("dtw"), T, eap.SeriesSet.from_packed(Qp))
    pos, dist = pos.cpu().numpy(), dist.cpu().numpy()
    assert pos[0] == -1 and math.isinf(dist[0])        # longer than the series
    # The query is normalised in double, windows from float32 sliding sums:
    # an exact copy is at distance ~0, not exactly 0.
    assert pos[1] == 0 and dist[1] < 1e-6              # the whole series: one window
    assert pos[2] == 50 and dist[2] < 1e-6             # an exact copy
    # Constant windows normalise to zeros: a flat query finds the flat stretch.
    flat = np.concatenate([T[:100], np.full(30, 2.0, np.float32), T[100:]]).astype(np.float32)
    pos, dist = eap.eap_subseq(eap.params("cdtw", window_ratio=0.1), flat,
                               eap.SeriesSet.from_packed(synth.pack([np.full(20, -3.0, np.float32)])))
    assert int(pos.item()) == 100 and float(dist.item()) == 0.0
    # Other distances and modes are rejected.
    with pytest.raises(eap.EapError):
        eap.eap_subseq(eap.params("msm"), T, eap.SeriesSet.from_packed(Qp))
    with pytest.raises(eap.EapError):
        eap.eap_subseq(eap.params("dtw", prune=0), T, eap.SeriesSet.from_packed(Qp))


def test_subseq_full_size_sampled(eap):
    """A 4M-point series, planted queries of 128 and 512 points (CDTW 10%):
    the GPU's distance is the oracle's at the returned window, and no window
    of a random sample (plus the planted one) is closer."""
    T = synth.long_series(1 << 22, 905)
    Qp, planted = synth.subseq_queries(T, [128, 512], 906, planted=True, noise=0.1)
    kw = {"window_ratio": 0.1}
    pos, dist, st = eap.eap_subseq(eap.params("cdtw", **kw), T, eap.SeriesSet.from_packed(Qp), with_stats=True)
    pos, dist = pos.cpu().numpy(), dist.cpu().numpy()
    assert st["pairs_lb_pruned"] > 0.9 * st["pairs"]
    p = O.make_params("cdtw", **kw)
    rng = np.random.default_rng(7)
    for k in range(2):
        q = Qp.series(k)
        m = len(q)
        d_at = O.subseq(p, T[pos[k]:pos[k] + m], q)[1]
        assert close(float(dist[k]), d_at), (k, dist[k], d_at)
        sample = list(rng.integers(0, len(T) - m + 1, size=300)) + [int(planted[k])]
        for i in sample:
            d_i = O.subseq(p, T[i:i + m], q)[1]
            assert d_i >= float(dist[k]) * (1 - REL_TOL), (k, i, d_i, dist[k])


def test_subseq_batch_equals_single_queries(eap):
    """Queries of equal length share the window statistics inside one call:
    the batch gives each query's result alone, bit for bit."""
    T = synth.long_series(30000, 907)
    Qp, _ = synth.subseq_queries(T, [64, 64, 100, 64, 100, 33], 908, planted=True, noise=0.3)
    p = eap.params("cdtw", window_ratio=0.1)
    pos, dist = [x.cpu().numpy() for x in eap.eap_subseq(p, T, eap.SeriesSet.from_packed(Qp))]
    for k in range(6):
        one = eap.SeriesSet.from_packed(synth.pack([Qp.series(k)]))
        p1, d1 = [x.cpu().numpy() for x in eap.eap_subseq(p, T, one)]
        assert p1[0] == pos[k] and d1[0] == dist[k], (k, p1, pos[k], d1, dist[k])
