"""The 1-NN search's lower-bound pass (Alg. 2 with the lb-keogh2 cascade of
Section 5.2) through eap_lb_matrix -- the envelope and LB-matrix kernels that
eap_nn1 runs ahead of the DP -- element by element against the oracle's
textbook LB_Keogh in both directions, and never above the pair's float32 DP
value."""
import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import REL_TOL

pytestmark = pytest.mark.gpu


def _expected(qp, rp, w_of, cost, two_way):
    out = np.zeros((qp.count, rp.count))
    for a in range(qp.count):
        q = qp.series(a)
        for b in range(rp.count):
            c = rp.series(b)
            if len(q) != len(c):
                continue
            w = w_of(len(q))
            v = O.lb_keogh(q, c, w, cost)                    # LB_Keogh(Q, C): Q's envelope bounds C
            if two_way:
                v = max(v, O.lb_keogh(c, q, w, cost))        # and LB_Keogh(C, Q)
            out[a, b] = v * (1.0 - (4 * len(q) + 16) * 2.0 ** -24)
    return out


@pytest.mark.parametrize("kind,window", [("cdtw", 0), ("cdtw", 3), ("cdtw", 51), ("cdtw", 200), ("dtw", None)])
@pytest.mark.parametrize("cost", [0, 1])
@pytest.mark.parametrize("two_way", [False, True])
def test_lb_matrix_matches_oracle(kind, window, cost, two_way):
    from paper_2102_05221_gb300 import eap
    rng = np.random.default_rng(600 + (window or 999) + 7 * cost)
    qlen = [300] * 9 + [150, 301, 300]
    rlen = [300] * 30 + [150] * 4 + [299, 300, 301] + [300] * 30
    qp = synth.ragged_walks(len(qlen), qlen, 611 + cost, n_classes=3)
    rp = synth.ragged_walks(len(rlen), rlen, 612 + cost, n_classes=3)
    Q, R = eap.SeriesSet.from_packed(qp), eap.SeriesSet.from_packed(rp)
    if kind == "cdtw":
        p = eap.params("cdtw", window=window, window_ratio=-1.0, cost=cost)
        w_of = lambda L: window
    else:
        p = eap.params("dtw", cost=cost)
        w_of = lambda L: L                                    # DTW: the whole series
    got = eap.eap_lb_matrix(p, Q, R, two_way=two_way).cpu().numpy().astype(np.float64)
    want = _expected(qp, rp, w_of, cost, two_way)
    zero = want == 0
    assert np.all(got[zero] == 0) or np.all(got[zero] <= 1e-6), (kind, window, cost)
    rel = np.abs(got - want) / np.maximum(want, 1e-30)
    assert np.all(rel[~zero] <= REL_TOL), (kind, window, cost, two_way, float(rel[~zero].max()))
    # A lower bound of the float32 DP value of every equal-length pair.
    ia, ib = np.nonzero(np.ones_like(got, dtype=bool))
    ia, ib = ia.astype(np.int32), ib.astype(np.int32)
    pd = eap.params(kind, cost=cost, prune=0, **({"window": window, "window_ratio": -1.0} if kind == "cdtw" else {}))
    d = eap.eap_pairs(pd, Q, R, ia, ib).cpu().numpy().reshape(got.shape)
    fin = np.isfinite(d)
    assert np.all(got[fin] <= d[fin]), (kind, window, cost)


def test_lb_matrix_long_series_use_the_scanning_envelope():
    """4000 points need 64 KB for the O(L) envelope's running extrema; those
    series take the scanning form, with the same bounds."""
    from paper_2102_05221_gb300 import eap
    qp = synth.ragged_walks(3, [4000] * 3, 621, n_classes=2)
    rp = synth.ragged_walks(5, [4000] * 5, 622, n_classes=2)
    Q, R = eap.SeriesSet.from_packed(qp), eap.SeriesSet.from_packed(rp)
    p = eap.params("cdtw", window=400, window_ratio=-1.0)
    got = eap.eap_lb_matrix(p, Q, R).cpu().numpy().astype(np.float64)
    want = _expected(qp, rp, lambda L: 400, 0, True)
    assert np.all(np.abs(got - want) <= REL_TOL * np.maximum(want, 1e-30))


def test_lb_matrix_rejects_other_distances():
    from paper_2102_05221_gb300 import eap
    s = eap.SeriesSet.from_packed(synth.ragged_walks(2, [16, 16], 1))
    with pytest.raises(eap.EapError):
        eap.eap_lb_matrix(eap.params("msm"), s, s)
