"""Pins of the FP64 oracle against what the paper and mathematics fix (CPU only).

Each test ties the oracle to something other than itself: the paper's worked
example (Fig. DTW, Section 4.2), brute-force enumeration of every alignment
path, closed forms, and invariants the paper states (Section 2.3, Section 4).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import brute
from paper_2102_05221_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KINDS = ["dtw", "cdtw", "wdtw", "erp", "msm", "twe"]


def _read_golden(name):
    rows = {}
    extra = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "EAPRUNED_CUTOFF":
                extra.append((float(parts[1]), float(parts[3]), int(parts[5])))
            elif parts[0] == "EABASE_CUTOFF":
                rows.setdefault("EABASE", []).append((float(parts[1]), float(parts[3]), int(parts[5])))
            else:
                rows[parts[0]] = [float(x) for x in parts[1:]]
    return rows, extra


def test_worked_example_dtw_is_9_and_pins_squared_cost():
    g, _ = _read_golden("dtw_worked_example.txt")
    S, T = g["S"], g["T"]
    assert O.distance(O.make_params("dtw"), S, T) == g["DTW"][0]
    # The absolute-difference cost would give 7, so the figure fixes the squared cost.
    assert O.distance(O.make_params("dtw", cost=O.COST_ABS), S, T) == 7.0
    # CDTW with a full window is DTW (Section 2.3.2).
    assert O.distance(O.make_params("cdtw", window=6), S, T) == 9.0


def test_worked_example_eapruned_cell_counts():
    g, runs = _read_golden("dtw_worked_example.txt")
    S, T = g["S"], g["T"]
    for cutoff, result, cells in runs:
        d, n = O.eapruned(O.make_params("dtw"), S, T, cutoff)
        assert n == cells, (cutoff, n)
        assert d == result
    # With no cut-off nothing is pruned: all 36 cells are computed.
    d, n = O.eapruned(O.make_params("dtw"), S, T, math.inf)
    assert (d, n) == (9.0, 36)


def test_cdtw_infeasible_window_is_inf():
    g, _ = _read_golden("cdtw_infeasible_window.txt")
    p = O.make_params("cdtw", window=int(g["W"][0]))
    assert O.distance(p, g["S"], g["U"]) == math.inf
    assert O.eapruned(p, g["S"], g["U"], math.inf)[0] == math.inf
    # One more unit of window makes (6,8) reachable.
    assert math.isfinite(O.distance(O.make_params("cdtw", window=2), g["S"], g["U"]))


def _bf_kwargs(kind, window):
    kw = {}
    if kind in ("cdtw", "erp"):
        kw["window"] = window
    return kw


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("cost", [0, 1])
def test_oracle_equals_bruteforce_on_tiny_series(kind, cost):
    """Exact FP64 equality with the minimum over every alignment path."""
    rng = np.random.default_rng(11 + 7 * KINDS.index(kind) + cost)
    cases = [(1, 1), (1, 4), (4, 1), (2, 3), (5, 5), (4, 6), (6, 4), (6, 6)]
    for ls, lt in cases:
        s = rng.uniform(-2, 2, ls).astype(np.float32)
        t = rng.uniform(-2, 2, lt).astype(np.float32)
        windows = [None] if kind not in ("cdtw", "erp") else [None, 0, 1, 2, 3]
        for w in windows:
            p = O.make_params(kind, cost=cost, window=-1 if w is None else w,
                              erp_gap=0.3, msm_c=0.5, twe_nu=0.25, twe_lambda=0.5, wdtw_g=0.4)
            got = O.distance(p, s, t)
            bf = brute.brute_distance(kind, s, t, cost, gap=float(np.float32(0.3)),
                                      msm_c=0.5, nu=0.25, lam=0.5, g=float(np.float32(0.4)),
                                      **_bf_kwargs(kind, w))
            assert got == bf, (kind, cost, ls, lt, w, got, bf)


def test_bruteforce_enumerates_delannoy_many_paths():
    for m, n in [(1, 1), (2, 3), (4, 4), (5, 6)]:
        assert sum(1 for _ in brute.all_paths(m, n)) == brute.delannoy(m, n)
    assert brute.delannoy(7, 7) == 48639


def _walks(n, L, seed):
    return synth.random_walks(np.random.default_rng(seed), n, L).astype(np.float32)


def test_cdtw_window_zero_is_squared_euclidean():
    x = _walks(6, 40, 1)
    for a in range(3):
        s, t = x[a], x[a + 3]
        sq = 0.0
        for i in range(len(s)):
            d = float(s[i]) - float(t[i])
            sq = sq + d * d
        assert O.distance(O.make_params("cdtw", window=0), s, t) == sq


def test_cdtw_full_window_is_dtw():
    x = _walks(6, 33, 2)
    for a in range(3):
        s, t = x[a], x[a + 3]
        d = O.distance(O.make_params("dtw"), s, t)
        for w in (33, 40, 1000):
            assert O.distance(O.make_params("cdtw", window=w), s, t) == d
        # And the window only ever raises the cost.
        assert O.distance(O.make_params("cdtw", window=3), s, t) >= d


def test_wdtw_with_g_zero_is_half_dtw():
    # g = 0 makes every weight wmax / 2 (Eq. WDTW); with wmax = 1 the factor
    # 1/2 is exact in binary floating point.
    x = _walks(4, 30, 3)
    for a in range(2):
        s, t = x[a], x[a + 2]
        assert O.distance(O.make_params("wdtw", wdtw_g=0.0), s, t) == 0.5 * O.distance(O.make_params("dtw"), s, t)


def test_erp_against_constant_gap_series_is_l1_to_gap():
    # Against a series made only of the gap value, matching s_i with g and
    # deleting s_i both cost |s_i - g| and deleting g costs 0, so every path
    # costs sum_i |s_i - g| in the same order (Eq. ERP).
    g = np.float32(0.25)
    x = _walks(3, 17, 4)
    for s in x:
        ref = 0.0
        for v in s:
            ref = ref + abs(float(v) - float(g))
        for m in (1, 5, 17, 30):
            t = np.full(m, g, dtype=np.float32)
            assert O.distance(O.make_params("erp", erp_gap=float(g)), s, t) == ref


def test_msm_split_and_move_semantics():
    # Eq. MSM: one split of x into (x, x) costs c; splitting 0 and moving the
    # copy to 5 costs c + 5; a single move costs |a - b|.
    c = 0.5
    p = O.make_params("msm", msm_c=c)
    assert O.distance(p, [1.5], [1.5, 1.5]) == c
    assert O.distance(p, [1.5], [1.5] * 5) == 4 * c
    assert O.distance(p, [0.0], [0.0, 5.0]) == c + 5.0
    assert O.distance(p, [2.0], [-1.0]) == 3.0
    # A merge is the mirror of a split.
    assert O.distance(p, [0.0, 5.0], [0.0]) == c + 5.0


def test_twe_single_points_and_deletion_cost():
    # Eq. TWE on one point each: the match (1,1) costs cost(s1,t1) + cost(s0,t0) = |a-b|.
    p = O.make_params("twe", twe_nu=0.25, twe_lambda=0.5)
    assert O.distance(p, [2.0], [-1.0]) == 3.0
    # (a) vs (a, a): one deleteB of the repeated point: |a - a| + nu + lambda.
    nu, lam = float(np.float32(0.25)), float(np.float32(0.5))
    assert O.distance(p, [1.0], [1.0, 1.0]) == 0.0 + nu * 1.0 + lam


@pytest.mark.parametrize("kind", KINDS)
def test_identity_and_symmetry(kind):
    x = synth.ragged_walks(8, [7, 19, 33, 33, 50, 12, 64, 40], 5)
    p = O.make_params(kind, window_ratio=0.3 if kind in ("cdtw", "erp") else -1)
    for i in range(x.count):
        assert O.distance(p, x.series(i), x.series(i)) == 0.0
    for i in range(x.count):
        for j in range(i + 1, x.count):
            a = O.distance(p, x.series(i), x.series(j))
            b = O.distance(p, x.series(j), x.series(i))
            if math.isinf(a) or math.isinf(b):
                assert a == b
            else:
                assert abs(a - b) <= 1e-12 * max(1.0, abs(a)), (kind, i, j, a, b)


@pytest.mark.parametrize("kind", ["msm", "twe", "erp"])
def test_triangle_inequality_of_the_metrics(kind):
    # MSM (Section 2.3.5), TWE with L1 cost, and ERP with L1 cost and no
    # window (Section 2.3.4) are metrics.
    x = synth.ragged_walks(9, [10, 14, 9, 20, 16, 11, 25, 8, 13], 6)
    p = O.make_params(kind)
    n = x.count
    D = [[O.distance(p, x.series(i), x.series(j)) for j in range(n)] for i in range(n)]
    for a in range(n):
        for b in range(n):
            for c in range(n):
                assert D[a][c] <= D[a][b] + D[b][c] + 1e-9, (kind, a, b, c)


def test_dtw_is_not_a_metric_but_msm_is_translation_invariant():
    s = _walks(2, 24, 8)
    p = O.make_params("msm")
    a = O.distance(p, s[0], s[1])
    b = O.distance(p, s[0] + np.float32(3.0), s[1] + np.float32(3.0))
    assert abs(a - b) <= 1e-5 * a


def test_scaling_laws():
    # Scaling both series by k scales the squared-cost DTW by k^2 and the
    # L1 ERP (gap 0) by |k|; powers of two keep this exact.
    x = _walks(2, 20, 9)
    s, t = x[0], x[1]
    k = np.float32(4.0)
    assert O.distance(O.make_params("dtw"), s * k, t * k) == 16.0 * O.distance(O.make_params("dtw"), s, t)
    assert O.distance(O.make_params("erp", erp_gap=0.0), s * k, t * k) == 4.0 * O.distance(O.make_params("erp", erp_gap=0.0), s, t)


KIND_EA = ["dtw", "cdtw", "wdtw", "erp", "msm", "twe"]


@pytest.mark.parametrize("kind", KIND_EA)
def test_eapruned_returns_inf_exactly_when_distance_exceeds_cutoff(kind):
    """Algorithm 5 returns D when D <= cut-off and +inf otherwise (Section 2.2,
    Section 4.3), for cut-offs on both sides of D."""
    x = synth.ragged_walks(10, [30, 30, 42, 25, 30, 55, 30, 31, 29, 44], 10)
    p = O.make_params(kind, window_ratio=0.2 if kind in ("cdtw", "erp") else -1)
    for i in range(0, x.count, 2):
        s, t = x.series(i), x.series(i + 1)
        d = O.distance(p, s, t)
        for cut in [d, d * (1 + 1e-9), d * (1 - 1e-9), 0.0, math.inf, 2 * d, 0.5 * d]:
            got, cells = O.eapruned(p, s, t, cut)
            if math.isinf(d):
                assert math.isinf(got)
            elif d <= cut:
                assert abs(got - d) <= 1e-12 * max(1.0, d), (kind, i, cut, got, d)
            else:
                assert math.isinf(got), (kind, i, cut, got, d)
            assert 0 <= cells <= len(s) * len(t)


def test_eapruned_complexity_depends_on_candidate_order():
    # Section 4.3.1: nearest-first ordering leaves later candidates almost free;
    # furthest-first computes (almost) everything.
    ds = synth.make_dataset(20, 1, 64, 3, 123)
    q = ds.test[0]
    p = O.make_params("dtw")
    dists = [O.distance(p, q, c) for c in ds.train]
    order = np.argsort(dists)

    def run(seq):
        dnn, total = math.inf, 0
        for c in seq:
            d, n = O.eapruned(p, q, ds.train[c], dnn)
            total += n
            if d < dnn:
                dnn = d
        return dnn, total

    best_near, cells_near = run(order)
    best_far, cells_far = run(order[::-1])
    assert best_near == best_far == min(dists)
    assert cells_near * 3 < cells_far


def test_nn1_and_pairwise_match_distance():
    ds = synth.make_dataset(12, 5, 20, 3, 77)
    tr, te = synth.pack(ds.train), synth.pack(ds.test)
    p = O.make_params("dtw")
    idx, dist = O.nn1(p, te, tr, nthreads=2)
    for q in range(te.count):
        ds_ = [O.distance(p, te.series(q), tr.series(c)) for c in range(tr.count)]
        best = min(range(len(ds_)), key=lambda c: (ds_[c], c))
        assert idx[q] == best and dist[q] == ds_[best]
    M = O.pairwise(p, tr, nthreads=3)
    assert M.shape == (12, 12)
    for i in range(12):
        assert M[i, i] == 0.0
        for j in range(12):
            assert M[i, j] == O.distance(p, tr.series(i), tr.series(j))


@pytest.mark.parametrize("kind", KINDS)
def test_nn1_eapruned_equals_plain_nn1(kind):
    # The paper's exactness claim (Section 5): every implementation of a
    # distance gives the same NN result.  Alg. 1 driving Alg. 5 with the
    # best-so-far as cut-off must return the plain search's index (lowest on
    # ties) and distance, bit for bit in FP64, while computing fewer cells
    # than the full matrices.  Ragged lengths, and exact duplicates of the
    # query among the candidates, exercise the tie and the zero-distance case.
    rng = np.random.default_rng(31 + KINDS.index(kind))
    refs = [synth.random_walks(rng, 1, int(n))[0].astype(np.float32) for n in rng.integers(18, 30, size=14)]
    qs = [synth.random_walks(rng, 1, int(n))[0].astype(np.float32) for n in rng.integers(18, 30, size=5)]
    refs[9] = qs[2].copy()
    refs[11] = qs[2].copy()
    kw = {"window_ratio": 0.3} if kind in ("cdtw", "erp") else {}
    p = O.make_params(kind, **kw)
    tr, te = synth.pack(refs), synth.pack(qs)
    idx, dist = O.nn1(p, te, tr, nthreads=1)
    idx2, dist2, cells = O.nn1_eapruned(p, te, tr)
    assert list(idx2) == list(idx)
    assert list(dist2) == list(dist)
    assert idx[2] == 9 and dist[2] == 0.0
    full = sum(len(q) * len(r) for q in qs for r in refs)
    assert 0 < cells < full


def test_nn1_ties_go_to_lowest_index_and_empty_is_minus_one():
    p = O.make_params("dtw")
    q = synth.pack([np.array([0.0, 1.0, 2.0], np.float32)])
    refs = synth.pack([np.array([5.0, 5.0], np.float32), np.array([0.0, 1.0, 2.0], np.float32),
                       np.array([0.0, 1.0, 2.0], np.float32)])
    idx, dist = O.nn1(p, q, refs, nthreads=1)
    assert idx[0] == 1 and dist[0] == 0.0
    # With a window too small for every candidate, nothing is found (Alg. 1 returns (inf, none)).
    pc = O.make_params("cdtw", window=0)
    refs2 = synth.pack([np.zeros(5, np.float32), np.zeros(7, np.float32)])
    idx, dist = O.nn1(pc, q, refs2, nthreads=1)
    assert idx[0] == -1 and math.isinf(dist[0])


def test_lb_keogh_bounds_cdtw_and_equals_sqed_at_window_zero():
    x = _walks(8, 50, 12)
    for a in range(4):
        q, c = x[a], x[a + 4]
        for w in (0, 2, 5, 50):
            lb = O.lb_keogh(q, c, w)
            d = O.distance(O.make_params("cdtw", window=w), q, c)
            assert lb <= d + 1e-12
        sq = O.distance(O.make_params("cdtw", window=0), q, c)
        assert abs(O.lb_keogh(q, c, 0) - sq) <= 1e-12 * sq
        U, L = O.envelope(q, 3)
        for i in range(len(q)):
            win = q[max(0, i - 3): i + 4].astype(np.float64)
            assert U[i] == win.max() and L[i] == win.min()


def test_window_ratio_reading():
    # w = floor(r * max(L_S, L_T)): 10% of 512 is 51.
    s = _walks(2, 512, 13)
    d51 = O.distance(O.make_params("cdtw", window=51), s[0], s[1])
    assert O.distance(O.make_params("cdtw", window_ratio=0.1), s[0], s[1]) == d51


def test_twe_match_cost_uses_previous_points():
    # Hand evaluation of Eq. TWECost/Eq. TWE on S = (1, 2), T = (3, 2), L1 cost:
    #   M(1,1) = |1-3| + |0-0| = 2
    #   M(2,2) = min(M(1,1) + |2-2| + |1-3| + 0,           (match: 4)
    #                M(1,2) + gamma_A = 3+nu+lam + 1+nu+lam, (deleteA)
    #                M(2,1) + gamma_B = 3+nu+lam + 1+nu+lam) (deleteB)
    # so TWE = 4; dropping the cost(s_{i-1}, t_{j-1}) term would give 2.
    p = O.make_params("twe", twe_nu=0.25, twe_lambda=0.5)
    assert O.distance(p, [1.0, 2.0], [3.0, 2.0]) == 4.0
    assert brute.brute_distance("twe", [1.0, 2.0], [3.0, 2.0], 1, nu=0.25, lam=0.5) == 4.0


def test_msm_hand_evaluated_example():
    # Eq. MSM on S = (0, 3), T = (1, 2), c = 0.5:
    #   M(1,1) = 1, M(1,2) = 1 + (0.5 + 1) = 2.5, M(2,1) = 1 + (0.5 + 2) = 3.5,
    #   M(2,2) = min(1 + |3-2|, 2.5 + (0.5 + 1), 3.5 + 0.5) = 2.
    p = O.make_params("msm", msm_c=0.5)
    assert O.distance(p, [0.0, 3.0], [1.0, 2.0]) == 2.0
    assert O.distance(p, [0.0, 3.0], [1.0]) == 1.0 + 0.5 + 2.0


# ---------------------------------------------------------------------------
# Derivative distances (Section 2.3: DDTW and the other derivative variants
# apply the distance to the first-derivative series, after Keogh & Pazzani).

def test_derivative_hand_values():
    # x = 0 1 3 6: interior estimates ((1-0) + (3-0)/2)/2 = 1.25 and
    # ((3-1) + (6-1)/2)/2 = 2.25; the ends copy them.  Against a constant series
    # (derivative 0) every alignment covers each row, so the diagonal is optimal.
    x = [0.0, 1.0, 3.0, 6.0]
    z = [5.0, 5.0, 5.0, 5.0]
    assert O.distance(O.make_params("dtw", derivative=1), x, z) == 2 * 1.25 ** 2 + 2 * 2.25 ** 2
    assert O.distance(O.make_params("dtw", cost=O.COST_ABS, derivative=1), x, z) == 7.0
    # Without the derivative the same pair is far apart.
    assert O.distance(O.make_params("dtw"), x, z) != 13.25


@pytest.mark.parametrize("kind,cost,expect", [("dtw", 0, 16 * 0.0625), ("cdtw", 0, 16 * 0.0625),
                                              ("erp", 1, 16 * 0.25), ("twe", 1, 0.25 + 15 * 0.5)])
def test_derivative_of_lines_is_constant_slope(kind, cost, expect):
    # Lines of slope 1/2 and 1/4 have constant derivatives 1/2 and 1/4.
    # DTW/CDTW: 16 diagonal cells of (1/4)^2.  ERP (gap 0): 16 matches of 1/4
    # beat 32 gap steps.  TWE (nu, lambda large): the diagonal costs
    # |1/2-1/4| + |0-0| on the first step and 2 * 1/4 on each later one.
    x = [0.5 * i for i in range(16)]
    y = [0.25 * i - 3.0 for i in range(16)]
    p = O.make_params(kind, cost=cost, window=0 if kind == "cdtw" else -1, erp_gap=0.0,
                      twe_nu=1.0, twe_lambda=1.0, derivative=1)
    assert O.distance(p, x, y) == expect


def test_derivative_of_one_or_two_points_is_zero():
    rng = np.random.default_rng(5)
    for kind in KINDS:
        # Unequal lengths need a split (MSM) or a deletion (TWE), which costs even on zeros.
        for la, lb in [(1, 1), (2, 2)] + ([(1, 2)] if kind not in ("msm", "twe") else []):
            a = rng.normal(size=la).astype(np.float32)
            b = rng.normal(size=lb).astype(np.float32)
            assert O.distance(O.make_params(kind, derivative=1, erp_gap=0.0), a, b) == 0.0


@pytest.mark.parametrize("kind", KINDS)
def test_derivative_distance_ignores_offsets(kind):
    # Values on a 1/8 grid keep x + 3 exact in float32, so the derivatives agree exactly.
    rng = np.random.default_rng(17 + KINDS.index(kind))
    for L in (3, 9, 40):
        x = (rng.integers(-16, 16, L) / 8.0).astype(np.float32)
        assert O.distance(O.make_params(kind, derivative=1), x, x + np.float32(3.0)) == 0.0
        assert O.eapruned(O.make_params(kind, derivative=1), x, x + np.float32(3.0), 0.0)[0] == 0.0


def _keogh_pazzani(x):
    x = [float(v) for v in x]
    n = len(x)
    if n <= 2:
        return [0.0] * n
    d = [0.0] * n
    for i in range(1, n - 1):
        d[i] = ((x[i] - x[i - 1]) + (x[i + 1] - x[i - 1]) / 2.0) / 2.0
    d[0], d[-1] = d[1], d[-2]
    return d


@pytest.mark.parametrize("kind", KINDS)
def test_derivative_oracle_equals_bruteforce(kind):
    """The derivative variant is the brute-force minimum over paths of the derivative series."""
    rng = np.random.default_rng(40 + KINDS.index(kind))
    cost = 0 if kind in ("dtw", "cdtw", "wdtw") else 1
    for ls, lt in [(3, 3), (4, 6), (6, 4), (6, 6)]:
        s = rng.uniform(-2, 2, ls).astype(np.float32)
        t = rng.uniform(-2, 2, lt).astype(np.float32)
        windows = [None] if kind not in ("cdtw", "erp") else [None, 1, 2]
        for w in windows:
            p = O.make_params(kind, cost=cost, window=-1 if w is None else w, erp_gap=0.3,
                              msm_c=0.5, twe_nu=0.25, twe_lambda=0.5, wdtw_g=0.4, derivative=1)
            bf = brute.brute_distance(kind, _keogh_pazzani(s), _keogh_pazzani(t), cost,
                                      gap=float(np.float32(0.3)), msm_c=0.5, nu=0.25, lam=0.5,
                                      g=float(np.float32(0.4)), **_bf_kwargs(kind, w))
            assert O.distance(p, s, t) == bf, (kind, ls, lt, w)
            # Alg. 5 on the derivative series: exact at cut-off D, +inf below it.
            if math.isfinite(bf):
                assert O.eapruned(p, s, t, bf)[0] == bf
                assert O.eapruned(p, s, t, bf * 0.999)[0] == math.inf


# ---------------------------------------------------------------------------
# Algorithm 4 (EABase: Base with the usual early abandoning on the row minimum).

def test_eabase_worked_example_cell_counts():
    g, _ = _read_golden("dtw_worked_example.txt")
    S, T = g["S"], g["T"]
    for cutoff, result, cells in g["EABASE"]:
        d, n = O.eabase(O.make_params("dtw"), S, T, cutoff)
        assert (d, n) == (result, cells), (cutoff, d, n)
    assert O.eabase(O.make_params("dtw"), S, T, math.inf) == (9.0, 36)


@pytest.mark.parametrize("kind", KINDS)
def test_eabase_contract_and_bruteforce(kind):
    """D exactly when D <= cut-off; when D > cut-off, D or +inf; and the
    brute-force minimum over paths when no cut-off is given."""
    rng = np.random.default_rng(70 + KINDS.index(kind))
    cost = 0 if kind in ("dtw", "cdtw", "wdtw") else 1
    for ls, lt in [(1, 1), (3, 5), (5, 3), (6, 6)]:
        s = rng.uniform(-2, 2, ls).astype(np.float32)
        t = rng.uniform(-2, 2, lt).astype(np.float32)
        for w in ([None] if kind not in ("cdtw", "erp") else [None, 1, 2]):
            p = O.make_params(kind, cost=cost, window=-1 if w is None else w, erp_gap=0.3,
                              msm_c=0.5, twe_nu=0.25, twe_lambda=0.5, wdtw_g=0.4)
            bf = brute.brute_distance(kind, s, t, cost, gap=float(np.float32(0.3)), msm_c=0.5, nu=0.25,
                                      lam=0.5, g=float(np.float32(0.4)), **_bf_kwargs(kind, w))
            assert O.eabase(p, s, t, math.inf)[0] == bf
            if not math.isfinite(bf):
                continue
            for cut in (bf, bf * 1.5, bf * 0.999, bf * 0.5, 0.0):
                d, _ = O.eabase(p, s, t, cut)
                if bf <= cut:
                    assert d == bf, (kind, ls, lt, w, cut, d, bf)
                else:
                    assert d == bf or d == math.inf, (kind, ls, lt, w, cut, d, bf)


def test_eabase_abandons_on_a_row_above_the_cutoff():
    # A cut-off below every cell of the first row abandons after that row;
    # rows never exceed L_co cells.
    x = _walks(2, 50, 9)
    s, t = x[0], x[1] + np.float32(10.0)
    d, n = O.eabase(O.make_params("dtw"), s, t, 1.0)
    assert d == math.inf and n == 50
    # A cut-off at D never abandons and computes the whole matrix.
    D = O.distance(O.make_params("dtw"), s, t)
    assert O.eabase(O.make_params("dtw"), s, t, D) == (D, 2500)


def test_eabase_erp_row_minimum_includes_the_vertical_border():
    # S = (0, 0, 0, 5), T = (5), gap 0: the optimal path runs down the border
    # (cost 0) and matches 5 with 5 last, so ERP = 0, while the first row's
    # only interior cell costs 5.  A row minimum without the border cell would
    # abandon this pair at cut-off 4.
    p = O.make_params("erp", cost=O.COST_ABS, erp_gap=0.0)
    s, t = [0.0, 0.0, 0.0, 5.0], [5.0]
    assert O.distance(p, s, t) == 0.0
    assert O.eabase(p, s, t, 4.0)[0] == 0.0
    assert O.eapruned(p, s, t, 4.0)[0] == 0.0


# ---------------------------------------------------------------------------
# Sub-sequence search (Section 5.3): z-normalised windows of a long series.

def _znorm_np(x):
    x = np.asarray(x, dtype=np.float64)
    mu = x.mean()
    sd = np.sqrt(((x - mu) ** 2).mean())
    return (x - mu) / sd if sd > 1e-8 else np.zeros_like(x)


def test_subseq_finds_a_planted_copy_and_ignores_scale_and_offset():
    T = _walks(1, 4000, 21)[0]
    q = T[1717:1717 + 96].copy()
    p = O.make_params("cdtw", window_ratio=0.1)
    assert O.subseq(p, T, q) == (1717, 0.0)
    pos, d = O.subseq(p, T, (q * np.float32(2.5) - np.float32(4.0)).astype(np.float32))
    assert pos == 1717 and d < 1e-9


def test_subseq_window_zero_is_znormalised_euclidean_search():
    T = _walks(1, 1500, 22)[0]
    q = _walks(1, 40, 23)[0]
    win = np.lib.stride_tricks.sliding_window_view(T.astype(np.float64), 40)
    zq = _znorm_np(q)
    ed = np.array([((zq - _znorm_np(w)) ** 2).sum() for w in win])
    pos, d = O.subseq(O.make_params("cdtw", window=0), T, q)
    assert pos == int(np.argmin(ed))
    assert abs(d - ed.min()) <= 1e-12 * ed.min()


def test_subseq_equals_bruteforce_paths_on_tiny_series():
    rng = np.random.default_rng(24)
    for kind, kw in [("dtw", {}), ("cdtw", {"window": 1})]:
        T = rng.uniform(-2, 2, 14).astype(np.float32)
        q = rng.uniform(-2, 2, 4).astype(np.float32)
        zq = list(_znorm_np(q))
        d_bf = [brute.brute_distance(kind, zq, list(_znorm_np(T[i:i + 4])), 0, **kw) for i in range(11)]
        pos, d = O.subseq(O.make_params(kind, **kw), T, q)
        assert pos == int(np.argmin(d_bf))
        assert abs(d - min(d_bf)) <= 1e-12 * max(1.0, min(d_bf))


def test_subseq_edge_cases():
    p = O.make_params("dtw")
    T = _walks(1, 50, 25)[0]
    assert O.subseq(p, T[:10], T[:11]) == (-1, math.inf)     # query longer than the series
    assert O.subseq(p, T[:10], T[:10]) == (0, 0.0)           # one position
    flat = np.concatenate([T[:20], np.full(12, 3.0, np.float32), T[20:]]).astype(np.float32)
    pos, d = O.subseq(p, flat, np.full(12, -1.0, np.float32))
    assert pos == 20 and d == 0.0                             # constant windows normalise to zeros
