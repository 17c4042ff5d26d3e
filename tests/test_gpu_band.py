"""Base DP of the windowed distances (CDTW, ERP) in band coordinates
(band_dp_kernel): bit-identical to the column-panel kernels (the band
mapping forced with EAP_BAND=2, switched off with EAP_BAND=0) and within
tolerance of the FP64
oracle, on ragged lengths, windows at and around every built band width,
the degenerate windows (w = 0, w = |L_A - L_B|) and the three entry points
that run the Base DP (pairs, 1-NN with prune = 0, all-pairs matrix)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import close, check_nn, gpu_params, oracle_params

pytestmark = pytest.mark.gpu

# A band row is 2w + 2 positions (the window and the cell left of it).  The
# padded launches hold 32, 64, 112, 128 and 256 positions and need 2w + 3;
# the exact launches hold 2w + 2 = 104 (w = 51: 8 lanes x 13, 4 lanes x 26).
BAND_WINDOWS = [0, 1, 2, 14, 15, 30, 31, 50, 51, 54, 55, 62, 63, 126, 127]


@pytest.fixture(scope="module")
def eap():
    from paper_2102_05221_gb300 import eap as E
    E.load()
    return E


def _run(fn, band, **env):
    """Runs fn with the band mapping forced (EAP_BAND=2: whenever the band
    fits a launch, even where the default keeps the panel kernels) or off,
    and any other EAP_* variables given (EAP_BAND_G, EAP_BAND_EXACT)."""
    env = dict(env, EAP_BAND="2" if band else "0")
    old = {k: os.environ.get(k) for k in env}
    os.environ.update({k: str(v) for k, v in env.items()})
    try:
        return fn()
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


@pytest.mark.parametrize("kind", ["cdtw", "erp"])
@pytest.mark.parametrize("cost", [0, 1])
@pytest.mark.parametrize("w", BAND_WINDOWS)
def test_band_pairs_match_panels_and_oracle(eap, kind, cost, w):
    rng = np.random.default_rng(7000 + 31 * w + cost + (kind == "erp") * 1000)
    L = max(2 * w + 3, 40)
    # Equal lengths, lengths differing by up to w, and a few short series.
    la = [L, L, L + 1, L + w, max(1, L - w), L + 3 if w >= 3 else L, 2 * w + 3, 1 if w >= 1 else L]
    lb = [L, L + w, L, L, L, L, 2 * w + 3, 2 if w >= 1 else L]
    Ap = synth.ragged_walks(len(la), la, 900 + w, n_classes=2)
    Bp = synth.ragged_walks(len(lb), lb, 901 + w, n_classes=2)
    A, B = eap.SeriesSet.from_packed(Ap), eap.SeriesSet.from_packed(Bp)
    kw = {"window": w, "cost": cost}
    if kind == "erp":
        kw["erp_gap"] = float(np.float32(rng.uniform(-0.5, 0.5)))
    p = gpu_params(eap, kind, prune=0, **kw)
    ia = np.repeat(np.arange(len(la)), len(lb)).astype(np.int32)
    ib = np.tile(np.arange(len(lb)), len(la)).astype(np.int32)
    got_band, st = _run(lambda: eap.eap_pairs(p, A, B, ia, ib, with_stats=True), True)
    got_panel = _run(lambda: eap.eap_pairs(p, A, B, ia, ib), False)
    got_band = got_band.cpu().numpy()
    got_panel = got_panel.cpu().numpy()
    assert np.array_equal(got_band, got_panel), (kind, cost, w, np.flatnonzero(got_band != got_panel)[:5])
    D = O.cross(oracle_params(kind, **kw), Ap, Bp)
    for k in range(len(ia)):
        d = float(D[ia[k], ib[k]])
        if np.isinf(d):
            assert np.isinf(got_band[k]), (kind, cost, w, k)
        else:
            assert close(float(got_band[k]), d), (kind, cost, w, k, got_band[k], d)
    assert st["pairs"] == len(ia)


@pytest.mark.parametrize("kind", ["cdtw", "erp"])
def test_band_nn1_base_matches_panels(eap, kind):
    rng = np.random.default_rng(77 + (kind == "erp"))
    qlen = list(rng.integers(100, 140, size=12))
    rlen = list(rng.integers(100, 140, size=50))
    Qp = synth.ragged_walks(len(qlen), qlen, 311, n_classes=3)
    Rp = synth.ragged_walks(len(rlen), rlen, 312, n_classes=3)
    Q, R = eap.SeriesSet.from_packed(Qp), eap.SeriesSet.from_packed(Rp)
    kw = {"window_ratio": 0.15}
    p = gpu_params(eap, kind, prune=0, **kw)
    i1, d1 = _run(lambda: eap.eap_nn1(p, Q, R), True)
    i0, d0 = _run(lambda: eap.eap_nn1(p, Q, R), False)
    assert np.array_equal(i1.cpu().numpy(), i0.cpu().numpy())
    assert np.array_equal(d1.cpu().numpy(), d0.cpu().numpy())
    D = O.cross(oracle_params(kind, **kw), Qp, Rp)
    check_nn(i1.cpu().numpy(), d1.cpu().numpy(), D)


@pytest.mark.parametrize("kind", ["cdtw", "erp"])
def test_band_pairwise_base_matches_panels(eap, kind):
    x = synth.random_walks(np.random.default_rng(5), 24, 300).astype(np.float32)
    S = eap.SeriesSet.from_matrix(x)
    p = gpu_params(eap, kind, window=20, cost=1 if kind == "erp" else 0)
    m1 = _run(lambda: eap.eap_pairwise(p, S, mode=eap.EAP_BASE), True).cpu().numpy()
    m0 = _run(lambda: eap.eap_pairwise(p, S, mode=eap.EAP_BASE), False).cpu().numpy()
    assert np.array_equal(m1, m0)


def test_band_cells_and_workload_sample(eap):
    """1000 x 1000 x 512 CDTW (w = 51, the exact 8 x 13 launch): 2w + 1 = 103
    window positions counted per series row, and sampled 1-NN equal to the
    oracle."""
    ds = synth.workload_nn1_512()
    tr, te = synth.pack(ds.train), synth.pack(ds.test)
    R, Q = eap.SeriesSet.from_packed(tr), eap.SeriesSet.from_packed(te)
    p = gpu_params(eap, "cdtw", prune=0, window_ratio=0.1)
    idx, dist, st = eap.eap_nn1(p, Q, R, with_stats=True)
    assert st["pairs"] == 1000 * 1000
    assert st["cells_computed"] == 1000 * 1000 * 512 * 103
    rows = list(np.random.default_rng(11).choice(1000, size=6, replace=False))
    D = O.cross(oracle_params("cdtw", window_ratio=0.1), synth.pack([ds.test[r] for r in rows]), tr)
    check_nn(idx.cpu().numpy(), dist.cpu().numpy(), D, rows=rows)


@pytest.mark.parametrize("kind", ["cdtw", "erp"])
@pytest.mark.parametrize("w", [0, 3, 30, 54, 126])
def test_band_eapruned_pairs_contract(eap, kind, w):
    """Explicit cut-offs: D exactly when D <= cut-off, +inf above, and the
    same outputs as the column-panel EAPruned kernel."""
    rng = np.random.default_rng(4100 + w + (kind == "erp") * 500)
    L = max(2 * w + 3, 48)
    la = [L, L, L + w, max(1, L - w), L + 1, 2 * w + 3]
    lb = [L, L + w, L, L, L, 2 * w + 3]
    Ap = synth.ragged_walks(len(la), la, 1200 + w, n_classes=2)
    Bp = synth.ragged_walks(len(lb), lb, 1201 + w, n_classes=2)
    A, B = eap.SeriesSet.from_packed(Ap), eap.SeriesSet.from_packed(Bp)
    kw = {"window": w}
    ia = np.repeat(np.arange(len(la)), len(lb)).astype(np.int32)
    ib = np.tile(np.arange(len(lb)), len(la)).astype(np.int32)
    base = _run(lambda: eap.eap_pairs(gpu_params(eap, kind, prune=0, **kw), A, B, ia, ib), True).cpu().numpy()
    p1 = gpu_params(eap, kind, prune=1, **kw)
    fin = np.isfinite(base)
    for scale in (0.0, 0.5, 0.9, 1.0, 1.1, 2.0):
        cut = np.where(fin, np.where(fin, base, np.float32(0)) * np.float32(scale), np.float32(1.0)).astype(np.float32)
        got, st = _run(lambda: eap.eap_pairs(p1, A, B, ia, ib, cut, with_stats=True), True)
        ref = _run(lambda: eap.eap_pairs(p1, A, B, ia, ib, cut), False)
        got, ref = got.cpu().numpy(), ref.cpu().numpy()
        want = np.where(fin & (base <= cut), base, np.float32(np.inf))
        assert np.array_equal(got, want), (kind, w, scale, np.flatnonzero(got != want)[:5])
        assert np.array_equal(got, ref), (kind, w, scale)
        if scale < 1.0 and fin.any() and w >= 3:
            assert st["pairs_abandoned"] > 0


@pytest.mark.parametrize("kind", ["cdtw", "erp"])
@pytest.mark.parametrize("prune", [1, 2, 3])
def test_band_eapruned_nn1_matches_panels_and_oracle(eap, kind, prune):
    rng = np.random.default_rng(88 + prune + (kind == "erp"))
    qlen = list(rng.integers(120, 160, size=10))
    rlen = list(rng.integers(120, 160, size=60))
    Qp = synth.ragged_walks(len(qlen), qlen, 611, n_classes=4)
    Rp = synth.ragged_walks(len(rlen), rlen, 612, n_classes=4)
    Q, R = eap.SeriesSet.from_packed(Qp), eap.SeriesSet.from_packed(Rp)
    kw = {"window_ratio": 0.1}
    p = gpu_params(eap, kind, prune=prune, **kw)
    i1, d1, st = _run(lambda: eap.eap_nn1(p, Q, R, with_stats=True), True)
    i0, d0 = _run(lambda: eap.eap_nn1(p, Q, R), False)
    assert np.array_equal(i1.cpu().numpy(), i0.cpu().numpy())
    assert np.array_equal(d1.cpu().numpy(), d0.cpu().numpy())
    D = O.cross(oracle_params(kind, **kw), Qp, Rp)
    check_nn(i1.cpu().numpy(), d1.cpu().numpy(), D)
    if prune in (1, 2):
        assert st["pairs_abandoned"] > 0


def test_band_eapruned_lb_cascade(eap):
    """CDTW with the LB_Keogh cascade ahead of the band kernel (Alg. 2)."""
    ds = synth.make_dataset(200, 40, 256, 5, 97)
    R, Q = eap.SeriesSet.from_matrix(ds.train), eap.SeriesSet.from_matrix(ds.test)
    p = gpu_params(eap, "cdtw", prune=1, window_ratio=0.1, lb=2)
    i1, d1, st = _run(lambda: eap.eap_nn1(p, Q, R, with_stats=True), True)
    i0, d0 = _run(lambda: eap.eap_nn1(p, Q, R), False)
    assert np.array_equal(i1.cpu().numpy(), i0.cpu().numpy())
    assert np.array_equal(d1.cpu().numpy(), d0.cpu().numpy())
    assert st["pairs_lb_pruned"] > 0


def test_band_eapruned_workload_sample(eap):
    """1000 x 1000 x 512 ERP and CDTW, EAPruned in band coordinates: 1-NN
    equal to the column-panel kernel's and, on sampled queries, the oracle."""
    ds = synth.workload_nn1_512()
    tr, te = synth.pack(ds.train), synth.pack(ds.test)
    R, Q = eap.SeriesSet.from_packed(tr), eap.SeriesSet.from_packed(te)
    for kind, kw in (("erp", {"erp_gap": 0.0, "window_ratio": 0.1}), ("cdtw", {"window_ratio": 0.1})):
        p = gpu_params(eap, kind, prune=1, **kw)
        i1, d1 = _run(lambda: eap.eap_nn1(p, Q, R), True)
        i0, d0 = _run(lambda: eap.eap_nn1(p, Q, R), False)
        assert np.array_equal(i1.cpu().numpy(), i0.cpu().numpy())
        assert np.array_equal(d1.cpu().numpy(), d0.cpu().numpy())
        rows = list(np.random.default_rng(13).choice(1000, size=5, replace=False))
        D = O.cross(oracle_params(kind, **kw), synth.pack([ds.test[r] for r in rows]), tr)
        check_nn(i1.cpu().numpy(), d1.cpu().numpy(), D, rows=rows)


def test_band_default_choice(eap):
    """The default takes the band only where every series is at least as long
    as the widest band row: a set with a short series keeps the panel kernels
    (cells counted per band row would exceed the matrix)."""
    rng = np.random.default_rng(3)
    lens = [1, 5, 300] + list(rng.integers(200, 300, size=10))
    Ap = synth.ragged_walks(len(lens), lens, 71, n_classes=2)
    A = eap.SeriesSet.from_packed(Ap)
    p = gpu_params(eap, "erp", prune=0, window_ratio=0.1)
    ia = np.repeat(np.arange(len(lens)), len(lens)).astype(np.int32)
    ib = np.tile(np.arange(len(lens)), len(lens)).astype(np.int32)
    _, st = eap.eap_pairs(p, A, A, ia, ib, with_stats=True)
    L = np.asarray(lens, dtype=np.int64)
    assert st["cells_computed"] <= int((L[ia] * L[ib]).sum())


@pytest.mark.parametrize("kind", ["cdtw", "erp"])
@pytest.mark.parametrize("cost", [0, 1])
@pytest.mark.parametrize("launch", [{"EAP_BAND_G": 8}, {"EAP_BAND_G": 4}, {"EAP_BAND_EXACT": 0}])
def test_band_exact_launches_match_panels_and_oracle(eap, kind, cost, launch):
    """w = 51: the exact launches (8 lanes x 13, 4 lanes x 26 positions, no
    addend right of the window; ERP's top border cell M(0, w + 1) enters the
    last lane in row 1) and the padded launch, Base and EAPruned, against the
    column-panel kernels (bit for bit) and the oracle."""
    w = 51
    la = [104, 104, 130, 155, 104 + w, 120, 200, 104]
    lb = [104, 104 + w, 104, 140, 104, 171, 200, 150]
    Ap = synth.ragged_walks(len(la), la, 5100 + cost, n_classes=2)
    Bp = synth.ragged_walks(len(lb), lb, 5101 + cost, n_classes=2)
    A, B = eap.SeriesSet.from_packed(Ap), eap.SeriesSet.from_packed(Bp)
    kw = {"window": w, "cost": cost}
    if kind == "erp":
        kw["erp_gap"] = 0.25
    ia = np.repeat(np.arange(len(la)), len(lb)).astype(np.int32)
    ib = np.tile(np.arange(len(lb)), len(la)).astype(np.int32)
    p0 = gpu_params(eap, kind, prune=0, **kw)
    got, st = _run(lambda: eap.eap_pairs(p0, A, B, ia, ib, with_stats=True), True, **launch)
    ref = _run(lambda: eap.eap_pairs(p0, A, B, ia, ib), False)
    got, ref = got.cpu().numpy(), ref.cpu().numpy()
    assert np.array_equal(got, ref), (kind, cost, launch, np.flatnonzero(got != ref)[:5])
    D = O.cross(oracle_params(kind, **kw), Ap, Bp)
    for k in range(len(ia)):
        d = float(D[ia[k], ib[k]])
        assert np.isinf(got[k]) if np.isinf(d) else close(float(got[k]), d), (kind, cost, launch, k)
    # Counted cells: every row of a feasible pair holds the 2w + 1 window
    # positions; a pair with |L_A - L_B| > w is decided before any row.
    feas = [k for k in range(len(ia)) if abs(la[ia[k]] - lb[ib[k]]) <= w]
    assert st["cells_computed"] == sum(la[ia[k]] for k in feas) * (2 * w + 1)
    p1 = gpu_params(eap, kind, prune=1, **kw)
    fin = np.isfinite(got)
    for scale in (0.5, 1.0, 1.5):
        cut = np.where(fin, got * np.float32(scale), np.float32(1.0)).astype(np.float32)
        g1 = _run(lambda: eap.eap_pairs(p1, A, B, ia, ib, cut), True, **launch).cpu().numpy()
        want = np.where(fin & (got <= cut), got, np.float32(np.inf))
        assert np.array_equal(g1, want), (kind, cost, launch, scale)
