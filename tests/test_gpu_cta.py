"""CTA-per-pair mapping for long series: bit-identical to the warp-per-pair
mapping (same functors, same per-cell arithmetic), for lengths spanning one
panel up to several rounds of eight panels, with and without cut-offs."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import WORKLOAD_PARAMS, check_nn, close, gpu_params, oracle_params

pytestmark = pytest.mark.gpu
UNWINDOWED = ["dtw", "wdtw", "msm", "twe"]


def _with_map(mapping, fn, **env):
    env = {"EAP_MAP": mapping, **env}
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


@pytest.mark.parametrize("W", ["4", "8"])
@pytest.mark.parametrize("kind", UNWINDOWED)
def test_cta_pairs_match_warp_mapping_and_oracle(kind, W):
    # Both strip widths of the CTA kernel (8 by default, 4 when asked for):
    # every cell is the same operations at any width, so the results are
    # bit-identical to the warp mapping's.
    from paper_2102_05221_gb300 import eap
    rng = np.random.default_rng(21)
    la = [1, 5, 130, 700, 1030, 2500, 1500, 64]
    lb = [3, 127, 129, 1100, 2400, 900, 1500, 64]
    Ap = synth.ragged_walks(len(la), la, 301, n_classes=2)
    Bp = synth.ragged_walks(len(lb), lb, 302, n_classes=2)
    A, B = eap.SeriesSet.from_packed(Ap), eap.SeriesSet.from_packed(Bp)
    ia = np.arange(len(la), dtype=np.int32)
    ib = np.arange(len(lb), dtype=np.int32)
    kw = WORKLOAD_PARAMS[kind]
    p0 = gpu_params(eap, kind, prune=0, **kw)
    base_w = _with_map("warp", lambda: eap.eap_pairs(p0, A, B, ia, ib).cpu().numpy())
    base_c = _with_map("cta", lambda: eap.eap_pairs(p0, A, B, ia, ib).cpu().numpy(), EAP_W=W)
    assert np.array_equal(base_w, base_c), (kind, base_w, base_c)
    for k in range(len(la)):
        ref = O.distance(oracle_params(kind, **kw), Ap.series(k), Bp.series(k))
        assert close(float(base_c[k]), ref), (kind, k, base_c[k], ref)
    p1 = gpu_params(eap, kind, prune=1, **kw)
    fin = np.isfinite(base_w)
    for cut in (base_w, np.where(fin, np.nextafter(base_w, np.float32(0)), base_w).astype(np.float32),
                np.zeros_like(base_w), (base_w * np.float32(0.7)).astype(np.float32),
                (base_w * np.float32(1.2)).astype(np.float32)):
        got = _with_map("cta", lambda: eap.eap_pairs(p1, A, B, ia, ib, cut).cpu().numpy(), EAP_W=W)
        want = np.where(base_w <= cut, base_w, np.float32(np.inf))
        assert np.array_equal(got, want), (kind, got, want)


@pytest.mark.parametrize("kind", ["dtw", "msm"])
def test_cta_nn1_and_pairwise(kind):
    from paper_2102_05221_gb300 import eap
    ds = synth.make_dataset(60, 4, 3000, 3, 777)
    tr, te = synth.pack(ds.train), synth.pack(ds.test)
    R, Q = eap.SeriesSet.from_packed(tr), eap.SeriesSet.from_packed(te)
    p = gpu_params(eap, kind, **WORKLOAD_PARAMS[kind])
    iw, dw = _with_map("warp", lambda: eap.eap_nn1(p, Q, R))
    ic, dc = _with_map("cta", lambda: eap.eap_nn1(p, Q, R))
    assert np.array_equal(iw.cpu().numpy(), ic.cpu().numpy())
    assert np.array_equal(dw.cpu().numpy(), dc.cpu().numpy())
    D = O.cross(oracle_params(kind, **WORKLOAD_PARAMS[kind]), te, tr)
    check_nn(ic.cpu().numpy(), dc.cpu().numpy(), D)
    S = eap.SeriesSet.from_packed(synth.pack(list(ds.train[:10])))
    mw = _with_map("warp", lambda: eap.eap_pairwise(p, S, eap.EAP_PRUNE_ONLY).cpu().numpy())
    mc = _with_map("cta", lambda: eap.eap_pairwise(p, S, eap.EAP_PRUNE_ONLY).cpu().numpy())
    assert np.array_equal(mw, mc)


@pytest.mark.parametrize("kind", UNWINDOWED)
def test_cta_nn1_at_8192_against_full_oracle_rows(kind):
    """L = 8192, the length the CTA mapping exists for (the default from 6144
    up): 1-NN of 2 queries among 48 candidates against the oracle's complete
    distance rows (every candidate, FP64), and bit-identical to the warp
    mapping.  (This test found the CTA abandoning vote ignoring live boundary
    rows that wait for a busy warp's next panel.)"""
    from paper_2102_05221_gb300 import eap
    ds = synth.make_dataset(48, 2, 8192, 3, 8192 + UNWINDOWED.index(kind))
    tr, te = synth.pack(ds.train), synth.pack(ds.test)
    R, Q = eap.SeriesSet.from_packed(tr), eap.SeriesSet.from_packed(te)
    kw = WORKLOAD_PARAMS[kind]
    if kind == "wdtw":
        # g = 0.05 at L = 8192 puts every weight near exp(-205): below the
        # float32 range, all distances round to 0.  g = 0.01 keeps them in range.
        kw = dict(kw, wdtw_g=0.01)
    p = gpu_params(eap, kind, **kw)
    ic, dc = eap.eap_nn1(p, Q, R)                       # default mapping: CTA at this length
    ic2, dc2 = _with_map("cta", lambda: eap.eap_nn1(p, Q, R))
    iw, dw = _with_map("warp", lambda: eap.eap_nn1(p, Q, R))
    for i, d in ((ic2, dc2), (iw, dw)):
        assert np.array_equal(i.cpu().numpy(), ic.cpu().numpy())
        assert np.array_equal(d.cpu().numpy(), dc.cpu().numpy())
    D = O.cross(oracle_params(kind, **kw), te, tr)
    check_nn(ic.cpu().numpy(), dc.cpu().numpy(), D)


@pytest.mark.parametrize("W", ["4", "8"])
@pytest.mark.parametrize("L", [7168, 8192])
def test_cta_explicit_cutoffs_at_long_lengths(W, L):
    """Explicit cut-offs from D to 10 D on every pair of 2 x 48 series at
    7168 and 8192 points (several rounds of eight panels): the CTA mapping
    returns D exactly when D <= cut-off, for both strip widths."""
    from paper_2102_05221_gb300 import eap
    ds = synth.make_dataset(48, 2, 8192, 3, 8192)
    A = eap.SeriesSet.from_matrix(ds.test[:, :L])
    B = eap.SeriesSet.from_matrix(ds.train[:, :L])
    ia = np.repeat(np.arange(2), 48).astype(np.int32)
    ib = np.tile(np.arange(48), 2).astype(np.int32)
    old = os.environ.get("EAP_W")
    os.environ["EAP_W"] = W
    try:
        base = _with_map("cta", lambda: eap.eap_pairs(eap.params("dtw", prune=0), A, B, ia, ib).cpu().numpy())
        for sc in (1.0, 1.2, 1.5, 2.0, 3.0, 5.0, 10.0):
            cut = (base * np.float32(sc)).astype(np.float32)
            got = _with_map("cta", lambda: eap.eap_pairs(eap.params("dtw", prune=1), A, B, ia, ib, cut).cpu().numpy())
            assert np.array_equal(got, base), (W, L, sc, np.flatnonzero(got != base)[:6])
    finally:
        if old is None:
            os.environ.pop("EAP_W", None)
        else:
            os.environ["EAP_W"] = old
