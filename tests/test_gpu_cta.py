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


def _with_map(mapping, fn):
    old = os.environ.get("EAP_MAP")
    os.environ["EAP_MAP"] = mapping
    try:
        return fn()
    finally:
        if old is None:
            del os.environ["EAP_MAP"]
        else:
            os.environ["EAP_MAP"] = old


@pytest.mark.parametrize("kind", UNWINDOWED)
def test_cta_pairs_match_warp_mapping_and_oracle(kind):
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
    base_c = _with_map("cta", lambda: eap.eap_pairs(p0, A, B, ia, ib).cpu().numpy())
    assert np.array_equal(base_w, base_c), (kind, base_w, base_c)
    for k in range(len(la)):
        ref = O.distance(oracle_params(kind, **kw), Ap.series(k), Bp.series(k))
        assert close(float(base_c[k]), ref), (kind, k, base_c[k], ref)
    p1 = gpu_params(eap, kind, prune=1, **kw)
    fin = np.isfinite(base_w)
    for cut in (base_w, np.where(fin, np.nextafter(base_w, np.float32(0)), base_w).astype(np.float32),
                np.zeros_like(base_w), (base_w * np.float32(0.7)).astype(np.float32),
                (base_w * np.float32(1.2)).astype(np.float32)):
        got = _with_map("cta", lambda: eap.eap_pairs(p1, A, B, ia, ib, cut).cpu().numpy())
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
