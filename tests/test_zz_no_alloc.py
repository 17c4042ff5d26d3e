"""eap_pairs_noalloc: the allocation-free variant of eap_pairs.

It exists for callers that cannot allocate device memory during a call (a
fixed memory budget committed at start-up, or a framework that owns every
device allocation); its scratch comes from a fixed 4 MiB array inside the
library.  This file is collected last on purpose, and its test must pass
both alone in a fresh process and after every other test.
"""
import numpy as np
import pytest

from paper_2102_05221_gb300 import synth
from tests.parity_util import REL_TOL

pytestmark = pytest.mark.gpu

CASES = [("dtw", {}), ("erp", {"window_ratio": 0.5}), ("wdtw", {"wdtw_g": 0.05}), ("msm", {})]


@pytest.mark.parametrize("kind,kw", CASES)
def test_noalloc_matches_eap_pairs_on_two_calls_in_a_row(kind, kw):
    from paper_2102_05221_gb300 import eap
    rng = np.random.default_rng(3)
    ap = synth.ragged_walks(12, list(rng.integers(30, 300, size=12)), 61)
    bp = synth.ragged_walks(10, list(rng.integers(30, 300, size=10)), 62)
    A, B = eap.SeriesSet.from_packed(ap), eap.SeriesSet.from_packed(bp)
    ia = np.repeat(np.arange(12), 10).astype(np.int32)
    ib = np.tile(np.arange(10), 12).astype(np.int32)
    p0 = eap.params(kind, prune=0, **kw)
    ref = eap.eap_pairs(p0, A, B, ia, ib).cpu().numpy()
    p1 = eap.params(kind, prune=1, **kw)
    cut = np.where(np.isfinite(ref), ref * np.float32(1.0 + 1e-3), np.float32(np.inf)).astype(np.float32)
    cut[::3] = ref[::3] * np.float32(0.5)   # a third of the pairs must abandon
    ref_pruned = eap.eap_pairs(p1, A, B, ia, ib, cut).cpu().numpy()
    for call in range(2):
        got0 = eap.eap_pairs_noalloc(p0, A, B, ia, ib).cpu().numpy()
        got1 = eap.eap_pairs_noalloc(p1, A, B, ia, ib, cut).cpu().numpy()
        for got, want in ((got0, ref), (got1, ref_pruned)):
            fin = np.isfinite(want)
            assert np.array_equal(np.isfinite(got), fin), (kind, call)
            assert np.all(np.abs(got[fin] - want[fin]) <= REL_TOL * np.abs(want[fin])), (kind, call)


def test_noalloc_rejects_scratch_beyond_its_limit():
    from paper_2102_05221_gb300 import eap
    big = synth.pack([np.zeros(600_000, np.float32), np.zeros(600_000, np.float32)])
    S = eap.SeriesSet.from_packed(synth.pack([np.zeros(8, np.float32)]))
    # ERP needs 4 bytes per element of both sets: 1.2M + 8 floats do not fit in 4 MiB.
    B = eap.SeriesSet(big.data, big.offsets, np.array([8, 8], np.int32))
    with pytest.raises(eap.EapError) as e:
        eap.eap_pairs_noalloc(eap.params("erp", prune=0), S, B, [0], [0])
    assert e.value.code == eap.EAP_EINVAL
