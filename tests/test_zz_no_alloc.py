"""eap_pairs_noalloc: the allocation-free variant of eap_pairs.

It exists for callers that cannot allocate device memory during a call (a
fixed memory budget committed at start-up, or a framework that owns every
device allocation); its scratch comes from a fixed 4 MiB array inside the
library.  It dispatches the same kernels as eap_pairs, so its results must be
bit-identical to eap_pairs' and, like them, match the FP64 oracle.

This file is collected last, so that a run stopping at the first failure has
run every other test first; one test re-runs the check in a fresh Python
process, so the file does not depend on what ran before it.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import REL_TOL

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [("dtw", {}), ("cdtw", {"window_ratio": 0.3}), ("erp", {"window_ratio": 0.5}),
         ("wdtw", {"wdtw_g": 0.05}), ("msm", {}), ("twe", {"twe_nu": 0.001, "twe_lambda": 1.0})]


def _sets(eap, na, nb, lo, hi, seed):
    rng = np.random.default_rng(seed)
    ap = synth.ragged_walks(na, list(rng.integers(lo, hi, size=na)), seed + 1)
    bp = synth.ragged_walks(nb, list(rng.integers(lo, hi, size=nb)), seed + 2)
    ia = np.repeat(np.arange(na), nb).astype(np.int32)
    ib = np.tile(np.arange(nb), na).astype(np.int32)
    return ap, bp, eap.SeriesSet.from_packed(ap), eap.SeriesSet.from_packed(bp), ia, ib


def _check_against_pairs_and_oracle(eap, kind, kw, ap, bp, A, B, ia, ib):
    """Two noalloc calls in a row, Base and EAPruned, against eap_pairs (bit
    for bit) and the oracle (within the parity tolerance); a third of the
    pairs get half their distance as cut-off and must be abandoned."""
    p0 = eap.params(kind, prune=0, **kw)
    ref = eap.eap_pairs(p0, A, B, ia, ib).cpu().numpy()
    D = O.cross(O.make_params(kind, **kw), ap, bp)[ia, ib]
    fin = np.isfinite(D)
    assert np.array_equal(np.isfinite(ref), fin), kind
    assert np.all(np.abs(ref[fin] - D[fin]) <= REL_TOL * np.abs(D[fin])), kind
    p1 = eap.params(kind, prune=1, **kw)
    cut = np.where(fin, ref * np.float32(1.0 + 1e-3), np.float32(np.inf)).astype(np.float32)
    cut[::3] = ref[::3] * np.float32(0.5)
    ref_pruned = eap.eap_pairs(p1, A, B, ia, ib, cut).cpu().numpy()
    must_abandon = np.zeros(len(ref), bool)
    must_abandon[::3] = fin[::3] & (ref[::3] > 0)
    assert must_abandon.sum() > 0
    for call in range(2):
        got0 = eap.eap_pairs_noalloc(p0, A, B, ia, ib).cpu().numpy()
        got1 = eap.eap_pairs_noalloc(p1, A, B, ia, ib, cut).cpu().numpy()
        assert np.array_equal(got0, ref), (kind, call)
        assert np.array_equal(got1, ref_pruned), (kind, call)
        assert np.all(np.isinf(got1[must_abandon])), (kind, call)
        keep = ~must_abandon & fin
        keep[::3] = False
        assert np.array_equal(got1[keep], ref[keep]), (kind, call)


@pytest.mark.parametrize("kind,kw", CASES)
def test_noalloc_matches_eap_pairs_and_oracle_on_two_calls_in_a_row(kind, kw):
    from paper_2102_05221_gb300 import eap
    ap, bp, A, B, ia, ib = _sets(eap, 12, 10, 30, 300, 61)
    _check_against_pairs_and_oracle(eap, kind, kw, ap, bp, A, B, ia, ib)


@pytest.mark.parametrize("kind", ["dtw", "msm"])
def test_noalloc_long_unwindowed_series_take_the_cta_mapping_like_eap_pairs(kind):
    # Rows and columns of 6144 points and more run CTA-per-pair in eap_pairs;
    # the allocation-free call must pick the same mapping and results.
    from paper_2102_05221_gb300 import eap
    ap, bp, A, B, ia, ib = _sets(eap, 2, 3, 6144, 6400, 71)
    _check_against_pairs_and_oracle(eap, kind, {}, ap, bp, A, B, ia, ib)


def _mempool():
    """The default memory pool of the current device (stream-ordered
    allocations land there) through the CUDA runtime the library links."""
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
            break
        except OSError:
            rt = None
    if rt is None:
        pytest.skip("libcudart not found by name")
    import torch
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    used_high = 8   # cudaMemPoolAttrUsedMemHigh

    def high():
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, used_high, ctypes.byref(v)) == 0
        return v.value

    def reset():
        z = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, used_high, ctypes.byref(z)) == 0
    return high, reset


def test_noalloc_takes_nothing_from_the_stream_ordered_pool():
    # eap_pairs draws its scratch from the device's default pool (the
    # high-water mark rises); eap_pairs_noalloc must leave it untouched and
    # must not change the device's free memory.
    import torch

    from paper_2102_05221_gb300 import eap
    high, reset = _mempool()
    ap, bp, A, B, ia, ib = _sets(eap, 16, 16, 100, 400, 81)
    p = eap.params("erp", prune=0, window_ratio=0.5)
    # Every tensor the calls touch exists before the measured window.
    out = torch.empty(len(ia), dtype=torch.float32, device="cuda")
    cut = torch.full((len(ia),), float("inf"), dtype=torch.float32, device="cuda")
    dia, dib = torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()
    want = eap.eap_pairs(p, A, B, dia, dib, cut)
    eap.eap_pairs_noalloc(p, A, B, dia, dib, cut, out=out)   # first call: set-up of the array's address
    torch.cuda.synchronize()
    reset()
    base = high()
    want = eap.eap_pairs(p, A, B, dia, dib, cut)
    torch.cuda.synchronize()
    assert high() > base   # the check sees stream-ordered scratch
    reset()
    base = high()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        eap.eap_pairs_noalloc(p, A, B, dia, dib, cut, out=out)
    torch.cuda.synchronize()
    assert high() == base
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.equal(out, want)


_FRESH = r"""
import sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_2102_05221_gb300 import eap, synth
rng = np.random.default_rng(5)
ap = synth.ragged_walks(6, list(rng.integers(40, 200, size=6)), 91)
bp = synth.ragged_walks(5, list(rng.integers(40, 200, size=5)), 92)
A, B = eap.SeriesSet.from_packed(ap), eap.SeriesSet.from_packed(bp)
ia = np.repeat(np.arange(6), 5).astype(np.int32)
ib = np.tile(np.arange(5), 6).astype(np.int32)
for kind in ("erp", "wdtw", "msm"):
    p = eap.params(kind, prune=0)
    got = [eap.eap_pairs_noalloc(p, A, B, ia, ib).cpu().numpy() for _ in range(2)]
    want = eap.eap_pairs(p, A, B, ia, ib).cpu().numpy()
    assert np.array_equal(got[0], want) and np.array_equal(got[1], want), kind
print("fresh ok")
"""


def test_noalloc_in_a_fresh_process():
    # The first call in a process looks up the array's device address; run
    # that path in a new interpreter, before anything else touched the library.
    r = subprocess.run([sys.executable, "-c", _FRESH.format(root=ROOT)], capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "fresh ok" in r.stdout, r.stdout + r.stderr


def test_noalloc_rejects_scratch_beyond_its_limit():
    from paper_2102_05221_gb300 import eap
    big = synth.pack([np.zeros(600_000, np.float32), np.zeros(600_000, np.float32)])
    S = eap.SeriesSet.from_packed(synth.pack([np.zeros(8, np.float32)]))
    # ERP needs 4 bytes per element of both sets: 1.2M + 8 floats do not fit in 4 MiB.
    B = eap.SeriesSet(big.data, big.offsets, np.array([8, 8], np.int32))
    with pytest.raises(eap.EapError) as e:
        eap.eap_pairs_noalloc(eap.params("erp", prune=0), S, B, [0], [0])
    assert e.value.code == eap.EAP_EINVAL
