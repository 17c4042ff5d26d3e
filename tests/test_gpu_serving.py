"""Serving loop (eap_serve_*): resident sets, footprint admission, continuous
batching; each result must equal the same query's result alone (eap_nn1 on
its own), and the FP64 oracle within tolerance."""
import time

import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import KINDS, WORKLOAD_PARAMS, check_nn, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


def _wait(srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < timeout
    return out


def test_serving_mixed_distances_and_lengths_match_alone():
    from paper_2102_05221_gb300 import eap
    refs_fixed = synth.ragged_walks(300, [256] * 300, 71)
    refs_mixed = synth.ragged_walks(300, (64, 400), 72)
    qs = synth.ragged_walks(48, (64, 400), 73)
    q256 = synth.ragged_walks(24, [256] * 24, 74)
    with eap.Server(max_inflight=64) as srv:
        sid_fixed = srv.add_refset(refs_fixed)
        sid_mixed = srv.add_refset(refs_mixed)
        jobs = []
        rng = np.random.default_rng(0)
        for i in range(72):
            kind = KINDS[int(rng.integers(0, 6))]
            kw = dict(WORKLOAD_PARAMS[kind])
            if kind in ("cdtw", "erp"):
                kw["window_ratio"] = 0.5
            if i % 3 == 0:
                sid, q = sid_fixed, q256.series(i % 24)
            else:
                sid, q = sid_mixed, qs.series(i % 48)
            p = gpu_params(eap, kind, **kw)
            while True:
                t = srv.submit(sid, p, q)
                if t is not None:
                    break
                time.sleep(0.001)   # not admitted yet: slots free up as batches finish
            jobs.append((t, sid, kind, kw, q))
        res = _wait(srv, [j[0] for j in jobs])
        st = srv.stats()
        assert st["completed"] == 72 and st["inflight"] == 0 and st["batches"] >= 1
        assert st["lat_p99_ms"] >= st["lat_p50_ms"] > 0
    refsets = {sid_fixed: refs_fixed, sid_mixed: refs_mixed}
    R = {k: eap.SeriesSet.from_packed(v) for k, v in refsets.items()}
    for t, sid, kind, kw, q in jobs:
        idx, dist = res[t]
        Q = eap.SeriesSet.from_packed(synth.pack([q]))
        a_idx, a_dist = eap.eap_nn1(gpu_params(eap, kind, **kw), Q, R[sid])
        # The same float32 result alone and in the mix.
        assert idx == int(a_idx.item()) and dist == float(a_dist.item()), (kind, idx, a_idx.item(), dist, a_dist.item())
    # And the oracle agrees (a sample of the queries).
    for t, sid, kind, kw, q in jobs[:12]:
        idx, dist = res[t]
        D = O.cross(oracle_params(kind, **kw), synth.pack([q]), refsets[sid])
        check_nn(np.array([idx]), np.array([dist]), D)


def test_admission_by_footprint_and_slots():
    from paper_2102_05221_gb300 import eap
    refs = synth.ragged_walks(2000, [512] * 2000, 81)
    q = synth.ragged_walks(1, [512], 82).series(0)
    # A budget below one query's footprint admits nothing.
    with eap.Server(hbm_budget_bytes=1024) as srv:
        sid = srv.add_refset(refs)
        assert srv.submit(sid, eap.params("dtw"), q) is None
        assert srv.stats()["rejected"] == 1
    # One slot in flight: a second submit right after the first is refused
    # until the first completes, then admitted.
    with eap.Server(max_inflight=1) as srv:
        sid = srv.add_refset(refs)
        t1 = srv.submit(sid, eap.params("msm", prune=0), q)
        assert t1 is not None
        t2 = srv.submit(sid, eap.params("msm", prune=0), q)
        assert t2 is None
        srv.drain(60000)
        r1 = srv.poll(t1)
        assert r1 is not None
        t3 = srv.submit(sid, eap.params("msm", prune=0), q)
        assert t3 is not None
        srv.drain(60000)
        assert srv.poll(t3) == r1


def test_serving_rejects_bad_arguments():
    from paper_2102_05221_gb300 import eap
    with eap.Server() as srv:
        sid = srv.add_refset(synth.ragged_walks(4, [16] * 4, 1))
        with pytest.raises(eap.EapError):
            srv.submit(sid + 5, eap.params("dtw"), np.zeros(16, np.float32))
        with pytest.raises(eap.EapError):
            srv.submit(sid, eap.params("msm", msm_c=-1.0), np.zeros(16, np.float32))
        with pytest.raises(eap.EapError):
            srv.poll(12345)
