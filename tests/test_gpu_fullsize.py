"""Parity at the full sizes of the other workloads, on outputs the oracle can
compute one by one: the 256 x 4096 DTW and MSM prune-only matrices, the
64-dataset uneven batch in one launch, and 1-NN against the serving sets."""
import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import check_nn, close, oracle_params

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["dtw", "msm"])
def test_allpairs_4096_sampled(kind):
    from paper_2102_05221_gb300 import eap
    x = synth.workload_allpairs_4096()
    S = eap.SeriesSet.from_matrix(x)
    m = eap.eap_pairwise(eap.params(kind), S, eap.EAP_PRUNE_ONLY).cpu().numpy()
    assert np.all(np.diag(m) == 0) and np.array_equal(m, m.T) and np.all(np.isfinite(m))
    rng = np.random.default_rng(3)
    for _ in range(6):
        i, j = rng.choice(x.shape[0], size=2, replace=False)
        ref = O.distance(oracle_params(kind), x[i], x[j])
        assert close(float(m[i, j]), ref), (kind, i, j, m[i, j], ref)


def test_uneven_64_batch_sampled():
    from paper_2102_05221_gb300 import eap
    ds = synth.workload_uneven()
    tasks, meta = [], []
    for d in ds:
        R = eap.SeriesSet.from_matrix(d.data.train)
        Q = eap.SeriesSet.from_matrix(d.data.test)
        for kind, kw in (("cdtw", {"window_ratio": d.window_ratio, "lb": 2}),
                         ("erp", {"erp_gap": 0.0, "window_ratio": 0.1}),
                         ("twe", {"twe_nu": 0.001, "twe_lambda": 1.0})):
            tasks.append(eap.Nn1Task(eap.params(kind, **kw), Q, R))
            meta.append((kind, kw, d))
    eap.eap_nn1_batch(tasks)
    # Check 2 queries of every task whose oracle row is cheap enough.
    rng = np.random.default_rng(4)
    checked = 0
    for t, (kind, kw, d) in zip(tasks, meta):
        ntr, L = d.data.train.shape
        if ntr * L * L > 2.5e8:
            continue
        rows = list(rng.choice(d.data.test.shape[0], size=2, replace=False))
        okw = {k: v for k, v in kw.items() if k != "lb"}
        D = O.cross(oracle_params(kind, **okw), synth.pack([d.data.test[r] for r in rows]), synth.pack(d.data.train))
        check_nn(t.out_idx.cpu().numpy(), t.out_dist.cpu().numpy(), D, rows=rows)
        checked += 1
    assert checked >= 60


def test_serving_sets_sampled():
    from paper_2102_05221_gb300 import eap
    sets = synth.serving_refsets({128: 50000, 1024: 10000, 8192: 2000, "mixed": 20000})
    rng = np.random.default_rng(5)
    with eap.Server(max_inflight=64) as srv:
        sids = {L: srv.add_refset(p) for L, p in sets.items()}
        jobs = []
        for L, kind in ((128, "msm"), (1024, "dtw"), (8192, "twe"), ("mixed", "erp"), (128, "wdtw"), (1024, "cdtw")):
            qlen = L if L != "mixed" else 300
            q = synth.random_walks(rng, 1, qlen).astype(np.float32)[0]
            p = eap.params(kind)
            t = srv.submit(sids[L], p, q)
            assert t is not None
            jobs.append((t, L, kind, q))
        srv.drain(600000)
        for t, L, kind, q in jobs:
            idx, dist = srv.poll(t)
            refs = sets[L]
            op = oracle_params(kind, window_ratio=0.1) if kind in ("cdtw", "erp") else oracle_params(kind)
            if refs.count * float(np.mean(refs.lengths)) * qlen_of(L) <= 1.5e9:
                D = O.cross(op, synth.pack([q]), refs)   # the whole oracle row
                check_nn(np.array([idx]), np.array([dist]), D)
            else:
                # Large set: the returned candidate's distance, and no sampled
                # candidate clearly closer.
                assert close(float(dist), O.distance(op, q, refs.series(idx))), (L, kind)
                others = rng.choice(refs.count, size=24, replace=False)
                D = O.cross(op, synth.pack([q]), synth.pack([refs.series(c) for c in others]))
                assert np.all(D[0] >= float(dist) * (1 - 1e-4)), (L, kind)


def qlen_of(L):
    return L if L != "mixed" else 300
