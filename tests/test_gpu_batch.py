"""Batched uneven workload: many datasets of different lengths and distances
in one call (eap_nn1_batch: batched pre-passes, then each task's DP on the
kernel eap_nn1 picks for it), the autotuner, and CUDA-graph capture of the
whole batch."""
import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import KINDS, WORKLOAD_PARAMS, check_nn, gpu_params, oracle_params

pytestmark = pytest.mark.gpu


def _tasks(eap, n=12, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for d in range(n):
        L = int(np.clip(np.rint(np.exp(rng.uniform(np.log(24), np.log(600)))), 24, 600))
        ntr = int(rng.integers(16, 160))
        nte = int(rng.integers(4, 40))
        kind = KINDS[d % 6]
        kw = dict(WORKLOAD_PARAMS[kind])
        if kind in ("cdtw", "erp"):
            kw["window_ratio"] = float(rng.uniform(0.05, 0.2))
        if kind in ("dtw", "cdtw") and d % 2 == 0:
            kw["lb"] = 2
        ds = synth.make_dataset(ntr, nte, L, int(rng.integers(2, 8)), 9000 + d)
        tr, te = synth.pack(ds.train), synth.pack(ds.test)
        out.append((kind, kw, tr, te, eap.Nn1Task(gpu_params(eap, kind, **kw), eap.SeriesSet.from_packed(te),
                                                  eap.SeriesSet.from_packed(tr))))
    return out


def test_batch_equals_per_task_nn1_and_oracle():
    from paper_2102_05221_gb300 import eap
    import torch
    items = _tasks(eap)
    st = eap.eap_nn1_batch([t for *_, t in items], with_stats=True)
    torch.cuda.synchronize()
    assert st["pairs"] == sum(t.queries.count * t.refs.count for *_, t in items)
    for kind, kw, tr, te, t in items:
        i1, d1 = eap.eap_nn1(t.p, t.queries, t.refs)
        assert np.array_equal(t.out_idx.cpu().numpy(), i1.cpu().numpy()), kind
        assert np.array_equal(t.out_dist.cpu().numpy(), d1.cpu().numpy()), kind
    for kind, kw, tr, te, t in items[:6]:
        D = O.cross(oracle_params(kind, **kw), te, tr)
        check_nn(t.out_idx.cpu().numpy(), t.out_dist.cpu().numpy(), D)


def test_batch_in_a_captured_cuda_graph():
    from paper_2102_05221_gb300 import eap
    import torch
    items = _tasks(eap, n=8, seed=1)
    tasks = [t for *_, t in items]
    eap.eap_nn1_batch(tasks)
    torch.cuda.synchronize()
    ref = [(t.out_idx.clone(), t.out_dist.clone()) for t in tasks]
    for t in tasks:
        t.out_idx.fill_(-7)
        t.out_dist.fill_(-7.0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            eap.eap_nn1_batch(tasks, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        for t in tasks:
            t.out_idx.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        for t, (i0, d0) in zip(tasks, ref):
            assert torch.equal(t.out_idx, i0) and torch.equal(t.out_dist, d0)


def test_autotune_picks_a_width_and_keeps_results(tmp_path):
    from paper_2102_05221_gb300 import eap
    items = _tasks(eap, n=6, seed=2)
    tasks = [t for *_, t in items]
    path = str(tmp_path / "tune.txt")
    eap.eap_autotune_reset()
    eap.eap_autotune(tasks, cache_path=path)
    lines = open(path).read().split("\n")
    rows = [list(map(int, l.split())) for l in lines if l.strip()]
    assert rows and all(r[3] in (4, 5, 8, 16) and r[4] in (1, 2) for r in rows)
    eap.eap_autotune_reset()
    eap.eap_autotune_load(path)
    for kind, kw, tr, te, t in items:
        i1, d1 = eap.eap_nn1(t.p, t.queries, t.refs)
        D = O.cross(oracle_params(kind, **kw), te, tr)
        check_nn(i1.cpu().numpy(), d1.cpu().numpy(), D)
    eap.eap_autotune_reset()


def test_batch_runs_each_task_on_eap_nn1s_mapping():
    """A batch mixing the mappings: CDTW at 512 points (exact band launch),
    MSM (16-lane groups), DTW at 6200 points (CTA per pair by default), and a
    2500-point TWE task with the CTA mapping forced by the map override.  The
    batch must give the per-task eap_nn1 results bit for bit (same kernels,
    same candidate order and seeds) and agree with the oracle."""
    import os

    import torch

    from paper_2102_05221_gb300 import eap
    specs = [("cdtw", {"window_ratio": 0.1}, 512, 60, 6), ("msm", {"msm_c": 0.5}, 300, 50, 5),
             ("dtw", {}, 6200, 12, 2), ("twe", {"twe_nu": 0.001, "twe_lambda": 1.0}, 2500, 16, 2)]
    items = []
    for k, (kind, kw, L, ntr, nte) in enumerate(specs):
        ds = synth.make_dataset(ntr, nte, L, 3, 7700 + k)
        tr, te = synth.pack(ds.train), synth.pack(ds.test)
        items.append((kind, kw, tr, te, eap.Nn1Task(gpu_params(eap, kind, **kw), eap.SeriesSet.from_packed(te),
                                                    eap.SeriesSet.from_packed(tr))))
    old = os.environ.get("EAP_MAP")
    try:
        for mapping in (None, "cta"):
            if mapping:
                os.environ["EAP_MAP"] = mapping
            st = eap.eap_nn1_batch([t for *_, t in items], with_stats=True)
            torch.cuda.synchronize()
            assert st["dp_ms"] > 0
            for kind, kw, tr, te, t in items:
                i1, d1 = eap.eap_nn1(t.p, t.queries, t.refs)
                assert np.array_equal(t.out_idx.cpu().numpy(), i1.cpu().numpy()), (kind, mapping)
                assert np.array_equal(t.out_dist.cpu().numpy(), d1.cpu().numpy()), (kind, mapping)
    finally:
        if old is None:
            os.environ.pop("EAP_MAP", None)
        else:
            os.environ["EAP_MAP"] = old
    for kind, kw, tr, te, t in items:
        D = O.cross(oracle_params(kind, **kw), te, tr)
        check_nn(t.out_idx.cpu().numpy(), t.out_dist.cpu().numpy(), D)
