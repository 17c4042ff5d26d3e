"""eap_nn1_plan: the kernel mapping and strip width an eap_nn1 call runs,
computed on the host by the same function eap_nn1 uses (no GPU needed).

Pins the mapping rules, each of which rests on a measurement recorded with
the kernels: 16-lane groups over column panels up to 2048 points (W = 5,
WDTW 4), band coordinates for windowed CDTW/ERP with the exact 8 x 13
launch at w = 51, a warp per pair above 2048 points, and one CTA per pair
from 6144 points, or from 2048 for DTW and MSM searches of at most 32
queries.  Environment overrides and invalid sizes are checked too.
"""
import os

import pytest

import bench
from paper_2102_05221_gb300 import eap

SIX = [("dtw", {}), ("cdtw", {"window_ratio": 0.1}), ("wdtw", {}), ("erp", {"window_ratio": 0.1}),
       ("msm", {}), ("twe", {})]


def _plan(kind, nq, L, lmin=None, **kw):
    return eap.eap_nn1_plan(eap.params(kind, **kw), nq, lmin or L, L, L)


def _with_env(env, fn):
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


def test_benchmark_workload_runs_the_kernels_bench_names():
    # 1000 x 1000 x 512 with the benchmark's parameters: the labels bench.py
    # reports (DP_KERNELS) are the kernels eap_nn1 runs.
    for kind, _ in SIX:
        pl = eap.eap_nn1_plan(eap.params(kind, **bench.KIND_PARAMS[kind]), 1000, 512, 512, 512)
        label = bench.DP_KERNELS[kind]
        if kind in ("cdtw", "erp"):
            assert pl == {"mapping": "band", "strip_width": 13, "lanes_per_pair": 8, "band_exact": True}, kind
            assert label.startswith("band_dp_kernel") and "W=13, G=8, exact" in label
        else:
            assert pl["mapping"] == "group" and pl["lanes_per_pair"] == 16, kind
            assert label == f"group_dp_kernel<{kind}, W={pl['strip_width']}, G=16>", (kind, pl, label)


@pytest.mark.parametrize("kind", ["dtw", "wdtw", "msm", "twe"])
def test_long_unwindowed_series_run_one_cta_per_pair_at_strip_width_8(kind):
    for nq in (1, 1000):
        assert _plan(kind, nq, 8192) == {"mapping": "cta", "strip_width": 8, "lanes_per_pair": 256,
                                         "band_exact": False}
        assert _plan(kind, nq, 6144)["mapping"] == "cta"


def test_few_query_searches_take_the_cta_mapping_from_2048_points_for_dtw_and_msm():
    for kind in ("dtw", "msm"):
        assert _plan(kind, 16, 4096)["mapping"] == "cta"
        assert _plan(kind, 32, 2048)["mapping"] == "cta"
        assert _plan(kind, 33, 4096)["mapping"] == "warp"      # more queries: the warp mapping
        assert _plan(kind, 16, 2047)["mapping"] == "group"     # below 2048: 16-lane groups
    for kind in ("twe", "wdtw"):                                 # no consistent gain measured
        assert _plan(kind, 16, 4096)["mapping"] == "warp"


def test_medium_series_run_a_warp_per_pair():
    assert _plan("dtw", 1000, 4096) == {"mapping": "warp", "strip_width": 4, "lanes_per_pair": 32,
                                        "band_exact": False}
    assert _plan("twe", 1000, 4096)["strip_width"] == 8        # TWE's 7-op cell amortises W = 8
    assert _plan("msm", 1000, 2048)["mapping"] == "group"
    assert _plan("msm", 1000, 2049)["mapping"] == "warp"


def test_modes_other_than_eapruned():
    # EABase runs a warp per pair only; Prune (each pair's own bound) never
    # takes the CTA mapping; Base of the windowed distances runs in bands.
    assert _plan("dtw", 8, 8192, prune=2)["mapping"] == "warp"
    assert _plan("msm", 8, 8192, prune=3)["mapping"] == "warp"
    assert _plan("cdtw", 1000, 512, prune=0, window_ratio=0.1)["mapping"] == "band"
    assert _plan("dtw", 1000, 512, prune=0)["mapping"] == "warp"   # unwindowed Base: a warp, W = 16
    assert _plan("dtw", 1000, 512, prune=0)["strip_width"] == 16


def test_environment_overrides():
    assert _with_env({"EAP_MAP": "warp"}, lambda: _plan("msm", 4, 8192))["mapping"] == "warp"
    assert _with_env({"EAP_MAP": "cta"}, lambda: _plan("msm", 1000, 512))["mapping"] == "cta"
    assert _with_env({"EAP_W": "4"}, lambda: _plan("dtw", 4, 8192))["strip_width"] == 4
    assert _with_env({"EAP_BAND": "0"}, lambda: _plan("erp", 1000, 512, window_ratio=0.1))["mapping"] != "band"


def test_invalid_sizes_are_rejected():
    p = eap.params("dtw")
    for args in ((-1, 512, 512, 512), (10, 0, 512, 512), (10, 600, 512, 512), (10, 512, 9000, 512),
                 (10, 512, 512, 9000)):
        with pytest.raises(eap.EapError) as e:
            eap.eap_nn1_plan(p, *args)
        assert e.value.code == eap.EAP_EINVAL
