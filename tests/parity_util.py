"""Helpers shared by the GPU parity tests: oracle parameter mapping and the
1-NN comparison rule (indices exact except flagged near-ties, distances
within 1e-4 relative of the FP64 oracle)."""
import math

import numpy as np

import oracle as O

REL_TOL = 1e-4        # float32 distances vs the FP64 oracle
TIE_REL = 2e-4        # oracle top-2 gap below this is a flagged near-tie

KINDS = ["dtw", "cdtw", "wdtw", "erp", "msm", "twe"]

# Parameters of the 1000 x 1000 x 512 workload (CDTW and ERP windows are 10%).
WORKLOAD_PARAMS = {
    "dtw": {}, "cdtw": {"window_ratio": 0.1}, "wdtw": {"wdtw_g": 0.05, "wdtw_wmax": 1.0},
    "erp": {"erp_gap": 0.0, "window_ratio": 0.1}, "msm": {"msm_c": 0.5},
    "twe": {"twe_nu": 0.001, "twe_lambda": 1.0},
}


def oracle_params(kind, **kw):
    kw = dict(kw)
    kw.pop("prune", None)
    kw.pop("lb", None)
    return O.make_params(kind, **kw)


def gpu_params(eap, kind, **kw):
    kw = dict(kw)
    if kind not in ("cdtw", "erp"):
        kw.pop("window_ratio", None)
        kw.pop("window", None)
    if "window" in kw and "window_ratio" not in kw:
        kw["window_ratio"] = -1.0
    return eap.params(kind, **kw)


def close(a, b, rel=REL_TOL):
    if math.isinf(a) or math.isinf(b):
        return a == b
    return abs(a - b) <= rel * max(abs(b), 1e-30) or abs(a - b) <= 1e-6 * rel


def check_nn(gpu_idx, gpu_dist, D, rows=None, rel=REL_TOL):
    """Compare GPU 1-NN results with the oracle's distance matrix D
    ([queries x candidates], FP64).  Returns the number of flagged near-ties."""
    gpu_idx = np.asarray(gpu_idx)
    gpu_dist = np.asarray(gpu_dist, dtype=np.float64)
    rows = range(D.shape[0]) if rows is None else rows
    ties = 0
    for k, q in enumerate(rows):
        d = D[k]
        finite = np.isfinite(d)
        if not finite.any():
            assert gpu_idx[q] == -1 and math.isinf(gpu_dist[q]), (q, gpu_idx[q], gpu_dist[q])
            continue
        best = int(np.argmin(d))          # lowest index among equal minima
        dmin = d[best]
        srt = np.sort(d[finite])
        gap = (srt[1] - srt[0]) if len(srt) > 1 else math.inf
        assert close(float(gpu_dist[q]), float(dmin), rel), (q, float(gpu_dist[q]), float(dmin))
        if gpu_idx[q] != best:
            # Allowed only for a flagged near-tie, and the GPU's pick must be
            # one of the near-minimal candidates.
            assert gap <= TIE_REL * max(dmin, 1e-30), (q, int(gpu_idx[q]), best, gap, dmin)
            assert close(float(d[gpu_idx[q]]), float(dmin), 2 * TIE_REL), (q, int(gpu_idx[q]), best)
            ties += 1
    return ties
