"""Randomised parity sweep: seeded random configurations (distance, cost,
window, parameters, mode, derivative, lengths around the panel widths of
every mapping) through eap_nn1 and eap_pairs against the FP64 oracle; for
CDTW and ERP also with the band mapping forced."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2102_05221_gb300 import synth
from tests.parity_util import KINDS, check_nn, close

pytestmark = pytest.mark.gpu

# Lengths at and around the panel widths of 16-lane groups (W = 4, 5: 64, 80)
# and of a warp per pair (W = 4, 8, 16: 128, 256, 512).
EDGE_LENGTHS = [1, 2, 3, 15, 16, 17, 63, 64, 65, 79, 80, 81, 127, 128, 129, 159, 160, 161, 255, 256, 257, 511, 512, 513]


def _config(rng):
    kind = KINDS[int(rng.integers(0, 6))]
    cfg = {"kind": kind, "gpu": {}, "orc": {}}
    cost = int(rng.integers(0, 2)) if kind != "msm" else 1
    cfg["gpu"]["cost"] = cost
    cfg["orc"]["cost"] = cost
    if kind in ("cdtw", "erp"):
        if rng.random() < 0.5:
            w = int(rng.integers(0, 40))
            cfg["gpu"].update(window=w, window_ratio=-1.0)
            cfg["orc"]["window"] = w
        else:
            r = float(np.float32(rng.uniform(0.02, 1.0)))
            cfg["gpu"]["window_ratio"] = r
            cfg["orc"]["window_ratio"] = r
    if kind == "wdtw":
        g = float(np.float32(rng.uniform(0.0, 0.5)))
        cfg["gpu"]["wdtw_g"] = g
        cfg["orc"]["wdtw_g"] = g
    if kind == "erp":
        g = float(np.float32(rng.uniform(-1.0, 1.0)))
        cfg["gpu"]["erp_gap"] = g
        cfg["orc"]["erp_gap"] = g
    if kind == "msm":
        c = float(np.float32(rng.uniform(0.0, 2.0)))
        cfg["gpu"]["msm_c"] = c
        cfg["orc"]["msm_c"] = c
    if kind == "twe":
        nu = float(np.float32(rng.uniform(0.0, 0.1)))
        lam = float(np.float32(rng.uniform(0.0, 2.0)))
        cfg["gpu"].update(twe_nu=nu, twe_lambda=lam)
        cfg["orc"].update(twe_nu=nu, twe_lambda=lam)
    d = int(rng.random() < 0.2)
    cfg["gpu"]["derivative"] = d
    cfg["orc"]["derivative"] = d
    cfg["gpu"]["prune"] = int(rng.choice([1, 1, 1, 0, 2, 3]))
    return cfg


@pytest.mark.parametrize("seed", range(64))
def test_random_configuration_matches_oracle(seed):
    from paper_2102_05221_gb300 import eap
    rng = np.random.default_rng(10_000 + seed)
    cfg = _config(rng)
    nq, nr = int(rng.integers(1, 12)), int(rng.integers(1, 40))
    pool = EDGE_LENGTHS + list(rng.integers(1, 600, size=8))
    qlen = [int(rng.choice(pool)) for _ in range(nq)]
    rlen = [int(rng.choice(pool)) for _ in range(nr)]
    Qp = synth.ragged_walks(nq, qlen, 20_000 + seed, n_classes=3)
    Rp = synth.ragged_walks(nr, rlen, 30_000 + seed, n_classes=3)
    Q, R = eap.SeriesSet.from_packed(Qp), eap.SeriesSet.from_packed(Rp)
    p = eap.params(cfg["kind"], **cfg["gpu"])
    idx, dist = eap.eap_nn1(p, Q, R)
    D = O.cross(O.make_params(cfg["kind"], **cfg["orc"]), Qp, Rp)
    check_nn(idx.cpu().numpy(), dist.cpu().numpy(), D)
    if cfg["kind"] in ("cdtw", "erp"):
        # The band mapping forced (it takes any band that fits a launch):
        # the same 1-NN, bit for bit.
        old = os.environ.get("EAP_BAND")
        os.environ["EAP_BAND"] = "2"
        try:
            ib, db = eap.eap_nn1(p, Q, R)
        finally:
            if old is None:
                os.environ.pop("EAP_BAND", None)
            else:
                os.environ["EAP_BAND"] = old
        assert np.array_equal(ib.cpu().numpy(), idx.cpu().numpy()), cfg
        assert np.array_equal(db.cpu().numpy(), dist.cpu().numpy()), cfg
    # Explicit pairs with cut-offs around the oracle's distances (EAPruned only).
    if cfg["gpu"]["prune"] == 1:
        ia = np.repeat(np.arange(nq), nr).astype(np.int32)
        ib = np.tile(np.arange(nr), nq).astype(np.int32)
        ref = D[ia, ib]
        cut = np.where(np.isfinite(ref), ref * rng.choice([0.5, 0.99, 1.01, 2.0], size=ref.shape), 1.0)
        got = eap.eap_pairs(p, Q, R, ia, ib, cut.astype(np.float32)).cpu().numpy()
        for k in range(len(ia)):
            d = float(ref[k])
            c = float(np.float32(cut[k]))
            if math.isfinite(d) and d <= c * (1 - 2e-4):
                assert close(float(got[k]), d), (cfg, k, got[k], d, c)
            elif not math.isfinite(d) or d > c * (1 + 2e-4):
                assert math.isinf(got[k]), (cfg, k, got[k], d, c)
