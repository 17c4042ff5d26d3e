#!/usr/bin/env python3
"""Benchmark: EAPruned 1-NN for the six elastic distances on one GB300.

Workload (one "step"): 1000 test x 1000 train z-normalised random-walk +
sine-template series of length 512, 10 classes; 1-NN of every test series
under DTW, CDTW (window 10%), WDTW (g=0.05, wmax=1), ERP (g=0, window 10%),
MSM (c=0.5) and TWE (nu=0.001, lambda=1), each through the C ABI
(eap_nn1).  A query = one (test series, distance) 1-NN search, so one step
answers 6000 queries.

Prints one JSON line (rank 0).  `value` = queries/s with the inputs resident
in HBM; `e2e` = the same through eap_nn1_host with pinned host buffers
(host->device copies and the result read-back inside the timed region);
`roofline` = the dominant DP kernel's algorithmic FP32 op rate against the
ALU peak; `cpu_baseline` = the FP64 CPU oracle on a bounded sample.

`--impl reference` times the oracle instead (the program the CUDA path is
checked against), on the same workload, metric and unit.

Multi-GPU (torchrun): each rank answers its own 1000 test series (a
different seed) against the same train set; there is no collective on the
data path (weak scaling); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

KIND_PARAMS = {
    "dtw": {}, "cdtw": {"window_ratio": 0.1}, "wdtw": {"wdtw_g": 0.05, "wdtw_wmax": 1.0},
    "erp": {"erp_gap": 0.0, "window_ratio": 0.1}, "msm": {"msm_c": 0.5},
    "twe": {"twe_nu": 0.001, "twe_lambda": 1.0},
}
# Algorithmic FP32 instructions per cell update of each distance's recurrence
# (the minimum the cell needs: see the functors in csrc/eap_device.cuh).
OPS_PER_CELL = {"dtw": 3, "cdtw": 3, "wdtw": 4, "erp": 5, "msm": 9, "twe": 7}
# Kernels this library launches per eap_nn1 call: init, upper bound, sort,
# DP, unpack; ERP adds two border kernels, WDTW one weight table.
LAUNCHES = {"dtw": 5, "cdtw": 5, "wdtw": 6, "erp": 8, "msm": 6, "twe": 6}
N_TRAIN, N_TEST, LENGTH, N_CLASSES = 1000, 1000, 512, 10
# DRAM bytes (read + write) of the dominant DP launch on this workload, from
# one ncu capture (profiles/group_dp_kernel_msm_nn1_512_traffic.md), valid only for
# the library build whose source fingerprint is recorded with it.
# The EAPruned DP launch of this workload (L = 512) per distance: 16 lanes per
# pair over column panels (W = 5, WDTW 4), CDTW and ERP in band coordinates
# (8 lanes x 13 cells = the 2w + 2 = 104 positions of a band row).
DP_KERNELS = {"dtw": "group_dp_kernel<dtw, W=5, G=16>", "wdtw": "group_dp_kernel<wdtw, W=4, G=16>",
              "msm": "group_dp_kernel<msm, W=5, G=16>", "twe": "group_dp_kernel<twe, W=5, G=16>",
              "cdtw": "band_dp_kernel<cdtw, W=13, G=8, exact>", "erp": "band_dp_kernel<erp, W=13, G=8, exact>"}
TRAFFIC = {"kernel": "group_dp_kernel<msm, W=5, G=16>", "bytes": 14997760 + 0,
           "fingerprint": "36f88f7bd2e70e992531c82fc20bd24ccd06b22326dde33b36ef223a7d797ec4"}
METRIC = "1-NN queries/s (six distances, EAPruned, 1000 train x 1000 test, L=512)"
UNIT = "queries/s"
L2_FLUSH_BYTES = 512 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def alu_peak_ops(sms: int, mhz: float) -> float:
    """FP32 lane-instruction peak: SMs x 128 FP32 lanes x clock."""
    return sms * 128 * mhz * 1e6


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="eap_clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            os.unlink(self.path)
        except Exception:
            return out
        sm, mx, busy, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            try:
                if len(r) > 9 and float(r[9]) > 0:
                    busy.append(float(r[1]))   # a sample taken while kernels were running
            except ValueError:
                pass
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            # The median under load: samples taken while the GPU was busy
            # (host-side set-up of a workload leaves it idle at low clocks).
            load = busy if busy else sm
            out = {"sm_mhz": statistics.median(load), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm), "samples_under_load": len(busy),
                   "sm_mhz_all_samples": statistics.median(sm)}
        return out


def make_inputs(rank: int):
    from paper_2102_05221_gb300 import synth
    ds = synth.workload_nn1_512(N_TRAIN, N_TEST, seed_offset=0)
    if rank:
        # Each rank answers its own test series (weak scaling), same train set.
        ds_r = synth.workload_nn1_512(N_TRAIN, N_TEST, seed_offset=rank)
        ds.test = ds_r.test
    return ds


# ---------------------------------------------------------------------------
# Reference arm: the FP64 CPU oracle on a bounded sample of the workload.
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np

    import oracle as O
    from paper_2102_05221_gb300 import synth
    ds = make_inputs(0)
    tr = synth.pack(ds.train)
    cores = os.cpu_count() or 1
    nq = max(1, min(args.ref_queries or cores, N_TEST))
    rng = np.random.default_rng(0)

    def step(i):
        rows = rng.choice(N_TEST, size=nq, replace=False)
        q = synth.pack([ds.test[r] for r in rows])
        for kind, kw in KIND_PARAMS.items():
            O.nn1(O.make_params(kind, **kw), q, tr, nthreads=cores)
        return nq * len(KIND_PARAMS)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    done = 0
    for i in range(args.steps):
        done += step(i)
    dt = time.perf_counter() - t0
    value = done / dt
    sample = f"{nq} random test series x 1000 train x 6 distances per step (FP64 oracle, {cores} threads)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": "nn1_six_distances_1000x1000_L512",
                                            "sample_queries_per_step": nq},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(ds, budget_s: float, n_test: int):
    """The oracle as it stands, timed on this host's cores on a bounded sample:
    full FP64 distance rows (plain definition, no pruning) of the first nq test
    series against every train series, per distance.  Returns the baseline
    entry and the rows (for the sampled parity check)."""
    import oracle as O
    from paper_2102_05221_gb300 import synth
    cores = os.cpu_count() or 1
    tr = synth.pack(ds.train)
    # Calibrate on 1 query per distance, then size the sample to the budget.
    t0 = time.perf_counter()
    q1 = synth.pack([ds.test[0]])
    for kind, kw in KIND_PARAMS.items():
        O.cross(O.make_params(kind, **kw), q1, tr, nthreads=cores)
    t1 = time.perf_counter() - t0
    per_q = t1 / len(KIND_PARAMS)   # one query on one thread ~ cores x this when threads split the queries
    nq = int(max(cores, min(256, budget_s / max(per_q, 1e-6) * cores / len(KIND_PARAMS))))
    nq = min(n_test, (nq // cores) * cores or cores)
    q = synth.pack([ds.test[i] for i in range(nq)])
    rows = {}
    t0 = time.perf_counter()
    for kind, kw in KIND_PARAMS.items():
        rows[kind] = O.cross(O.make_params(kind, **kw), q, tr, nthreads=cores)
    dt = time.perf_counter() - t0
    entry = {"value": nq * len(KIND_PARAMS) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"test series 0..{nq - 1} x 1000 train x 6 distances, FP64 oracle (full distance rows, "
                       f"no pruning), {cores} threads, {dt:.1f} s"}
    return entry, rows


def cpu_alg5_baseline(ds, budget_s: float):
    """The paper's own design on the CPU, like for like: Alg. 1 calling Alg. 5
    (EAPruned, FP64) with the best-so-far as cut-off, candidates in index
    order, ONE thread; whole rounds of one query per distance until the
    budget is spent.  Returns the entry and the (index, distance) results."""
    import oracle as O
    from paper_2102_05221_gb300 import synth
    tr = synth.pack(ds.train)
    res = {k: [] for k in KIND_PARAMS}
    t0 = time.perf_counter()
    rounds, cells = 0, 0
    while rounds == 0 or time.perf_counter() - t0 < budget_s:
        q = synth.pack([ds.test[rounds]])
        for kind, kw in KIND_PARAMS.items():
            idx, dist, c = O.nn1_eapruned(O.make_params(kind, **kw), q, tr)
            res[kind].append((int(idx[0]), float(dist[0])))
            cells += c
        rounds += 1
    dt = time.perf_counter() - t0
    entry = {"value": rounds * len(KIND_PARAMS) / dt, "unit": UNIT, "cores": 1, "kind": "oracle_alg5",
             "sample": f"test series 0..{rounds - 1} x 1000 train x 6 distances, Alg. 1 + Alg. 5 (FP64, "
                       f"cut-off = best so far, index order), one thread, {dt:.1f} s",
             "cells_computed_over_effective": cells / (rounds * len(KIND_PARAMS) * N_TRAIN * LENGTH * LENGTH)}
    return entry, res


def sampled_parity(rows, out_idx, out_dist):
    """GPU 1-NN results of the sampled test series against the oracle's full
    distance rows: indices exact unless the oracle's top-2 gap is under
    2e-4 relative (a near-tie: flagged and counted), distances within 1e-4
    relative of FP64."""
    import numpy as np
    res = {"queries": 0, "index_mismatches": 0, "near_ties": 0, "near_tie_index_differs": 0,
           "max_rel_err": 0.0, "tolerance_rel": 1e-4}
    for kind, D in rows.items():
        gi = out_idx[kind][:D.shape[0]].cpu().numpy()
        gd = out_dist[kind][:D.shape[0]].cpu().numpy().astype(np.float64)
        for q in range(D.shape[0]):
            best = int(np.argmin(D[q]))
            ref = float(D[q, best])
            srt = np.sort(D[q])
            tie = len(srt) > 1 and srt[1] - srt[0] <= 2e-4 * max(ref, 1e-30)
            res["queries"] += 1
            res["near_ties"] += int(tie)
            if int(gi[q]) != best:
                if tie:
                    res["near_tie_index_differs"] += 1
                else:
                    res["index_mismatches"] += 1
            res["max_rel_err"] = max(res["max_rel_err"], abs(float(gd[q]) - ref) / max(ref, 1e-30))
    res["ok"] = res["index_mismatches"] == 0 and res["max_rel_err"] <= 1e-4
    return res


def _near_tie(row) -> bool:
    import numpy as np
    srt = np.sort(row)
    return len(srt) > 1 and srt[1] - srt[0] <= 2e-4 * max(float(srt[0]), 1e-30)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-queries", type=int, default=0,
                    help="test series per step of the reference arm (0: one per host core)")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--alg5-budget", type=float, default=8.0,
                    help="seconds of the single-thread Alg. 1 + Alg. 5 CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-unpruned", action="store_true",
                    help="skip the unpruned (Base) DP block of the benchmark line")
    ap.add_argument("--unpruned-steps", type=int, default=2)
    ap.add_argument("--stats-steps", type=int, default=3,
                    help="untimed steps after the timed region for the per-distance statistics")
    ap.add_argument("--kinds", default=",".join(KIND_PARAMS),
                    help="subset of distances (profiling runs only; the benchmark is all six)")
    ap.add_argument("--n-test", type=int, default=N_TEST, help="test series per rank (profiling runs only)")
    ap.add_argument("--mode", default="per-distance", choices=["per-distance", "batch"],
                    help="per-distance: one eap_nn1 call per distance; batch: all six in one eap_nn1_batch launch")
    ap.add_argument("--workload", default="nn1_512",
                    choices=["nn1_512", "unpruned_512", "modes_512", "subseq", "allpairs_4096", "nn1_8192", "uneven_64",
                             "serving", "lb_cascade"],
                    help="nn1_512 is the benchmark; the others measure the remaining workloads")
    args = ap.parse_args()
    kinds = [k for k in args.kinds.split(",") if k]
    n_test = args.n_test

    if args.gpus < 1:
        raise SystemExit("--gpus must be >= 1")
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # One process per GPU: re-launch this command under torchrun.
        import socket
        with socket.socket() as sk:
            sk.bind(("127.0.0.1", 0))
            port = sk.getsockname()[1]
        cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={args.gpus}",
               "--master-addr=127.0.0.1", f"--master-port={port}", os.path.abspath(__file__)] + sys.argv[1:]
        return subprocess.call(cmd)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus:
        raise SystemExit(f"bench.py --gpus {args.gpus} runs with WORLD_SIZE={world}: launch one rank per GPU")
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "nn1_512":
        return run_other_workload(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2102_05221_gb300 import eap
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    if torch.cuda.device_count() <= local:
        raise SystemExit(f"rank {rank}: LOCAL_RANK {local} but only {torch.cuda.device_count()} GPU(s) visible")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")

    def barrier():
        if world > 1:
            dist.barrier()

    eap.load()
    ds = make_inputs(rank)
    R = eap.SeriesSet.from_matrix(ds.train)
    ds.test = ds.test[:n_test]
    Q = eap.SeriesSet.from_matrix(ds.test)
    stream = torch.cuda.current_stream()
    params = {k: eap.params(k, **KIND_PARAMS[k]) for k in kinds}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out_idx = {k: torch.empty(n_test, dtype=torch.int32, device="cuda") for k in kinds}
    out_dist = {k: torch.empty(n_test, dtype=torch.float32, device="cuda") for k in kinds}

    batch_tasks = [eap.Nn1Task(params[k], Q, R, out_idx[k], out_dist[k]) for k in kinds]

    def step(collect):
        flush.fill_(1.0)   # L2 flush between steps (inputs are smaller than L2)
        if args.mode == "batch":
            st = eap.eap_nn1_batch(batch_tasks, stream=stream, with_stats=collect is not None)
            if collect is not None:
                c = collect.setdefault("batch", {"cells_computed": 0, "cells_effective": 0, "calls": 0})
                c["cells_computed"] += st["cells_computed"]
                c["cells_effective"] += st["cells_effective"]
                c["calls"] += 1
            return
        if collect is not None:
            # Per-distance statistics (DP time by the library's CUDA events,
            # cell counters): one distance at a time, each call synchronised.
            for k in kinds:
                _, _, st = eap.eap_nn1(params[k], Q, R, stream=stream, with_stats=True,
                                       out_idx=out_idx[k], out_dist=out_dist[k])
                c = collect.setdefault(k, {"dp_ms": 0.0, "cells_computed": 0, "cells_effective": 0, "calls": 0})
                c["dp_ms"] += st["dp_ms"]
                c["cells_computed"] += st["cells_computed"]
                c["cells_effective"] += st["cells_effective"]
                c["calls"] += 1
            return
        # The timed step: the six 1-NN searches back to back on the step's
        # stream, nothing synchronised on the host.  (Each search's DP is a
        # persistent launch that fills the GPU, so running them on concurrent
        # streams measured no faster and varied more.)
        for k in kinds:
            eap.eap_nn1(params[k], Q, R, stream=stream, out_idx=out_idx[k], out_dist=out_dist[k])

    for _ in range(max(3, args.warmup)):
        step(None)
    torch.cuda.synchronize()
    barrier()
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    per = {}
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(None)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop() if sampler else None
    t_ms = e0.elapsed_time(e1)
    # Per-distance breakdown, after the timed region (untimed steps).
    for _ in range(max(1, args.stats_steps)):
        step(per)
    torch.cuda.synchronize()
    if world > 1:
        t = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    queries = n_test * len(kinds) * args.steps * world
    value = queries / (t_ms / 1e3)

    # End to end through the host-buffer entry point (pinned host memory).
    e2e = None
    if not args.no_e2e:
        from paper_2102_05221_gb300 import synth
        trp, tep = synth.pack(ds.train), synth.pack(ds.test)

        def pin(a):
            return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()

        class H:
            pass
        hq, hr = H(), H()
        hq.data, hq.offsets, hq.lengths = pin(tep.data), pin(tep.offsets), pin(tep.lengths)
        hr.data, hr.offsets, hr.lengths = pin(trp.data), pin(trp.offsets), pin(trp.lengths)
        hidx = torch.empty(n_test, dtype=torch.int32).pin_memory()
        hdist = torch.empty(n_test, dtype=torch.float32).pin_memory()

        def e2e_step():
            for k in kinds:
                eap.eap_nn1_host(params[k], hq, hr, out_idx=hidx, out_dist=hdist)

        for _ in range(2):
            e2e_step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        barrier()
        te = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([te], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            te = float(t.item())
        h2d = len(kinds) * (tep.data.nbytes + trp.data.nbytes + tep.offsets.nbytes + tep.lengths.nbytes
                                  + trp.offsets.nbytes + trp.lengths.nbytes)
        d2h = len(kinds) * n_test * (4 + 4)
        e2e = {"value": n_test * len(kinds) * args.steps * world / te, "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    props = torch.cuda.get_device_properties(local)
    if args.mode == "batch":
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "nn1_six_distances_1000x1000_L512", "mode": "batch"},
                "stats": per.get("batch"), "e2e": e2e}
        print(json.dumps(line), flush=True)
        return 0
    # Dominant kernel: the DP of the distance with the largest device time.
    peaks = _peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    per_dist = {}
    for k, c in per.items():
        s = c["dp_ms"] / 1e3
        per_dist[k] = {
            "dp_ms_per_call": c["dp_ms"] / c["calls"],
            "queries_per_s_dp": n_test * c["calls"] / s if s else None,
            "effective_cells_per_s": c["cells_effective"] / s if s else None,
            "computed_cells_per_s": c["cells_computed"] / s if s else None,
            "computed_over_effective": c["cells_computed"] / max(1, c["cells_effective"]),
            "ops_per_cell": OPS_PER_CELL[k],
            "alu_frac": (c["cells_computed"] * OPS_PER_CELL[k] / s) / alu_peak_ops(props.multi_processor_count, max_mhz)
            if s else None,
        }
    dom = max(per, key=lambda k: per[k]["dp_ms"])
    c = per[dom]
    s = c["dp_ms"] / 1e3
    peak = alu_peak_ops(props.multi_processor_count, max_mhz) / 1e12
    achieved = c["cells_computed"] * OPS_PER_CELL[dom] / s / 1e12
    traffic = None
    try:
        from paper_2102_05221_gb300 import build as _b
        if TRAFFIC["kernel"] == DP_KERNELS[dom] and TRAFFIC["fingerprint"] == _b._fingerprint():
            traffic = TRAFFIC["bytes"]
    except Exception:
        traffic = None
    roofline = {"bound": "alu", "kernel": DP_KERNELS[dom], "achieved": achieved, "peak": peak,
                "unit": "Tops/s", "frac": achieved / peak, "traffic": traffic,
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {max_mhz:.0f} MHz (max SM clock)",
                "work_basis": f"{OPS_PER_CELL[dom]} FP32 ops per computed cell"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "nn1_six_distances_1000x1000_L512", "n_train": N_TRAIN, "n_test": N_TEST,
                   "length": LENGTH, "classes": N_CLASSES, "distances": KIND_PARAMS,
                   "l2": "flushed between steps (512 MiB write); inputs 4 MB < L2"},
        "roofline": roofline,
        "per_distance": per_dist,
        "gpu_launches": sum(LAUNCHES[k] for k in kinds) * args.steps,
        "clocks": clocks,
    }
    if e2e:
        line["e2e"] = e2e
    if kinds != list(KIND_PARAMS) or n_test != N_TEST:
        line["config"]["profiling_subset"] = {"kinds": kinds, "n_test": n_test}
    if not args.no_unpruned:
        # Base (Alg. 3) DP of every distance on the same inputs: the ALU
        # roofline of the unpruned recurrence, with its own clock record.
        us = ClockSampler(local)
        us.start()
        time.sleep(0.3)
        rows = unpruned_rows(eap, R, Q, LENGTH, kinds, args.unpruned_steps, 1, alu_peak_ops(
            props.multi_processor_count, max_mhz), flush)
        line["unpruned"] = {"workload": f"base_dp_{N_TRAIN}x{n_test}_L{LENGTH}", "per_distance": rows,
                            "clocks": us.stop(),
                            "basis": "algorithmic cells (windowed: |i-j| <= w only) x ops/cell / DP event time"}
    if not args.no_cpu_baseline and world == 1 and kinds == list(KIND_PARAMS):
        line["cpu_baseline"], orows = cpu_baseline(ds, args.cpu_budget, n_test)
        line["parity_sample"] = sampled_parity(orows, out_idx, out_dist)
        line["cpu_baseline_alg5"], a5 = cpu_alg5_baseline(ds, args.alg5_budget)
        # The single-thread Alg. 5 search must agree with the GPU on its queries too.
        a5_bad = 0
        for k, lst in a5.items():
            gi = out_idx[k].cpu().numpy()
            gd = out_dist[k].cpu().numpy()
            for q, (i5, d5) in enumerate(lst):
                tie = q < orows[k].shape[0] and _near_tie(orows[k][q])
                if abs(float(gd[q]) - d5) > 1e-4 * max(d5, 1e-30) or (int(gi[q]) != i5 and not tie):
                    a5_bad += 1
        line["cpu_baseline_alg5"]["disagreements_with_gpu"] = a5_bad
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# The other workloads (one JSON line each; the benchmark itself is nn1_512).
# ---------------------------------------------------------------------------
def _sync_time(fn, reps=1):
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _alu_peak(props):
    return alu_peak_ops(props.multi_processor_count, float(_peaks().get("sm_max_mhz", 2070.0)))


def algorithmic_cells(kind: str, L: int) -> int:
    """Cells of one L x L pair that the recurrence defines: every cell, or for
    a windowed distance only those with |i - j| <= w."""
    import numpy as np
    if "window_ratio" in KIND_PARAMS[kind]:
        w = int(math.floor(float(np.float32(KIND_PARAMS[kind]["window_ratio"])) * L))
        return sum(min(L, i + w) - max(1, i - w) + 1 for i in range(1, L + 1))
    return L * L


def unpruned_rows(eap, R, Q, L, kinds, steps, warmup, peak, flush):
    """Base (Alg. 3) 1-NN DP per distance on R x Q: DP time from the library's
    CUDA events on the launching stream, L2 flushed before every call;
    algorithmic cell updates/s and their fraction of the FP32 ALU roofline."""
    out = {}
    for k in kinds:
        p = eap.params(k, prune=0, **KIND_PARAMS[k])
        for _ in range(max(1, warmup)):
            eap.eap_nn1(p, Q, R)
        ms, cells = 0.0, 0
        for _ in range(steps):
            flush.fill_(1.0)
            _, _, st = eap.eap_nn1(p, Q, R, with_stats=True)
            ms += st["dp_ms"]
            cells += st["cells_computed"]
        band = algorithmic_cells(k, L)
        alg = band * R.count * Q.count * steps
        rate = alg / (ms / 1e3)
        out[k] = {"dp_ms": ms / steps, "cells_per_s": rate, "ops_per_cell": OPS_PER_CELL[k],
                  "alu_frac": rate * OPS_PER_CELL[k] / peak,
                  "cells_roofline_per_s": peak / OPS_PER_CELL[k],
                  "algorithmic_cells_per_pair": band,
                  "computed_cells_per_pair": cells / (steps * R.count * Q.count)}
    return out


def workload_unpruned_512(args):
    """Base (unpruned) DP on the 1000 x 1000 x 512 workload: the ALU roofline."""
    import torch

    from paper_2102_05221_gb300 import eap
    ds = make_inputs(0)
    R, Q = eap.SeriesSet.from_matrix(ds.train), eap.SeriesSet.from_matrix(ds.test)
    props = torch.cuda.get_device_properties(0)
    peak = _alu_peak(props)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = unpruned_rows(eap, R, Q, ds.train.shape[1], args.kinds.split(","), args.steps, args.warmup, peak, flush)
    return {"metric": "unpruned (Base) DP algorithmic cell updates/s vs FP32 ALU roofline, 1000 x 1000 x 512",
            "value": out["dtw"]["cells_per_s"] if "dtw" in out else None, "unit": "cells/s",
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "base_dp_1000x1000_L512", "l2": "flushed before each call (512 MiB write)"},
            "per_distance": out, "roofline_peak_ops": peak}


def workload_lb_cascade(args):
    """The envelope + LB_Keogh pass (Alg. 2, the lb-keogh2 cascade of Section
    5.2) ahead of the EAPruned CDTW DP: 64 queries against 40,000 candidates
    of length 512 (z-normalised random walks; candidates and their envelopes
    take 246 MB, more than the 129 MB L2).  The pass is timed by the library
    with CUDA events on the launching stream (stats lb_ms); its HBM roofline
    counts the bytes it must move: every series read once, every envelope
    written once and read once, the bound matrix written once."""
    import numpy as np
    import torch

    from paper_2102_05221_gb300 import eap, synth
    nq, nr, L = 64, 40000, 512
    rng = np.random.default_rng(5120)
    R = eap.SeriesSet.from_matrix(synth.random_walks(rng, nr, L).astype(np.float32))
    Q = eap.SeriesSet.from_matrix(synth.random_walks(rng, nq, L).astype(np.float32))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    p = eap.params("cdtw", window_ratio=0.1, lb=2)
    for _ in range(max(1, args.warmup)):
        eap.eap_nn1(p, Q, R)
    lb_ms, dp_ms, pruned, pairs = [], [], 0, 0
    for _ in range(args.steps):
        flush.fill_(1.0)
        _, _, st = eap.eap_nn1(p, Q, R, with_stats=True)
        lb_ms.append(st["lb_ms"])
        dp_ms.append(st["dp_ms"])
        pruned += st["pairs_lb_pruned"]
        pairs += st["pairs"]
    t = statistics.median(lb_ms)
    elems = (nq + nr) * L
    unique = elems * 4 + elems * 8 + elems * 8 + nq * nr * 4   # series read, envelopes written + read, bounds written
    per_pair = nq * nr * L * 12                                # 4 B + 8 B (reverse) per element per pair, no reuse
    hbm = float(_peaks().get("hbm_gbs", 6800.0))
    props = torch.cuda.get_device_properties(0)
    alu = _alu_peak(props)
    ops = nq * nr * L * 2 * 4   # per point and direction: max, min, sub, fma (clamp, difference, squared sum)
    return {"metric": "envelope + LB_Keogh2 pass, point-pairs/s (64 x 40,000 x 512, CDTW 10%)",
            "value": nq * nr * L / (t / 1e3), "unit": "point-pairs/s", "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "lb_keogh2_64x40000_L512", "l2": "flushed before each call (512 MiB write); "
                       "candidates + envelopes 246 MB > L2"},
            "lb_ms": t, "dp_ms": statistics.median(dp_ms), "pairs_lb_pruned_frac": pruned / max(1, pairs),
            "roofline": {"bound": "alu", "achieved": ops / (t / 1e3) / 1e12, "peak": alu / 1e12, "unit": "Tops/s",
                         "frac": ops / (t / 1e3) / alu, "traffic": None,
                         "basis": "8 FP32 ops per point-pair (both directions) over the whole pass (envelopes "
                                  "included in the time)"},
            "hbm": {"unique_bytes": unique, "gbs": unique / (t / 1e3) / 1e9, "peak_gbs": hbm,
                    "frac": unique / (t / 1e3) / 1e9 / hbm,
                    "basis": "series 4 B/elem read, envelopes 8 B/elem written and read, bounds 4 B/pair written"},
            "algorithmic_per_pair_gbs": per_pair / (t / 1e3) / 1e9}


def workload_modes_512(args):
    """Base, Prune, EABase and EAPruned 1-NN (the four implementations of the
    paper's NN experiment, Section 5.1) on the 1000 x 1000 x 512 workload:
    whole eap_nn1 calls (upper bounds, sort and DP) timed with CUDA events,
    L2 flushed before each call."""
    import statistics

    import torch

    from paper_2102_05221_gb300 import eap
    ds = make_inputs(0)
    R, Q = eap.SeriesSet.from_matrix(ds.train), eap.SeriesSet.from_matrix(ds.test)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    modes = {"base": 0, "prune": 3, "eabase": 2, "eapruned": 1}
    out, total = {}, {m: 0.0 for m in modes}
    for k in args.kinds.split(","):
        row = {}
        for name, m in modes.items():
            p = eap.params(k, prune=m, **KIND_PARAMS[k])
            for _ in range(max(1, args.warmup)):
                eap.eap_nn1(p, Q, R)
            ms = []
            for _ in range(args.steps):
                flush.fill_(1.0)
                ms.append(_sync_time(lambda: eap.eap_nn1(p, Q, R)))
            _, _, st = eap.eap_nn1(p, Q, R, with_stats=True)
            t = statistics.median(ms)
            total[name] += t
            row[name] = {"ms": t, "queries_per_s": Q.count / (t / 1e3),
                         "cells_computed_over_effective": st["cells_computed"] / max(1, st["cells_effective"]),
                         "pairs_abandoned": st["pairs_abandoned"]}
        e = row["eapruned"]["ms"]
        row["eapruned_speedup"] = {"vs_base": row["base"]["ms"] / e, "vs_eabase": row["eabase"]["ms"] / e,
                                   "vs_prune": row["prune"]["ms"] / e}
        out[k] = row
    e = total["eapruned"]
    return {"metric": "1-NN time per implementation: Base / Prune / EABase / EAPruned, 1000 x 1000 x 512",
            "value": total["base"] / e, "unit": "x (EAPruned speed-up over Base, six distances summed)",
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "nn1_modes_1000x1000_L512", "steps": args.steps,
                       "l2": "flushed before each call (512 MiB write)"},
            "total_ms": total,
            "speedup_all": {"vs_base": total["base"] / e, "vs_eabase": total["eabase"] / e,
                            "vs_prune": total["prune"] / e},
            "paper_cpu_context": {"vs_base": 7.61, "vs_eabase": 2.86,
                                  "note": "UCR archive, 85 datasets, one Opteron core (Section 5.1)"},
            "per_distance": out}


def workload_subseq(args):
    """Sub-sequence search (Section 5.3): a 16M-point series, queries of 128 to
    1024 points planted with N(0, 0.1) noise, CDTW (10% window) and DTW."""
    import time

    import torch

    import oracle as O
    from paper_2102_05221_gb300 import eap, synth
    n = 1 << 24
    T = synth.long_series(n, synth.seed_for(6))
    lens = [128, 128, 256, 256, 512, 512, 1024, 1024]
    Qp, planted = synth.subseq_queries(T, lens, synth.seed_for(6, 1), planted=True, noise=0.1)
    Tdev = torch.from_numpy(T).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    for kind, kw in (("cdtw", {"window_ratio": 0.1}), ("dtw", {})):
        p = eap.params(kind, **kw)
        per_len = {}
        for m in sorted(set(lens)):
            sel = [k for k, L in enumerate(lens) if L == m]
            Q = eap.SeriesSet.from_packed(synth.pack([Qp.series(k) for k in sel]))
            for _ in range(max(1, args.warmup)):
                eap.eap_subseq(p, Tdev, Q)
            ms = []
            for _ in range(args.steps):
                flush.fill_(1.0)
                ms.append(_sync_time(lambda: eap.eap_subseq(p, Tdev, Q)))
            pos, dist, st = eap.eap_subseq(p, Tdev, Q, with_stats=True)
            t = sorted(ms)[len(ms) // 2] / len(sel)
            per_len[m] = {"ms_per_query": t, "windows_per_s": (n - m + 1) / (t / 1e3),
                          "windows_pruned_by_bounds": st["pairs_lb_pruned"] / st["pairs"],
                          "cells_computed_over_effective": st["cells_computed"] / max(1, st["cells_effective"]),
                          "found_planted": int(sum(int(a) == int(planted[k]) for a, k in zip(pos.cpu().numpy(), sel)))}
        out[kind] = per_len
    # The oracle (every window in full, FP64) on a bounded sample of windows of one 256-point query.
    q = Qp.series(2)
    sample = 4000
    t0 = time.perf_counter()
    O.subseq(O.make_params("cdtw", window_ratio=0.1), T[:sample + 255], q)
    cpu_wps = sample / (time.perf_counter() - t0)
    head = out["cdtw"][256]["windows_per_s"]
    return {"metric": "sub-sequence search windows/s (16M-point series, z-normalised CDTW 10%, 256-point queries)",
            "value": head, "unit": "windows/s", "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "subseq_16M", "n": n, "query_lengths": lens, "noise": 0.1,
                       "l2": "flushed before each call (512 MiB write); series 64 MB < L2 not guaranteed resident"},
            "per_distance": out,
            "cpu_baseline": {"value": cpu_wps, "unit": "windows/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{sample} windows of one 256-point query, CDTW 10%, every window in full"}}


def workload_allpairs_4096(args):
    """256 random walks of length 4096: full DTW and MSM matrices, prune-only."""
    import torch

    from paper_2102_05221_gb300 import eap, synth
    x = synth.workload_allpairs_4096()
    S = eap.SeriesSet.from_matrix(x)
    n = x.shape[0]
    pairs = n * (n - 1) // 2
    props = torch.cuda.get_device_properties(0)
    res = {}
    for k in ("dtw", "msm"):
        p = eap.params(k, **KIND_PARAMS[k])
        eap.eap_pairwise(p, S, eap.EAP_PRUNE_ONLY)
        m, st = eap.eap_pairwise(p, S, eap.EAP_PRUNE_ONLY, with_stats=True)
        t = _sync_time(lambda: eap.eap_pairwise(p, S, eap.EAP_PRUNE_ONLY), reps=args.steps)
        mb, stb = eap.eap_pairwise(p, S, eap.EAP_BASE, with_stats=True)
        same = bool(torch.equal(m, mb))
        res[k] = {"ms": t, "pairs_per_s": pairs / (t / 1e3), "effective_cells_per_s": st["cells_effective"] / (t / 1e3),
                  "computed_over_effective": st["cells_computed"] / st["cells_effective"],
                  "base_dp_ms": stb["dp_ms"], "prune_dp_ms": st["dp_ms"],
                  "base_alu_frac": st["cells_effective"] / (stb["dp_ms"] / 1e3) * OPS_PER_CELL[k] / _alu_peak(props),
                  "prune_only_equals_base": same}
    tot = sum(r["ms"] for r in res.values())
    return {"metric": "all-pairs matrices (DTW + MSM, prune-only), 256 x 4096", "value": 2 * pairs / (tot / 1e3),
            "unit": "pairs/s", "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "allpairs_256_L4096", "n": n, "length": int(x.shape[1])}, "per_distance": res}


def workload_nn1_8192(args):
    """1-NN of 16 queries against 200 candidates of 8192 points, EAPruned, for
    DTW, MSM and TWE (unwindowed: one CTA per pair at this length; WDTW's
    weights underflow float32 there at the benchmark's g): whole-call time,
    DP time and the DP's fraction of the ALU roofline on computed cells."""
    import torch

    from paper_2102_05221_gb300 import eap, synth
    ds = synth.workload_nn1_8192()
    R = eap.SeriesSet.from_matrix(ds.train)
    Q = eap.SeriesSet.from_matrix(ds.test)
    props = torch.cuda.get_device_properties(0)
    res = {}
    for k in ("dtw", "msm", "twe"):
        p = eap.params(k, **KIND_PARAMS[k])
        eap.eap_nn1(p, Q, R)
        t = _sync_time(lambda: eap.eap_nn1(p, Q, R), reps=max(1, args.steps))
        _, _, st = eap.eap_nn1(p, Q, R, with_stats=True)
        res[k] = {"ms_per_call": t, "dp_ms": st["dp_ms"], "queries_per_s": Q.count / (t / 1e3),
                  "computed_over_effective": st["cells_computed"] / st["cells_effective"],
                  "alu_frac": st["cells_computed"] / (st["dp_ms"] / 1e3) * OPS_PER_CELL[k] / _alu_peak(props)}
    tot = sum(r["ms_per_call"] for r in res.values())
    return {"metric": "1-NN queries/s, long series (DTW, MSM, TWE; EAPruned; 200 train x 16 test, L=8192)",
            "value": len(res) * Q.count / (tot / 1e3), "unit": "queries/s", "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "nn1_long_200x16_L8192", "n_train": R.count, "n_test": Q.count, "length": 8192,
                       "mapping": "one CTA (8 warps) per pair, the default from 6144 points"},
            "per_distance": res}


def _uneven_tasks(eap, synth):
    ds = synth.workload_uneven()
    tasks, meta = [], []
    for d in ds:
        R = eap.SeriesSet.from_matrix(d.data.train)
        Q = eap.SeriesSet.from_matrix(d.data.test)
        for kind, kw in (("cdtw", {"window_ratio": d.window_ratio, "lb": 2}),
                         ("erp", {"erp_gap": 0.0, "window_ratio": 0.1}),
                         ("twe", {"twe_nu": 0.001, "twe_lambda": 1.0})):
            tasks.append(eap.Nn1Task(eap.params(kind, **kw), Q, R))
            meta.append((kind, d.length, Q.count, R.count))
    return tasks, meta


def workload_uneven_64(args):
    """64 datasets (L 24..2048), CDTW+LB_Keogh2, ERP and TWE: one
    eap_nn1_batch call per step (batched pre-passes, each task's DP on its
    own kernel) replayed from a CUDA graph, against one launch per query."""
    import numpy as np
    import torch

    from paper_2102_05221_gb300 import eap, synth
    tasks, meta = _uneven_tasks(eap, synth)
    nq = sum(t.queries.count for t in tasks)
    eap.eap_autotune_reset()
    t0 = time.perf_counter()
    eap.eap_autotune(tasks)
    tune_s = time.perf_counter() - t0
    st = eap.eap_nn1_batch(tasks, with_stats=True)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            eap.eap_nn1_batch(tasks, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(max(1, args.warmup)):
        g.replay()
    t_batch = _sync_time(g.replay, reps=args.steps)
    q_batch = nq / (t_batch / 1e3)
    # One launch (one eap_nn1 call) per query, plain EAPruned, on a sample.
    rng = np.random.default_rng(0)
    sample = [(ti, int(rng.integers(0, t.queries.count))) for ti, t in enumerate(tasks) for _ in range(2)]
    singles = []
    for ti, qi in sample:
        t = tasks[ti]
        o = int(t.queries.h_offsets[qi])
        L = int(t.queries.h_lengths[qi])
        singles.append((t.p, eap.SeriesSet(t.queries.data[o:o + L], [0], [L]), t.refs))
    for p, Q1, R in singles[:8]:
        eap.eap_nn1(p, Q1, R)

    def run_singles():
        for p, Q1, R in singles:
            eap.eap_nn1(p, Q1, R)
    t_single = _sync_time(run_singles, reps=1)
    q_single = len(singles) / (t_single / 1e3)
    return {"metric": "batched uneven 1-NN queries/s (64 datasets, CDTW+LB_Keogh2, ERP, TWE), one graph-captured eap_nn1_batch call",
            "value": q_batch, "unit": "queries/s", "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "ms_per_step": t_batch, "steps": args.steps,
            "config": {"workload": "uneven_64_datasets_L24_2048", "tasks": len(tasks), "queries_per_step": nq},
            "one_launch_per_query": {"value": q_single, "unit": "queries/s", "sample_queries": len(singles)},
            "speedup_vs_one_launch_per_query": q_batch / q_single,
            "autotune_s": tune_s, "stats_one_step": st}


def workload_serving(args):
    """Serving loop: 8 resident sets, Poisson arrivals, uniform over distances
    and sets; p50/p99 latency and sustained queries/s per offered rate."""
    import numpy as np

    from paper_2102_05221_gb300 import eap, synth
    sizes = {128: 50000, 256: 30000, 512: 20000, 1024: 10000, 2048: 5000, 4096: 3000, 8192: 2000, "mixed": 20000}
    if args.n_test != N_TEST:   # smaller sets for quick runs
        f = args.n_test / N_TEST
        sizes = {k: max(64, int(v * f)) for k, v in sizes.items()}
    refsets = synth.serving_refsets(sizes)
    qpool = {L: synth.random_walks(np.random.default_rng(77 + i), 64, L if L != "mixed" else 512).astype(np.float32)
             for i, L in enumerate(sizes)}
    rates = [50, 100, 200, 400, 1000, 5000, 20000, 50000]
    duration = 1.5
    kinds = list(KIND_PARAMS)
    params = {k: eap.params(k, **KIND_PARAMS[k]) for k in kinds}
    out = {}
    with eap.Server(max_inflight=128) as srv:
        sids = {L: srv.add_refset(p) for L, p in refsets.items()}
        keys = list(sids)
        rng = np.random.default_rng(5)
        # warm-up: one query per (set, distance)
        wt = [srv.submit(sids[L], params[k], qpool[L][0]) for L in keys for k in kinds]
        srv.drain(600000)
        for t in wt:
            srv.poll(t)
        srv.stats(reset=True)
        for rate in rates:
            n = int(rate * duration)
            arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n))
            choice_L = rng.integers(0, len(keys), size=n)
            choice_k = rng.integers(0, len(kinds), size=n)
            choice_q = rng.integers(0, 64, size=n)
            tickets = []
            t0 = time.perf_counter()
            for i in range(n):
                while time.perf_counter() - t0 < arrivals[i]:
                    pass
                L = keys[choice_L[i]]
                t = srv.submit(sids[L], params[kinds[choice_k[i]]], qpool[L][choice_q[i]])
                if t is not None:
                    tickets.append(t)
            srv.drain(600000)
            t_end = time.perf_counter() - t0
            for t in tickets:
                srv.poll(t)
            st = srv.stats(reset=True)
            out[str(rate)] = {"offered_per_s": n / arrivals[-1], "admitted": st["submitted"], "rejected": st["rejected"],
                              "completed_per_s": st["completed"] / t_end, "p50_ms": st["lat_p50_ms"],
                              "p99_ms": st["lat_p99_ms"], "batches": st["batches"]}
        # Per-set capacity, closed loop: M queries of one set (distances in
        # turn) submitted as fast as admission allows, against the same
        # queries as one eap_nn1 launch each (synchronised, plain EAPruned).
        per_set = {}
        import torch
        gsets = {L: eap.SeriesSet.from_packed(p) for L, p in refsets.items()}
        m_of = {128: 192, 256: 192, 512: 96, 1024: 48, 2048: 24, 4096: 12, 8192: 6, "mixed": 192}
        for L in keys:
            m = m_of.get(L, 24)
            qs = [(kinds[i % len(kinds)], qpool[L][i % 64]) for i in range(m)]
            srv.stats(reset=True)
            t0 = time.perf_counter()
            tickets = []
            for kind, q in qs:
                while True:
                    t = srv.submit(sids[L], params[kind], q)
                    if t is not None:
                        break
                    time.sleep(0.0002)
                tickets.append(t)
            srv.drain(600000)
            served = m / (time.perf_counter() - t0)
            for t in tickets:
                srv.poll(t)
            st = srv.stats(reset=True)
            singles = [(params[kind], eap.SeriesSet.from_matrix(q[None, :])) for kind, q in qs]
            for p1, Q1 in singles[:6]:
                eap.eap_nn1(p1, Q1, gsets[L])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for p1, Q1 in singles:
                eap.eap_nn1(p1, Q1, gsets[L])
                torch.cuda.synchronize()
            single = m / (time.perf_counter() - t0)
            per_set[str(L)] = {"queries": m, "served_per_s": served, "one_launch_per_query_per_s": single,
                               "speedup": served / single, "batches": st["batches"],
                               "p50_ms": st["lat_p50_ms"], "p99_ms": st["lat_p99_ms"]}
    best = max(v["completed_per_s"] for v in out.values())
    # One launch per query (plain eap_nn1 on one query at a time) on the same
    # mix of sets and distances, as the baseline for batching.
    rng2 = np.random.default_rng(9)
    sample = [(keys[int(rng2.integers(0, len(keys)))], kinds[int(rng2.integers(0, len(kinds)))],
               int(rng2.integers(0, 64))) for _ in range(96)]
    singles = [(params[k], eap.SeriesSet.from_matrix(qpool[L][q:q + 1]), gsets[L]) for L, k, q in sample]
    for p, Q1, R in singles[:6]:
        eap.eap_nn1(p, Q1, R)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for p, Q1, R in singles:
        eap.eap_nn1(p, Q1, R)
    torch.cuda.synchronize()
    single_qps = len(singles) / (time.perf_counter() - t0)
    return {"metric": "served 1-NN queries/s with p50/p99 latency (8 resident sets, Poisson arrivals)",
            "value": best, "unit": "queries/s", "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serving_8_sets", "sizes": {str(k): v for k, v in sizes.items()},
                       "duration_s_per_rate": duration, "max_inflight": 128}, "per_rate": out,
            "one_launch_per_query": {"value": single_qps, "unit": "queries/s", "sample_queries": len(singles)},
            "speedup_vs_one_launch_per_query": best / single_qps, "per_set_closed_loop": per_set}


def run_other_workload(args):
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    from paper_2102_05221_gb300 import eap
    eap.load()
    fn = {"unpruned_512": workload_unpruned_512, "modes_512": workload_modes_512, "subseq": workload_subseq,
          "allpairs_4096": workload_allpairs_4096, "nn1_8192": workload_nn1_8192,
          "uneven_64": workload_uneven_64, "serving": workload_serving, "lb_cascade": workload_lb_cascade}[args.workload]
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    line = fn(args)
    line["clocks"] = sampler.stop()
    line.setdefault("n_gpus", 1)
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
