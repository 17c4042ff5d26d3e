"""Candidate sharding over world_size-2 gloo ranks on CPU: each rank searches
its slice of the references (here with the oracle), the one exchange step
(min of packed keys) must give the global 1-NN with lowest-index ties; a
rank that fails before the exchange must make the other rank error out, not
hang."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2102_05221_gb300 import shard, synth


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q_out):
    import datetime

    import torch.distributed as dist

    import oracle as O
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
    try:
        ds = synth.make_dataset(41, 9, 40, 3, 515)
        tr = ds.train.copy()
        tr[30] = tr[3]      # an exact duplicate in the other shard: ties must go to index 3
        qs = synth.pack(ds.test)
        qs_dup = synth.pack([ds.train[3]] + list(ds.test))
        p = O.make_params("dtw")

        def local(b, e):
            if mode == "fail" and rank == 1:
                raise RuntimeError("rank 1 fails before the exchange")
            idx, d = O.nn1(p, qs_dup, synth.pack(list(tr[b:e])), nthreads=1)
            return idx, d.astype(np.float32)

        try:
            idx, dist_ = shard.nn1_candidate_sharded(local, len(tr), rank, world)
            q_out.put((rank, "ok", idx.tolist(), dist_.tolist()))
        except Exception as ex:   # the failing rank, and the survivor's timed-out collective
            q_out.put((rank, "error", type(ex).__name__, str(ex)[:200]))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(2):
        r = q.get(timeout=120)
        out[r[0]] = r
    for p in ps:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    return out


def test_pack_unpack_roundtrip_and_order():
    idx = np.array([2, -1, 0, 5], np.int32)
    d = np.array([1.5, np.inf, 0.0, 1.5], np.float32)
    k = shard.pack_nn(idx, d, 10)
    i2, d2 = shard.unpack_nn(k)
    assert list(i2) == [12, -1, 10, 15] and np.array_equal(d2, d)
    # The key orders by distance, then index.
    assert k[0] < k[3] and k[2] < k[0] and k[1] > k[0]
    assert shard.candidate_shard(10, 0, 3) == (0, 3) and shard.candidate_shard(10, 2, 3) == (6, 10)


def test_two_gloo_ranks_give_the_global_1nn():
    import oracle as O
    out = _run("ok")
    ds = synth.make_dataset(41, 9, 40, 3, 515)
    tr = ds.train.copy()
    tr[30] = tr[3]
    qs_dup = synth.pack([ds.train[3]] + list(ds.test))
    idx, d = O.nn1(O.make_params("dtw"), qs_dup, synth.pack(list(tr)), nthreads=2)
    for r in (0, 1):
        assert out[r][1] == "ok", out[r]
        assert out[r][2] == idx.tolist()
        assert np.allclose(out[r][3], d, rtol=1e-6)
    assert out[0][2][0] == 3          # duplicate at 3 and 30: lowest index wins


def test_a_failing_rank_makes_the_other_error_not_hang():
    out = _run("fail")
    assert out[1][1] == "error" and "fails before the exchange" in out[1][3]
    assert out[0][1] == "error"       # the survivor's all_reduce times out or sees the peer close
