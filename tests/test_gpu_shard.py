"""Candidate sharding through the product path: two gloo ranks (processes)
share the GPU, each searches its slice of the references with the library
(eap_nn1_keys), the one exchange step is the MIN all-reduce of the packed
keys, and eap_keys_unpack gives every rank the 1-NN over the whole set --
equal to a single eap_nn1 call and to the FP64 oracle (Alg. 1), with an
exact duplicate in the second shard to check that ties go to the lowest
global index.  The kernels of the two ranks never wait on each other."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2102_05221_gb300 import shard, synth

pytestmark = pytest.mark.gpu

KINDS = [("dtw", {}), ("erp", {"window_ratio": 0.2}), ("msm", {})]


def _data():
    ds = synth.make_dataset(57, 11, 64, 3, 909)
    tr = ds.train.copy()
    tr[40] = tr[5]   # exact duplicate in the other shard: ties go to 5
    qs = np.concatenate([ds.train[5:6], ds.test], axis=0)
    return tr, qs


def _worker(rank, world, port, q_out):
    import datetime

    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    try:
        from paper_2102_05221_gb300 import eap
        torch.cuda.set_device(0)
        tr, qs = _data()
        b, e = shard.candidate_shard(len(tr), rank, world)
        Q = eap.SeriesSet.from_matrix(qs)
        R = eap.SeriesSet.from_matrix(tr[b:e])
        res = {}
        for kind, kw in KINDS:
            idx, d = shard.nn1_candidate_sharded_gpu(eap.params(kind, **kw), Q, R, b)
            res[kind] = (idx.cpu().numpy().tolist(), d.cpu().numpy().tolist())
        q_out.put((rank, "ok", res))
    except Exception as ex:
        q_out.put((rank, "error", repr(ex)[:300]))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_two_ranks_on_the_product_path_give_the_global_1nn():
    import oracle as O
    from paper_2102_05221_gb300 import eap
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(2):
        r = q.get(timeout=300)
        out[r[0]] = r
    for p in ps:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    tr, qs = _data()
    Q, R = eap.SeriesSet.from_matrix(qs), eap.SeriesSet.from_matrix(tr)
    for kind, kw in KINDS:
        i1, d1 = eap.eap_nn1(eap.params(kind, **kw), Q, R)
        i1, d1 = i1.cpu().numpy(), d1.cpu().numpy()
        oi, od = O.nn1(O.make_params(kind, **kw), synth.pack(list(qs)), synth.pack(list(tr)))
        for rank in (0, 1):
            assert out[rank][1] == "ok", out[rank]
            idx, d = out[rank][2][kind]
            assert idx == i1.tolist(), (kind, rank)
            assert np.array_equal(np.asarray(d, np.float32), d1), (kind, rank)
            assert idx == oi.tolist(), (kind, rank)
            assert np.allclose(d, od, rtol=1e-4), (kind, rank)
        assert out[0][2][kind][0][0] == 5   # duplicate at 5 and 40: the lowest global index


def test_keys_pack_and_unpack_on_the_device():
    import torch

    from paper_2102_05221_gb300 import eap
    tr, qs = _data()
    Q, R = eap.SeriesSet.from_matrix(qs), eap.SeriesSet.from_matrix(tr[10:30])
    p = eap.params("dtw")
    keys = eap.eap_nn1_keys(p, Q, R, 10)
    idx, d = eap.eap_nn1(p, Q, R)
    k = keys.cpu().numpy()
    assert np.array_equal((k & 0xFFFFFFFF).astype(np.int64), idx.cpu().numpy().astype(np.int64) + 10)
    assert np.array_equal(((k >> 32).astype(np.uint32)).view(np.float32), d.cpu().numpy())
    i2, d2 = eap.eap_keys_unpack(keys)
    assert np.array_equal(i2.cpu().numpy(), idx.cpu().numpy() + 10)
    assert torch.equal(d2, d)
    # An empty shard says "none" for every query; an offset that would reach
    # the "none" index is rejected.
    E = eap.SeriesSet.from_matrix(tr[:0])
    ke = eap.eap_nn1_keys(p, Q, E, 57)
    ie, de = eap.eap_keys_unpack(ke)
    assert (ie.cpu().numpy() == -1).all() and np.isinf(de.cpu().numpy()).all()
    with pytest.raises(eap.EapError):
        eap.eap_nn1_keys(p, Q, R, 0xFFFFFFFF - 5)
