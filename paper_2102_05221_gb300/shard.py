"""Multi-GPU sharding of 1-NN search (one process per GPU).

Queries are independent, so sharding by query needs no exchange: each rank
answers its own queries against the whole reference set (this is what
``bench.py --gpus N`` does).  Sharding by candidate needs exactly one
exchange: every rank searches its slice of the references, then the ranks
take, per query, the minimum of the packed key
``(float bits of the distance) << 32 | global candidate index`` -- the same
packing the kernels use for their best-so-far, so the reduction keeps the
smallest distance and, among equal distances, the lowest index (Alg. 1's
strict "<" over candidates in index order).  Distances are >= 0 (or +inf),
so their float bits order like the values and the key fits in a
non-negative int64.

On the GPU the keys never leave the device: ``eap_nn1_keys`` (the library's
1-NN on this rank's slice, packed with global indices) -> one all-reduce MIN
of an int64 tensor (NCCL on device memory; gloo through host memory) ->
``eap_keys_unpack``.  The numpy helpers below are the same packing for host
arrays.
"""
from __future__ import annotations

import numpy as np

NO_INDEX = 0xFFFFFFFF


def candidate_shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous slice [begin, end) of n candidates owned by `rank`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    return (n * rank) // world, (n * (rank + 1)) // world


def pack_nn(idx, dist, offset: int) -> np.ndarray:
    """Local results (index into the shard, -1 = none; float32 distance)
    to int64 keys with global indices."""
    idx = np.asarray(idx, dtype=np.int64)
    d = np.asarray(dist, dtype=np.float32)
    if np.any(d < 0) or np.any(np.isnan(d)):
        raise ValueError("distances must be >= 0 or +inf")
    bits = d.view(np.uint32).astype(np.int64)
    gidx = np.where(idx >= 0, idx + offset, NO_INDEX).astype(np.int64)
    return (bits << 32) | gidx


def unpack_nn(keys):
    keys = np.asarray(keys, dtype=np.int64)
    low = keys & 0xFFFFFFFF
    bits = (keys >> 32).astype(np.uint32)
    dist = bits.view(np.float32).copy()
    idx = np.where(low == NO_INDEX, -1, low).astype(np.int32)
    dist[idx < 0] = np.inf
    return idx, dist


def allreduce_nn(keys: np.ndarray, group=None) -> np.ndarray:
    """The one exchange step: elementwise MIN of the keys over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(keys, dtype=np.int64))
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return t.cpu().numpy()


def nn1_candidate_sharded(local_search, n_refs: int, rank: int, world: int, group=None):
    """Runs ``local_search(begin, end) -> (idx, dist)`` on this rank's slice of
    the references and combines the slices of all ranks."""
    b, e = candidate_shard(n_refs, rank, world)
    idx, dist = local_search(b, e)
    keys = allreduce_nn(pack_nn(idx, dist, b), group)
    return unpack_nn(keys)


def nn1_candidate_sharded_gpu(p, queries, refs_local, index_offset: int, group=None, stream=None):
    """1-NN over the union of every rank's candidate shard, on the product
    path: this rank's shard (``refs_local``, global indices starting at
    ``index_offset``) through eap_nn1_keys, the MIN all-reduce of the keys,
    then eap_keys_unpack.  Returns (idx, dist) device tensors, identical on
    every rank."""
    import torch.distributed as dist

    from . import eap
    keys = eap.eap_nn1_keys(p, queries, refs_local, index_offset, stream=stream)
    if dist.get_backend(group) == "nccl":
        dist.all_reduce(keys, op=dist.ReduceOp.MIN, group=group)
    else:
        if stream is not None:
            stream.synchronize()
        host = keys.cpu()
        dist.all_reduce(host, op=dist.ReduceOp.MIN, group=group)
        keys.copy_(host)
    return eap.eap_keys_unpack(keys, stream=stream)
