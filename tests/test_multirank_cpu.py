"""The bench's multi-rank plumbing on CPU: two gloo ranks (world size 2) take disjoint
instance ids and agree on the max-reduced time, as bench.py does under torchrun."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench._dist()
        ids = bench._instance_ids(r, 5)
        t = bench._max_over_ranks(1.0 + r, w)
        bench._barrier(w)
        out[rank] = (w, r, ids, t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    (w0, r0, ids0, t0), (w1, r1, ids1, t1) = res[0], res[1]
    assert (w0, w1, r0, r1) == (2, 2, 0, 1)
    assert not set(ids0) & set(ids1) and len(ids0) == len(ids1) == 5
    assert t0 == t1 == 2.0
