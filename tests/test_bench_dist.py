"""bench.py's multi-rank host logic on CPU: two gloo ranks, a barrier, the
max-over-ranks timing reduction, and one reference shard per rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench

    class A:
        pass
    r, w = bench.dist_init(A())
    bench.barrier(w)
    t = bench.allmax(10.0 * (rank + 1), w)
    wl = bench.make_workload(2_000_000, rank)
    out[rank] = (r, w, t, bench.shard_seed(rank), bytes(wl.ref[:64]))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    for rank in range(world):
        r, w, t, seed, head = out[rank]
        assert (r, w) == (rank, world)
        assert t == 20.0                      # every rank sees the max
    assert out[0][3] != out[1][3]             # distinct shards
    assert out[0][4] != out[1][4]
