"""bench.py's multi-rank host logic on CPU: two gloo ranks, a barrier, the
max-over-ranks timing reduction, the sum of the ranks' work, and the split of
one reference by range (each rank builds only its range, byte for byte that
slice of the whole reference)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, ROOT)
    import bench

    class A:
        pass
    r, w = bench.dist_init(A())
    bench.barrier(w)
    t = bench.allmax(10.0 * (rank + 1), w)
    wl, lo, hi, halo = bench.make_workload(3_000_000, rank, w)
    _, qb = bench.nominal_work(wl, lo=lo, hi=hi)
    qb_all = bench.allsum(qb, w)
    out[rank] = (r, w, t, lo, hi, halo, wl.ref_offset, wl.ref.tobytes(), qb, qb_all)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_split_one_reference():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    import synth
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert sorted(out.keys()) == [0, 1]
    whole = synth.workload_4gbp(total=world * 3_000_000)
    total = int(whole.ref.size)
    _, qb_whole = bench.nominal_work(whole)
    ends = []
    for rank in range(world):
        r, w, t, lo, hi, halo, off, ref, qb, qb_all = out[rank]
        assert (r, w) == (rank, world)
        assert t == 20.0                               # every rank sees the max
        assert qb_all == float(qb_whole)               # the ranks' windows are one pass's windows
        ends.append((lo, hi))
        assert ref == whole.ref[off:hi].tobytes()      # its range (and halo), as in the whole
        if halo is not None:
            assert halo[2] == off and halo[3] == lo and hi > lo
    assert ends[0][0] == 0 and ends[0][1] == ends[1][0] and ends[1][1] == total
    assert out[0][8] + out[1][8] == qb_whole
