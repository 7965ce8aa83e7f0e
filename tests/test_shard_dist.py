"""Splitting one reference by range over ranks, on CPU: two (and three) gloo
ranks.

The paper splits its work over threads by contig (Methods, "Memory
Management").  Here the reference is split over GPUs by base range, which
may cut a contig: a range that starts inside a contig carries a halo of the
contig's L_max - 1 bases before it, and a window belongs to the range that
holds its last base.  No exchange step is needed: hits concatenate and
digests add.

Each rank takes its range from P.shard_range, the range's pieces from
P.segment_pieces(lo=, hi=) and its halo from P.shard_halo -- the host logic
the benchmark uses under torchrun -- and scans the range with the CPU
oracle: every contig span of the range, widened at the front by the halo
bases, is one oracle contig, a hit counts when its window's last base is in
the rank's range, and positions go back to contig coordinates.  Rank 0
gathers the hits: each of the whole reference's oracle hits must come from
exactly one rank, and the digests must add up to the whole digest."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_hits(wl, s, world, rank):
    import oracle
    import paper_2607_27291_b300 as P
    lens = wl.contig_len
    starts = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    lmax = max(len(q) for q in wl.queries)
    lo, hi = P.shard_range(int(starts[-1]), world, rank)
    halo = P.shard_halo(lens, lo, lmax)
    # the range's pieces (small segments), merged back into one span per contig
    spans = {}
    for a, b, pc in P.segment_pieces(lens, 997, lo=lo, hi=hi):
        for p in pc:
            c = int(p["contig"])
            g0 = a + int(p["start"])
            g1 = g0 + int(p["len"])
            spans[c] = (min(spans.get(c, (g0, g1))[0], g0), max(spans.get(c, (g0, g1))[1], g1))
    out = []
    for c, (g0, g1) in sorted(spans.items()):
        v0 = g0
        if halo is not None and c == halo[0] and g0 == lo:
            assert halo[3] == lo and halo[1] == halo[2] - starts[c]
            v0 = halo[2]
        h = oracle.brute(wl.queries, wl.ref[v0:g1], np.array([g1 - v0]), s, contig_ids=[c])
        last = v0 + h["pos"].astype(np.int64) + np.array([len(wl.queries[q]) for q in h["query"]],
                                                         dtype=np.int64) - 1
        h = h[last >= g0]
        h["pos"] = h["pos"] + (v0 - starts[c])
        out.append(h)
    return oracle.sort_hits(np.concatenate(out)) if out else np.zeros(0, oracle.HIT_DTYPE)


def _worker(rank, world, port, cases, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import oracle
    import synth
    dist.init_process_group("gloo")
    for i, (seed, s) in enumerate(cases):
        # contigs shorter and longer than the queries, so ranges cut contigs
        # near their start, near their end and in the middle
        wl = synth.small_workload(seed=seed, n_queries=5, lmin=6, lmax=30, n_contigs=9, cmin=5,
                                  cmax=700, plant_ks=[0, 1, 2, 3])
        h = _rank_hits(wl, s, world, rank)
        got = [None] * world
        dist.all_gather_object(got, (h.tobytes(), oracle.digest(h)))
        if rank == 0:
            out[i] = got
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_range_shards_partition_the_hits(world):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    cases = [(13, 2), (17, 4), (23, 6)]
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, cases, out), nprocs=world, join=True)
    for i, (seed, s) in enumerate(cases):
        wl = synth.small_workload(seed=seed, n_queries=5, lmin=6, lmax=30, n_contigs=9, cmin=5,
                                  cmax=700, plant_ks=[0, 1, 2, 3])
        exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s)
        parts = [np.frombuffer(b, dtype=oracle.HIT_DTYPE) for b, _ in out[i]]
        merged = oracle.sort_hits(np.concatenate(parts))
        assert merged.tobytes() == exp.tobytes()          # every hit, each exactly once
        cnt = sum(d[0] for _, d in out[i])
        ssum = sum(d[1] for _, d in out[i]) % (1 << 64)
        xr = 0
        for _, d in out[i]:
            xr ^= d[2]
        assert (cnt, ssum, xr) == oracle.digest(exp)
        assert all(len(p) > 0 for p in parts) or exp.size < 4 * world
