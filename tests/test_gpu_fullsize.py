"""Parity at the benchmark's full size and launch configuration.

The 4 Gbp, 10-query workload is scanned exactly as bench.py times it
(device-resident ASCII, 256 MB segments, brute force) at every maxSubs of
the sweep.  The oracle cannot scan 4 Gbp in test time, so it checks:
  * every hit on a sample of contigs -- the first ones, the contigs that
    straddle each 256 MB segment boundary (the halo path) and a seeded
    random draw -- against the oracle run on those contigs alone;
  * every planted hit with k <= maxSubs;
  * a random sample of all reported hits, recounted one by one;
  * digest count = drained hits, per-query counts add up."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import tuples

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SEG = 256 << 20


@pytest.fixture(scope="module")
def wl4g():
    return synth.workload_4gbp()


def _sample_contigs(wl, rng):
    starts = wl.contig_start
    ends = starts + wl.contig_len
    pick = set(range(12))
    for b in range(SEG, int(ends[-1]), SEG):   # contigs that straddle a segment boundary
        i = int(np.searchsorted(ends, b, side="right"))
        pick.update(j for j in (i - 1, i, i + 1) if 0 <= j < len(ends))
    pick.update(rng.choice(len(ends), size=30, replace=False).tolist())
    return np.array(sorted(pick))


def test_4gbp_sweep_sampled_parity(wl4g):
    import torch
    wl = wl4g
    rng = np.random.default_rng(5)
    sample = _sample_contigs(wl, rng)
    starts = wl.contig_start
    ref_dev = torch.from_numpy(wl.ref).cuda()
    h = P.ifa_create(hit_capacity=1 << 28, segment_bytes=SEG)
    try:
        P.ifa_load_queries(h, wl.queries)
        for s in (0, 4, 8, 16):
            P.ifa_reset_results(h)
            P.ifa_set_max_subs(h, s)
            for a, b, pc in P.segment_pieces(wl.contig_len, SEG):
                P.ifa_push_segment(h, ref_dev[a:b], pc)
            hits, over = P.ifa_drain_hits(h)
            dig, counts = P.ifa_get_digest(h, len(wl.queries))
            assert not over
            assert dig[0] == hits.size
            assert int(counts.sum()) == hits.size
            # sampled contigs: exact equality with the oracle
            sub_ref = np.concatenate([wl.contig(int(c)) for c in sample])
            exp = oracle.brute(wl.queries, sub_ref, wl.contig_len[sample], s, contig_ids=sample,
                               threads=16)
            mine = hits[np.isin(hits["contig"], sample)]
            assert tuples(mine) == tuples(exp), s
            # planted hits
            have = set(tuples(hits))
            for p in wl.plants:
                if p.k <= s:
                    assert (p.query, p.contig, p.pos, p.strand, p.k) in have
            # every sampled hit recounts to its reported mismatches
            idx = rng.choice(hits.size, size=min(20000, hits.size), replace=False)
            for hh in hits[idx]:
                mm = oracle.window_mismatches(wl.queries[hh["query"]], int(hh["strand"]),
                                              wl.contig(int(hh["contig"])), int(hh["pos"]))
                assert mm == hh["mismatches"] and mm <= s
    finally:
        P.ifa_destroy(h)
