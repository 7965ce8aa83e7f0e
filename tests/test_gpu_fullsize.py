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


# ------------------------------------------------ indexed mode at full size

TRIALS_1G = 100_000


@pytest.fixture(scope="module")
def wl1g():
    return synth.workload_1gbp_indexed()


def _digest_run(queries, ref, lens, s, ids, drop=None):
    """Count-only indexed pass over the reference (minus contigs `drop`),
    256 MB segments from device memory; returns (digest, per-query counts)."""
    import torch
    keep = np.ones(len(lens), bool)
    if drop is not None:
        keep[drop] = False
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    parts = [ref[starts[i]:starts[i] + lens[i]] for i in np.nonzero(keep)[0]]
    sub = np.concatenate(parts)
    dev = torch.from_numpy(sub).cuda()
    h = P.ifa_create(count_only=1, segment_bytes=SEG, minhits_trials=TRIALS_1G, minhits_seed=1)
    try:
        P.ifa_load_queries(h, queries)
        P.ifa_set_max_subs(h, s)
        P.ifa_set_mode(h, P.IFA_MODE_INDEXED)
        for a, b, pc in P.segment_pieces(lens[keep], SEG, contig_ids=ids[keep]):
            P.ifa_push_segment(h, dev[a:b], pc)
        return P.ifa_get_digest(h, len(queries))
    finally:
        P.ifa_destroy(h)


@pytest.mark.parametrize("s", [4, 8, 16])
def test_1gbp_indexed_digest_difference(wl1g, s):
    wl = wl1g
    ids = np.arange(len(wl.contig_len))
    # the two shortest contigs make an oracle-sized sample
    sample = np.argsort(wl.contig_len)[:2]
    full, cfull = _digest_run(wl.queries, wl.ref, wl.contig_len, s, ids)
    rest, crest = _digest_run(wl.queries, wl.ref, wl.contig_len, s, ids, drop=sample)
    diff = (full[0] - rest[0], (full[1] - rest[1]) % (1 << 64), full[2] ^ rest[2])
    by_len = {L: oracle.choose_k(L, s, trials=TRIALS_1G, seed=1) for L in {len(q) for q in wl.queries}}
    plan = [by_len[len(q)] for q in wl.queries]
    exh = [1 if st < 0 else 0 for st, _, _ in plan]
    sub_ref = np.concatenate([wl.contig(int(c)) for c in sample])
    exp = oracle.indexed(wl.queries, sub_ref, wl.contig_len[sample], s, [p[1] for p in plan],
                         [p[2] for p in plan], exh, contig_ids=sample, threads=16)
    assert diff == oracle.digest(exp)
    assert (cfull - crest).tolist() == np.bincount(exp["query"], minlength=len(wl.queries)).tolist()


def test_1gbp_plan_matches_oracle(wl1g):
    wl = wl1g
    h = P.ifa_create(minhits_trials=TRIALS_1G, minhits_seed=1, segment_bytes=1 << 20, hit_capacity=1024)
    try:
        P.ifa_load_queries(h, wl.queries)
        for s in (4, 8, 16):
            P.ifa_set_max_subs(h, s)
            k, m, ex = P.ifa_get_query_plan(h, len(wl.queries))
            cache = {}
            for i, q in enumerate(wl.queries):
                L = len(q)
                if L not in cache:
                    cache[L] = oracle.choose_k(L, s, trials=TRIALS_1G, seed=1)
                st, kk, mm = cache[L]
                assert (k[i], m[i], ex[i]) == (kk, mm, 1 if st < 0 else 0)
    finally:
        P.ifa_destroy(h)
