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


# ------------------------------- device-resident stores past 2^32 bases

def _append_counter_contigs(h, ref, keep=None, chunk=256 << 20):
    """Append the contigs of a synth.CounterReference (those with keep[i],
    default all) to the handle's store, each 256 MB chunk generated on the
    device; contig ids stay the reference's."""
    import torch
    from synth.devgen import DeviceFiller
    lens = ref.contig_len
    keep = np.ones(len(lens), bool) if keep is None else keep
    ids = np.nonzero(keep)[0]
    klens = lens[ids]
    ost = ref.contig_start[ids]                                  # original starts
    rst = np.concatenate([[0], np.cumsum(klens)[:-1]]).astype(np.int64)   # starts in the store
    fill = DeviceFiller(ref)
    P.ifa_ref_reserve(h, int(klens.sum()))
    buf = torch.empty(chunk, dtype=torch.uint8, device="cuda")
    for ra, rb, pc in P.segment_pieces(klens, chunk, contig_ids=ids):
        j = int(np.searchsorted(rst, ra, side="right")) - 1
        x = ra
        while x < rb:
            end = min(rb, int(rst[j] + klens[j]))
            fill.fill(buf[x - ra:end - ra], int(ost[j] + (x - rst[j])))
            x = end
            j += 1
        torch.cuda.synchronize()
        P.ifa_ref_append(h, buf[:rb - ra], pc)
    torch.cuda.synchronize()


def _sets(n, seed):
    sets = synth.query_sets(n, 1, 5000, 18, 50, 12, seed)
    return [(qs, s, P.IFA_MODE_BRUTE if len(qs) < 150 else P.IFA_MODE_INDEXED) for qs, s in sets]


def _batch_digest(ref, sets, keep=None):
    h = P.ifa_create(count_only=1, segment_bytes=256 << 20, minhits_trials=TRIALS_1G, minhits_seed=1)
    try:
        _append_counter_contigs(h, ref, keep)
        for qs, s, mode in sets:
            P.ifa_set_add(h, qs, s, mode)
        res = P.ifa_batch_run(h, P.IFA_BATCH_PERSISTENT, len(sets))
        assert [int(m) for m in res["mode"]] == [m for _, _, m in sets]
        return P.ifa_get_digest(h, sum(len(qs) for qs, _, _ in sets))
    finally:
        P.ifa_destroy(h)


def test_16gbp_store_batch_digest_difference():
    """The batched workload's store (16 Gbp: past 2^32 bases, so store
    offsets need 64 bits), 32 query sets (sizes log-uniform 1-5000, 18-50 bp,
    maxSubs 0-12; brute force below 150 queries, indexed above) in one
    persistent launch, count only.  Dropping three sampled contigs -- the
    two shortest and the shortest one starting past base 2^32 -- must change
    the digest and the per-query counts by exactly the oracle's hits on
    them."""
    ref = synth.sets_reference(16_000_000_000)
    assert ref.total > (1 << 32)
    st = ref.contig_start
    far = np.nonzero(st > (1 << 32) + (1 << 20))[0]
    sample = sorted(set(np.argsort(ref.contig_len)[:2].tolist()) |
                    {int(far[np.argmin(ref.contig_len[far])])})
    sets = _sets(32, 4)
    full, cfull = _batch_digest(ref, sets)
    keep = np.ones(len(ref.contig_len), bool)
    keep[sample] = False
    rest, crest = _batch_digest(ref, sets, keep)
    diff = (full[0] - rest[0], (full[1] - rest[1]) % (1 << 64), full[2] ^ rest[2])
    sub = np.concatenate([ref.bases(int(st[c]), int(st[c] + ref.contig_len[c])) for c in sample])
    lens = ref.contig_len[sample]
    parts, first = [], 0
    for qs, s, mode in sets:
        if mode == P.IFA_MODE_BRUTE:
            e = oracle.brute(qs, sub, lens, s, contig_ids=sample, threads=16)
        else:
            by_len = {L: oracle.choose_k(L, s, trials=TRIALS_1G, seed=1) for L in {len(q) for q in qs}}
            plan = [by_len[len(q)] for q in qs]
            e = oracle.indexed(qs, sub, lens, s, [p[1] for p in plan], [p[2] for p in plan],
                               [1 if p[0] < 0 else 0 for p in plan], contig_ids=sample, threads=16)
        e = e.copy()
        e["query"] += first
        parts.append(e)
        first += len(qs)
    exp = np.concatenate(parts)
    assert diff == oracle.digest(exp)
    assert (cfull - crest).tolist() == np.bincount(exp["query"], minlength=first).tolist()


def test_200gbp_serving_store_sampled_parity():
    """The serving workload's store at its stated size: 200 Gbp generated on
    the device into the 2-bit store (about 50 GB of HBM).  Two requests
    served by continuous batching for a full cycle; their hits on sampled
    contigs (the three shortest and five seeded others up to 200 kbp,
    regenerated on the host) equal the oracle's, and their digests count
    every hit drained."""
    import torch
    ref = synth.serving_reference(200_000_000_000)
    h = P.ifa_create(hit_capacity=1024, segment_bytes=256 << 20, minhits_trials=TRIALS_1G, minhits_seed=1)
    try:
        free0, _ = torch.cuda.mem_get_info()
        _append_counter_contigs(h, ref)
        used = free0 - torch.cuda.mem_get_info()[0]
        assert used < 0.27 * ref.total                   # 2 bits per base plus the sparse tables
        rq = [(synth.random_queries(4, 24, 30, 91), 3), (synth.random_queries(3, 28, 34, 92), 5)]
        P.ifa_serve_start(h, 16, 8 << 30, 1 << 22)
        ids = [P.ifa_serve_submit(h, qs, s, P.IFA_MODE_AUTO) for qs, s in rq]
        while P.ifa_serve_step(h)[0]:     # both are admitted at the first step
            pass
        rng = np.random.default_rng(17)
        small = np.nonzero(ref.contig_len <= 200_000)[0]
        sample = sorted(set(np.argsort(ref.contig_len)[:3].tolist()) |
                        set(rng.choice(small, size=5, replace=False).tolist()))
        st = ref.contig_start
        sub = np.concatenate([ref.bases(int(st[c]), int(st[c] + ref.contig_len[c])) for c in sample])
        for rid, (qs, s) in zip(ids, rq):
            info = P.ifa_serve_poll(h, rid)
            assert info["state"] == 2 and not info["overflowed"]
            assert info["mode"] == P.IFA_MODE_BRUTE      # the measured rates pick brute force for 3-4 queries
            hits, over = P.ifa_serve_drain(h, rid, 1 << 22)
            assert not over and hits.size == info["digest"][0] == info["hits"]
            mine = P.sort_hits(hits[np.isin(hits["contig"], sample)])
            exp = oracle.brute(qs, sub, ref.contig_len[sample], s, contig_ids=sample, threads=16)
            assert tuples(mine) == tuples(exp)
        P.ifa_serve_stop(h)
    finally:
        P.ifa_destroy(h)
