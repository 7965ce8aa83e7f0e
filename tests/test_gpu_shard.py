"""One reference split by range over several handles, on one GPU.

The multi-GPU form of the scan gives each GPU one range of the reference
(see tests/test_shard_dist.py for the host logic on gloo ranks).  Here the
ranges run one after the other on one device, each on its own handle: a
range that starts inside a contig is primed with that contig's bases before
it (ifa_prime_halo), then streamed.  The merged hits, digests and per-query
counts must equal one handle's pass over the whole reference -- and the
oracle's -- in brute-force mode (both kernels), with soft clipping, and in
indexed mode.  Cuts fall at contig starts, one base after, just before and
after a query length in, in the middle and one base before a contig end."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import gpu_scan, to_mem, tuples

pytestmark = pytest.mark.gpu


def _tuples6(h):
    return sorted(zip(h["query"].tolist(), h["contig"].tolist(), h["pos"].tolist(),
                      h["strand"].tolist(), h["mismatches"].tolist(), h["clips"].tolist()))


def scan_ranges(queries, ref, lens, s, cuts, mode=P.IFA_MODE_BRUTE, seg=777, mem="host", **cfg):
    lmax = max(len(q) for q in queries)
    hits, dig, counts = [], [0, 0, 0], np.zeros(len(queries), np.uint64)
    for lo, hi in zip(cuts[:-1], cuts[1:]):
        if hi <= lo:
            continue
        h = P.ifa_create(hit_capacity=1 << 20, segment_bytes=1 << 20, **cfg)
        try:
            P.ifa_load_queries(h, queries)
            P.ifa_set_max_subs(h, s)
            P.ifa_set_mode(h, mode)
            halo = P.shard_halo(lens, lo, lmax)
            keep = []
            if halo:
                buf = to_mem(ref[halo[2]:halo[3]], mem)
                keep.append(buf)
                P.ifa_prime_halo(h, halo[0], halo[1], buf)
            for a, b, pc in P.segment_pieces(lens, seg, lo=lo, hi=hi):
                buf = to_mem(ref[a:b], mem)
                keep.append(buf)
                P.ifa_push_segment(h, buf, pc)
            got, over = P.ifa_drain_hits(h)
            assert not over
            d, c = P.ifa_get_digest(h, len(queries))
        finally:
            P.ifa_destroy(h)
        hits.append(got)
        dig = [dig[0] + d[0], (dig[1] + d[1]) % (1 << 64), dig[2] ^ d[2]]
        counts += c
    return P.sort_hits(np.concatenate(hits)), tuple(dig), counts


def _cuts(lens, L):
    starts = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    total = int(starts[-1])
    big = [i for i in range(len(lens)) if lens[i] > 3 * L]
    c1, c2, c3 = big[0], big[len(big) // 2], big[-1]
    pts = {int(starts[c1]), int(starts[c1]) + 1, int(starts[c2]) + L - 2, int(starts[c2]) + L - 1,
           int(starts[c2]) + L, int(starts[c3]) + int(lens[c3]) // 2, int(starts[c3 + 1]) - 1}
    return [0] + sorted(p for p in pts if 0 < p < total) + [total]


@pytest.mark.parametrize("kernel", [P.IFA_BRUTE_POPC, P.IFA_BRUTE_TENSOR])
@pytest.mark.parametrize("mem", ["host", "device"])
def test_ranges_equal_one_pass_brute(kernel, mem):
    wl = synth.small_workload(seed=31, n_queries=40, lmin=12, lmax=60, n_contigs=24, cmin=3,
                              cmax=9000, plant_ks=[0, 1, 2, 3, 4])
    s = 4
    cuts = _cuts(wl.contig_len, 40)
    got, dig, counts = scan_ranges(wl.queries, wl.ref, wl.contig_len, s, cuts, mem=mem, brute_kernel=kernel)
    whole, over, wdig, wcounts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, seg_bytes=777,
                                             brute_kernel=kernel)
    assert not over
    assert tuples(got) == tuples(whole) == tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, s))
    assert dig == wdig
    assert counts.tolist() == wcounts.tolist()


@pytest.mark.parametrize("world", [2, 5])
def test_equal_ranges_with_soft_clipping(world):
    wl = synth.small_workload(seed=37, n_queries=12, lmin=6, lmax=40, n_contigs=30, cmin=2,
                              cmax=3000, plant_ks=[0, 1, 2, 3])
    s = 3
    total = int(wl.contig_len.sum())
    cuts = [P.shard_range(total, world, r)[0] for r in range(world)] + [total]
    # and cuts right after contig starts, so left-clipped windows straddle ranges
    starts = np.concatenate([[0], np.cumsum(wl.contig_len)]).astype(np.int64)
    cuts = sorted(set(cuts) | {int(starts[i]) + 3 for i in range(1, len(starts) - 1, 4)
                               if starts[i] + 3 < starts[i + 1]})
    got, dig, counts = scan_ranges(wl.queries, wl.ref, wl.contig_len, s, cuts, clip_pct=25)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s, clip_pct=25)
    assert _tuples6(got) == _tuples6(exp)
    assert dig == oracle.digest(exp)


def test_ranges_equal_one_pass_indexed():
    wl = synth.small_workload(seed=41, n_queries=30, lmin=18, lmax=40, n_contigs=16, cmin=50,
                              cmax=20000, plant_ks=[0, 1, 2, 3])
    s = 3
    cuts = _cuts(wl.contig_len, 30)
    got, dig, counts = scan_ranges(wl.queries, wl.ref, wl.contig_len, s, cuts, mode=P.IFA_MODE_INDEXED,
                                   minhits_trials=4000)
    whole, over, wdig, wcounts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, mode=P.IFA_MODE_INDEXED,
                                             seg_bytes=777, minhits_trials=4000)
    assert not over
    assert tuples(got) == tuples(whole)
    assert dig == wdig and counts.tolist() == wcounts.tolist()
    plan = [oracle.choose_k(len(q), s, trials=4000) for q in wl.queries]
    exp = oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, [p[1] for p in plan], [p[2] for p in plan],
                         [1 if p[0] < 0 else 0 for p in plan])
    assert tuples(got) == tuples(exp)


def test_prime_halo_errors():
    h = P.ifa_create(hit_capacity=1 << 10, segment_bytes=1 << 16)
    try:
        with pytest.raises(P.IfaError) as ei:
            P.ifa_prime_halo(h, 0, 5, np.frombuffer(b"ACGTACGT", np.uint8).copy())
        assert ei.value.status == P.IFA_ERR_BAD_STATE        # no queries yet
        P.ifa_load_queries(h, [b"ACGTACGTAC"])
        P.ifa_prime_halo(h, 3, 5, np.frombuffer(b"ACGTACGT", np.uint8).copy())
        with pytest.raises(P.IfaError) as ei:
            P.ifa_prime_halo(h, 4, 0, np.frombuffer(b"ACGT", np.uint8).copy())
        assert ei.value.status == P.IFA_ERR_BAD_STATE        # contig 3 still open
        with pytest.raises(P.IfaError) as ei:                # must continue contig 3 at 13
            P.ifa_push_segment(h, np.frombuffer(b"ACGT", np.uint8).copy(), [(3, 12, 0, 4, True)])
        assert ei.value.status == P.IFA_ERR_INVALID_ARG
        P.ifa_push_segment(h, np.frombuffer(b"ACGT", np.uint8).copy(), [(3, 13, 0, 4, True)])
        P.ifa_flush(h)
    finally:
        P.ifa_destroy(h)
