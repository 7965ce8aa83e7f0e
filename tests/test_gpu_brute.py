"""Brute-force mode on the GPU, element by element against the oracle.

Integer work, so the bar is bit-exact: the sorted (query, contig, pos,
strand, mismatches) tuples, the digest and the per-query counts must equal
the oracle's on the same seeded inputs."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import gpu_scan, tuples

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", [7, 11])
@pytest.mark.parametrize("s", [0, 2, 5, 9])
@pytest.mark.parametrize("seg_bytes", [None, 777, 4093])
def test_small_matches_oracle(seed, s, seg_bytes):
    wl = synth.small_workload(seed=seed, n_queries=6, lmin=5, lmax=70, n_contigs=14, cmax=2500,
                              lowercase_frac=0.05)
    got, over, dig, counts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, seg_bytes=seg_bytes)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s)
    assert not over
    assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(wl.queries)).tolist()


@pytest.mark.parametrize("mem", ["host", "pinned", "device", "pinned_async"])
def test_memory_kinds_agree(mem):
    wl = synth.small_workload(seed=5, n_queries=4, n_contigs=20, cmax=5000)
    got, *_ = gpu_scan(wl.queries, wl.ref, wl.contig_len, 4, seg_bytes=3001, mem=mem)
    assert tuples(got) == tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, 4))


@pytest.mark.parametrize("lens", [(1, 2, 3), (31, 32, 33), (63, 64, 65), (100, 127, 128, 129),
                                  (200, 255)])
def test_query_length_extremes(lens):
    rng = np.random.default_rng(sum(lens))
    queries = [rng.choice(np.frombuffer(b"ACGT", np.uint8), size=L).astype(np.uint8).tobytes()
               for L in lens]
    wl = synth.small_workload(seed=3, n_queries=1, n_contigs=10, cmin=1, cmax=3000)
    for s in (0, 3, max(lens) // 2):
        got, *_ = gpu_scan(queries, wl.ref, wl.contig_len, s, seg_bytes=1500)
        assert tuples(got) == tuples(oracle.brute(queries, wl.ref, wl.contig_len, s)), s


def test_every_window_when_subs_reach_length():
    wl = synth.small_workload(seed=9, n_queries=3, lmin=4, lmax=12, n_contigs=6, cmax=400)
    s = 12
    got, *_ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, seg_bytes=123)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s)
    assert tuples(got) == tuples(exp)
    assert got.size == 2 * sum(max(0, int(n) - len(q) + 1) for q in wl.queries for n in wl.contig_len)


@pytest.mark.parametrize("mode", [P.IFA_MODE_BRUTE, P.IFA_MODE_INDEXED])
def test_unlimited_max_subs(mode):
    """maxSubs has no upper limit (Methods): 2^32 - 1 must report every
    window, like any value at or above the query length, in both modes."""
    wl = synth.small_workload(seed=19, n_queries=3, lmin=4, lmax=40, n_contigs=6, cmax=400)
    n_win = 2 * sum(max(0, int(n) - len(q) + 1) for q in wl.queries for n in wl.contig_len)
    if mode == P.IFA_MODE_BRUTE:
        exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, 60)
        assert exp.size == n_win
    else:
        # s >= L leaves no error-free k-mer, so every query takes the clamped
        # plan (smallest k, threshold 1) and stays seed-filtered
        plan = [oracle.choose_k(len(q), 255, trials=1000) for q in wl.queries]
        exp = oracle.indexed(wl.queries, wl.ref, wl.contig_len, 255, [p[1] for p in plan],
                             [p[2] for p in plan], [1 if p[0] < 0 else 0 for p in plan])
    for s in (255, 1000, 0xFFFFFFFF):
        got, over, dig, _, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, mode=mode,
                                        seg_bytes=500, minhits_trials=1000)
        assert not over and got.size == dig[0]
        assert tuples(got) == tuples(exp)


def test_one_base_segments_and_tiny_contigs():
    queries = [b"ACGTA", b"GGT", b"TTTTTTTT"]
    rng = np.random.default_rng(1)
    lens = np.array([1, 2, 3, 5, 8, 13, 21, 4, 9], np.int64)
    ref = rng.choice(np.frombuffer(b"ACGT", np.uint8), size=int(lens.sum())).astype(np.uint8)
    for seg in (1, 2, 5):
        got, *_ = gpu_scan(queries, ref, lens, 2, seg_bytes=seg)
        assert tuples(got) == tuples(oracle.brute(queries, ref, lens, 2)), seg


def test_count_only_digest_and_counts():
    wl = synth.small_workload(seed=13, n_queries=5, n_contigs=10, cmax=4000)
    _, _, dig, counts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, 6, count_only=1)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, 6)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=5).tolist()


def test_overflow_keeps_digest_exact():
    wl = synth.small_workload(seed=17, n_queries=4, lmin=6, lmax=10, n_contigs=8, cmax=3000)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, 5)
    cap = exp.size // 3
    got, over, dig, counts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, 5, hit_capacity=cap)
    assert over
    assert got.size == cap
    assert set(tuples(got)) <= set(tuples(exp))
    assert dig == oracle.digest(exp)


@pytest.mark.parametrize("cap,count_only", [(128, 0), (700, 0), (128, 1), (1 << 22, 0)])
def test_event_buffer_too_small_rescans_in_line(cap, count_only):
    """Deferred hits: when a launch's window events overflow the event
    buffer (a single chunk of 128 records here, so any two warps with hits
    overflow it), the expansion kernel scans the range again with the hits
    expanded in line; tuples, digest and counts stay exact, with or without
    hit tuples.  A buffer large enough for every event takes the deferred
    path."""
    wl = synth.small_workload(seed=29, n_queries=5, lmin=8, lmax=40, n_contigs=12, cmin=100, cmax=20000)
    s = 5
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s)
    assert exp.size > 10 * 700   # far more events than the small buffers hold
    got, over, dig, counts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, seg_bytes=1 << 15,
                                         event_capacity=cap, count_only=count_only,
                                         brute_kernel=P.IFA_BRUTE_POPC)
    assert not over
    if not count_only:
        assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(wl.queries)).tolist()


def test_contig_ids_are_the_callers():
    wl = synth.small_workload(seed=19, n_queries=3, n_contigs=7, cmax=2000)
    ids = np.array([3, 10, 11, 40, 41, 1000, 70000], np.int64)
    got, *_ = gpu_scan(wl.queries, wl.ref, wl.contig_len, 3, seg_bytes=999, contig_ids=ids)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, 3, contig_ids=ids)
    assert tuples(got) == tuples(exp)


def test_same_handle_two_passes_and_reset():
    wl = synth.small_workload(seed=23, n_queries=4, n_contigs=9, cmax=3000)
    h = P.ifa_create(hit_capacity=1 << 20, segment_bytes=1 << 16)
    try:
        P.ifa_load_queries(h, wl.queries)
        for s in (1, 4, 0):
            P.ifa_reset_results(h)
            P.ifa_set_max_subs(h, s)
            for a, b, pc in P.segment_pieces(wl.contig_len, 2000):
                P.ifa_push_segment(h, wl.ref[a:b], pc)
            got, _ = P.ifa_drain_hits(h)
            assert tuples(got) == tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, s)), s
    finally:
        P.ifa_destroy(h)


def test_torch_stream_is_used():
    import torch
    wl = synth.small_workload(seed=29, n_queries=3, n_contigs=6, cmax=2000)
    st = torch.cuda.Stream()
    h = P.ifa_create(hit_capacity=1 << 20, segment_bytes=1 << 16)
    try:
        P.ifa_set_stream(h, st)
        P.ifa_load_queries(h, wl.queries)
        P.ifa_set_max_subs(h, 3)
        dev = torch.from_numpy(wl.ref).cuda()
        torch.cuda.synchronize()
        for a, b, pc in P.segment_pieces(wl.contig_len, 1 << 16):
            P.ifa_push_segment(h, dev[a:b], pc)
        got, _ = P.ifa_drain_hits(h)
        assert tuples(got) == tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, 3))
    finally:
        P.ifa_destroy(h)


def test_state_and_argument_errors():
    h = P.ifa_create(hit_capacity=1024, segment_bytes=4096)
    try:
        ref = np.frombuffer(b"ACGTACGTAC", np.uint8).copy()
        with pytest.raises(P.IfaError) as ei:
            P.ifa_push_segment(h, ref, [(0, 0, 0, 10, True)])
        assert ei.value.status == P.IFA_ERR_BAD_STATE
        P.ifa_load_queries(h, [b"ACG"])
        bad = [
            [(0, 0, 0, 9, True)],                          # does not cover
            [(0, 0, 0, 5, False), (1, 0, 5, 5, True)],     # only the last piece may continue
            [(0, 3, 0, 10, True)],                         # new contig not at offset 0
            [(5, 0, 0, 5, True), (5, 0, 5, 5, True)],      # ids must increase
        ]
        for pcs in bad:
            with pytest.raises(P.IfaError) as ei:
                P.ifa_push_segment(h, ref, pcs)
            assert ei.value.status == P.IFA_ERR_INVALID_ARG, pcs
        with pytest.raises(P.IfaError) as ei:
            P.ifa_push_segment(h, np.zeros(5000, np.uint8), [(0, 0, 0, 5000, True)])
        assert ei.value.status == P.IFA_ERR_INVALID_ARG
        P.ifa_push_segment(h, ref, [(7, 0, 0, 10, False)])
        with pytest.raises(P.IfaError) as ei:   # must continue contig 7 at offset 10
            P.ifa_push_segment(h, ref, [(8, 0, 0, 10, True)])
        assert ei.value.status == P.IFA_ERR_INVALID_ARG
        with pytest.raises(P.IfaError) as ei:
            P.ifa_load_queries(h, [b"ACGT"])
        assert ei.value.status == P.IFA_ERR_BAD_STATE
        with pytest.raises(P.IfaError):
            P.ifa_load_queries(h, [b""])
    finally:
        P.ifa_destroy(h)


def test_1mbp_x10_planted():
    """1 query of 20 bp against 10 x 1 Mbp at maxSubs 2 (the small brute-force workload)."""
    wl = synth.workload_1mbp_x10()
    got, over, dig, counts, stats = gpu_scan(wl.queries, wl.ref, wl.contig_len, 2,
                                             segment_bytes=4 << 20, seg_bytes=4 << 20)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, 2, threads=8)
    assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)
    have = set(tuples(got))
    for p in wl.plants:
        assert (p.query, p.contig, p.pos, p.strand, p.k) in have
    assert stats["windows"] == 2 * 10 * (1_000_000 - 20 + 1)


@pytest.mark.parametrize("s", [12, 16])
def test_candidates_staged_across_fast_and_generic_blocks(s):
    """At high maxSubs a third of the hot loop's groups fire and leave
    candidate events in the warp's staging buffer; blocks holding an N or a
    contig start (frequent here) take the generic path and may flush that
    buffer.  Every hit must still equal the oracle's."""
    wl = synth.small_workload(seed=83, n_queries=10, lmin=30, lmax=40, n_contigs=300, cmin=20,
                              cmax=12000, n_frac=0.01, plant_ks=[0, 4, 8, 12, 16] * 4)
    got, over, dig, counts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, seg_bytes=1 << 19,
                                         brute_kernel=P.IFA_BRUTE_POPC, hit_capacity=1 << 22)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s, threads=8)
    assert not over and exp.size > 100
    assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(wl.queries)).tolist()


@pytest.mark.parametrize("lens,s,min_hits", [((44, 60), 22, 1000), ((18, 22), 11, 1000), ((30, 34), 16, 1000),
                                             ((70, 120), 20, 10), ((200, 255), 28, 10)])
def test_candidate_queue_fills_within_a_block(lens, s, min_hits):
    """Word 0 passes in a fifth of the windows or more here, so a lane
    queues several of the 36 entries within one block of 128 windows and the
    warp drains its candidate queue before the block ends (class F entries,
    class M entries with an N or a partial first word, an AT-rich stretch
    that passes everywhere).  The long queries (4 and 8 words, maxSubs up to
    28: word 0 passes almost everywhere, few windows hit) drain with lanes
    on entries of different word counts.  Every hit must equal the
    oracle's."""
    rng = np.random.default_rng(1000 + s)
    wl = synth.small_workload(seed=300 + s, n_queries=16, lmin=lens[0], lmax=lens[1], n_contigs=40, cmin=50,
                              cmax=60000, n_frac=0.002, plant_ks=[0, s // 2, s] * 4)
    ref = wl.ref
    a = int(rng.integers(0, len(ref) - 20000))
    ref[a:a + 20000] = rng.choice(np.frombuffer(b"AT", np.uint8), 20000)
    qs = list(wl.queries)
    qs[3] = qs[3][:5] + b"N" + qs[3][6:]
    qs[7] = bytes(rng.choice(np.frombuffer(b"AT", np.uint8), len(qs[7])))
    qs.append(bytes(rng.choice(np.frombuffer(b"AAT", np.uint8), lens[1])))
    qs.append(b"N" + bytes(rng.choice(np.frombuffer(b"ACGT", np.uint8), lens[0] - 1)))
    got, over, dig, counts, _ = gpu_scan(qs, ref, wl.contig_len, s, seg_bytes=1 << 19,
                                         brute_kernel=P.IFA_BRUTE_POPC, hit_capacity=1 << 23)
    exp = oracle.brute(qs, ref, wl.contig_len, s, threads=8)
    assert not over and exp.size > min_hits
    assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(qs)).tolist()
