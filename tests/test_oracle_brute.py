"""Pins for the oracle's brute-force scan, each against something other than
the oracle itself: a library Hamming distance (scipy), a library substring
search (re), closed-form window counts, planted hits with a known number of
substitutions, reverse-complement symmetry and monotonicity in maxSubs.

The definition pinned is the brute-force mode of Methods, "Algorithm
Design" (every start position, both strands) with the Hamming metric of
the introduction; N (any byte other than A/C/G/T in either case) mismatches
everything."""
import re

import numpy as np
import pytest
from numpy.lib.stride_tricks import sliding_window_view
from scipy.spatial.distance import cdist

import oracle
import synth

# Independent coding for the scipy pin: bases 0..3 (either case); any other
# byte becomes a value that equals nothing on the other side.
_Q = np.full(256, 100, np.int16)
_R = np.full(256, 200, np.int16)
for _i, _c in enumerate(b"ACGT"):
    _Q[_c] = _Q[_c + 32] = _i
    _R[_c] = _R[_c + 32] = _i
_RC = bytes.maketrans(b"ACGTacgt", b"TGCAtgca")


def _revcomp_text(q: bytes) -> bytes:
    return q.translate(_RC)[::-1]


def scipy_hits(queries, wl_ref, lens, s):
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    out = []
    for qi, q in enumerate(queries):
        L = len(q)
        for t in (0, 1):
            qq = q if t == 0 else _revcomp_text(q)
            qa = _Q[np.frombuffer(qq, np.uint8)].astype(np.float64)[None, :]
            for c, (a, n) in enumerate(zip(starts, lens)):
                if n < L:
                    continue
                win = sliding_window_view(_R[wl_ref[a:a + n]], L).astype(np.float64)
                d = np.rint(cdist(qa, win, "hamming")[0] * L).astype(np.int64)
                for p in np.nonzero(d <= s)[0]:
                    out.append((qi, c, int(p), t, int(d[p])))
    return sorted(out)


def as_tuples(h):
    return sorted(zip(h["query"].tolist(), h["contig"].tolist(), h["pos"].tolist(),
                      h["strand"].tolist(), h["mismatches"].tolist()))


@pytest.mark.parametrize("seed", [7, 11, 12])
@pytest.mark.parametrize("s", [0, 1, 3, 6])
def test_brute_matches_scipy_hamming(seed, s):
    wl = synth.small_workload(seed=seed, n_queries=4, n_contigs=8, cmax=900,
                              lowercase_frac=0.1)
    got = oracle.brute(wl.queries, wl.ref, wl.contig_len, s)
    assert as_tuples(got) == scipy_hits(wl.queries, wl.ref, wl.contig_len, s)


def test_brute_with_n_in_query():
    # a query holding N and an IUPAC code: those positions always mismatch
    q = [b"ACGTNACGTR", b"acgtacgtac"]
    ref = np.frombuffer(b"ACGTAACGTAACGTNACGTRACGTACGTAC", np.uint8).copy()
    lens = np.array([20, 10])
    for s in range(0, 11):
        got = oracle.brute(q, ref, lens, s)
        assert as_tuples(got) == scipy_hits(q, ref, lens, s)
    # query 0 can never score below its own two N positions
    got = oracle.brute(q, ref, lens, 10)
    assert (got["mismatches"][got["query"] == 0] >= 2).all()


def test_exact_matching_is_substring_search(small_wl):
    wl = small_wl
    got = oracle.brute(wl.queries, wl.ref, wl.contig_len, 0)
    starts = wl.contig_start
    expect = []
    for qi, q in enumerate(wl.queries):
        for t, qq in ((0, q), (1, _revcomp_text(q))):
            if re.search(rb"[^ACGTacgt]", qq):
                continue
            pat = re.compile(b"(?=" + re.escape(qq.upper()) + b")")
            for c, (a, n) in enumerate(zip(starts, wl.contig_len)):
                text = bytes(wl.ref[a:a + n]).upper()
                for m in pat.finditer(text):
                    expect.append((qi, c, m.start(), t, 0))
    assert as_tuples(got) == sorted(expect)


def test_every_window_when_subs_reach_length(small_wl):
    wl = small_wl
    for qi, q in enumerate(wl.queries):
        L = len(q)
        got = oracle.brute([q], wl.ref, wl.contig_len, L)
        n_win = int(sum(max(0, int(n) - L + 1) for n in wl.contig_len))
        assert got.size == 2 * n_win
        # both strands of every window, once each
        assert np.unique(got[["contig", "pos", "strand"]]).size == got.size


def test_planted_hits_present_with_exact_count():
    wl = synth.small_workload(seed=21, n_queries=5, lmin=12, lmax=40, n_contigs=10,
                              cmin=200, cmax=2000, plant_ks=[0, 1, 2, 3, 4, 5, 6, 7] * 3)
    for s in (0, 3, 7):
        got = set(as_tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, s)))
        for p in wl.plants:
            key = (p.query, p.contig, p.pos, p.strand, p.k)
            assert (key in got) == (p.k <= s), (key, s)


def test_reverse_complement_symmetry(small_wl):
    wl = small_wl
    s = 4
    fwd = oracle.brute(wl.queries, wl.ref, wl.contig_len, s)
    rc_ref = np.concatenate([np.frombuffer(_revcomp_text(bytes(wl.contig(i))), np.uint8)
                             for i in range(len(wl.contig_len))]) if len(wl.contig_len) else wl.ref
    rev = oracle.brute(wl.queries, rc_ref, wl.contig_len, s)
    qlen = np.array([len(q) for q in wl.queries])
    mapped = sorted((q, c, int(wl.contig_len[c]) - int(qlen[q]) - p, 1 - t, mm)
                    for (q, c, p, t, mm) in as_tuples(fwd))
    assert mapped == as_tuples(rev)


def test_monotone_in_max_subs(small_wl):
    wl = small_wl
    prev = None
    for s in range(0, 9):
        cur = as_tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, s))
        if prev is not None:
            assert prev == [h for h in cur if h[4] <= s - 1]
        assert all(h[4] <= s for h in cur)
        prev = cur


def test_palindrome_reports_both_strands():
    q = b"ACGCGT"  # its own reverse complement
    ref = np.frombuffer(b"TTACGCGTTT", np.uint8).copy()
    got = as_tuples(oracle.brute([q], ref, [10], 0))
    assert got == [(0, 0, 2, 0, 0), (0, 0, 2, 1, 0)]


def test_short_contigs_and_empty_inputs():
    q = [b"AACCGGTA"]  # not its own reverse complement (TACCGGTT)
    ref = np.frombuffer(b"AACCGGTAACCGGTA", np.uint8).copy()
    # contigs of 7 and 8 bases: only the second can hold the 8 bp query
    got = as_tuples(oracle.brute(q, ref, [7, 8], 0))
    assert got == [(0, 1, 0, 0, 0)]
    assert oracle.brute([], ref, [7, 8], 3).size == 0
    assert oracle.brute(q, np.zeros(0, np.uint8), [], 3).size == 0


def test_window_mismatches_matches_hits(small_wl):
    wl = small_wl
    got = oracle.brute(wl.queries, wl.ref, wl.contig_len, 5)
    for h in got[:200]:
        mm = oracle.window_mismatches(wl.queries[h["query"]], int(h["strand"]),
                                      wl.contig(int(h["contig"])), int(h["pos"]))
        assert mm == h["mismatches"]


def test_thread_count_does_not_change_result(small_wl):
    wl = small_wl
    a = oracle.brute(wl.queries, wl.ref, wl.contig_len, 3, threads=1)
    b = oracle.brute(wl.queries, wl.ref, wl.contig_len, 3, threads=5)
    assert as_tuples(a) == as_tuples(b)


def test_digest_is_order_independent_and_sensitive(small_wl):
    wl = small_wl
    h = oracle.brute(wl.queries, wl.ref, wl.contig_len, 4)
    d = oracle.digest(h)
    assert d[0] == h.size
    rng = np.random.default_rng(0)
    assert oracle.digest(h[rng.permutation(h.size)]) == d
    for field in ("query", "contig", "pos", "strand", "mismatches"):
        h2 = h.copy()
        h2[field][0] += 1
        assert oracle.digest(h2) != d
