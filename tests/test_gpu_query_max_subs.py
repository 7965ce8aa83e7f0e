"""Each query with its own maxSubs on the streaming path.

The paper runs with one maxSubs for the whole query set (Methods, Algorithm
Design).  ifa_set_query_max_subs gives every query its own: query i reports
exactly the windows the paper's rule reports for maxSubs = s_i.  So the
expected hits are the union over queries of the oracle run on that query
alone at its own value, relabelled to its id; in indexed mode each query's
k and MinHits are the oracle's choice for (L_i, s_i).  Every streaming path
is covered: both brute-force kernels, the clip pass, indexed mode, AUTO,
a change between segments, and the way back to a single value."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import to_mem, tuples
from test_gpu_clip import _workload as _clip_workload

pytestmark = pytest.mark.gpu

TRIALS = 10_000


def _relabel(h, qid):
    h = h.copy()
    h["query"] = qid
    return h


def _cat(parts):
    return P.sort_hits(np.concatenate(parts)) if parts else np.zeros(0, P.HIT_DTYPE)


def _expected(queries, ref, contig_len, svec, mode=P.IFA_MODE_BRUTE, clip_pct=0, contig_ids=None):
    parts = []
    for i, (q, s) in enumerate(zip(queries, svec)):
        if mode == P.IFA_MODE_BRUTE:
            h = oracle.brute([q], ref, contig_len, s, clip_pct=clip_pct, contig_ids=contig_ids)
        else:
            st, k, m = oracle.choose_k(len(q), s, trials=TRIALS)
            h = oracle.indexed([q], ref, contig_len, s, [k], [m], [1 if st < 0 else 0], clip_pct=clip_pct,
                               contig_ids=contig_ids)
        parts.append(_relabel(h, i))
    return _cat(parts)


def _run(queries, wl, svec, mode=P.IFA_MODE_BRUTE, seg=1 << 15, mem="host", **cfg):
    h = P.ifa_create(hit_capacity=1 << 22, segment_bytes=1 << 20, minhits_trials=TRIALS, **cfg)
    try:
        P.ifa_load_queries(h, queries)
        P.ifa_set_max_subs(h, 99)      # replaced by the per-query values below
        P.ifa_set_query_max_subs(h, svec)
        P.ifa_set_mode(h, mode)
        keep = []
        for a, b, pc in P.segment_pieces(wl.contig_len, seg):
            buf = to_mem(wl.ref[a:b], mem)
            keep.append(buf)
            P.ifa_push_segment(h, buf, pc)
        P.ifa_flush(h)
        hits, over = P.ifa_drain_hits(h)
        assert not over
        plan = P.ifa_get_query_plan(h, len(queries)) if mode == P.IFA_MODE_INDEXED else None
        return P.sort_hits(hits), P.ifa_get_stats(h), plan
    finally:
        P.ifa_destroy(h)


def _workload(seed):
    return synth.small_workload(seed=seed, n_queries=8, lmin=12, lmax=60, n_contigs=20, cmin=1, cmax=6000,
                                plant_ks=[0, 1, 2, 3, 4, 6, 8] * 2, lowercase_frac=0.05)


SVEC = [0, 3, 1, 8, 2, 5, 0, 12]


@pytest.mark.parametrize("kernel,mem,seg", [(P.IFA_BRUTE_POPC, "host", 1 << 15), (P.IFA_BRUTE_POPC, "device", 777),
                                            (P.IFA_BRUTE_TENSOR, "pinned", 1 << 14)])
def test_brute_force_each_query_at_its_own_threshold(kernel, mem, seg):
    wl = _workload(301)
    got, stats, _ = _run(wl.queries, wl, SVEC, seg=seg, mem=mem, brute_kernel=kernel)
    exp = _expected(wl.queries, wl.ref, wl.contig_len, SVEC)
    assert len(exp) > 0
    # the thresholds matter: the queries at 0 miss the planted 1..8-substitution copies
    assert (exp["mismatches"] > 3).any()
    assert tuples(got) == tuples(exp)
    for i, s in enumerate(SVEC):
        assert (got["mismatches"][got["query"] == i] <= s).all()


def test_values_at_and_above_32_and_255():
    """maxSubs >= 32 takes the generic path for its entries only; 255 (and
    anything above, clamped) reports every valid window of its query."""
    wl = synth.small_workload(seed=302, n_queries=3, lmin=20, lmax=40, n_contigs=6, cmin=10, cmax=700,
                              plant_ks=[0, 1, 2])
    svec = [2, 33, 1000]
    got, _, _ = _run(wl.queries, wl, svec, brute_kernel=P.IFA_BRUTE_POPC)
    exp = _expected(wl.queries, wl.ref, wl.contig_len, [2, 33, 255])
    assert tuples(got) == tuples(exp)
    assert (got["query"] == 2).sum() > (got["query"] == 0).sum()


def test_clip_pass_each_query_at_its_own_threshold():
    wl = _clip_workload(303)         # copies overhanging contig ends planted
    svec = [1, 0, 4, 2, 6, 3]
    got, _, _ = _run(wl.queries, wl, svec, clip_pct=25, brute_kernel=P.IFA_BRUTE_POPC)
    exp = _expected(wl.queries, wl.ref, wl.contig_len, svec, clip_pct=25)
    assert (exp["clips"] != 0).any()
    assert sorted(zip(*(got[f].tolist() for f in ("query", "contig", "pos", "strand", "mismatches", "clips")))) == \
        sorted(zip(*(exp[f].tolist() for f in ("query", "contig", "pos", "strand", "mismatches", "clips"))))


def test_indexed_mode_plans_each_query_for_its_own_threshold():
    wl = synth.small_workload(seed=304, n_queries=6, lmin=24, lmax=60, n_contigs=16, cmin=100, cmax=8000,
                              plant_ks=[0, 1, 2, 3, 4] * 2)
    svec = [0, 4, 1, 3, 2, 8]
    got, _, (k, m, ex) = _run(wl.queries, wl, svec, mode=P.IFA_MODE_INDEXED)
    for i, (q, s) in enumerate(zip(wl.queries, svec)):
        st, ko, mo = oracle.choose_k(len(q), s, trials=TRIALS)
        assert int(ex[i]) == (1 if st < 0 else 0)
        if st >= 0:
            assert (int(k[i]), int(m[i])) == (ko, mo)
    exp = _expected(wl.queries, wl.ref, wl.contig_len, svec, mode=P.IFA_MODE_INDEXED)
    assert len(exp) > 0
    assert tuples(got) == tuples(exp)


def test_auto_mode_takes_the_per_query_values():
    """AUTO picks a mode for the per-query costs; the hits are the oracle's
    for whichever mode it reports."""
    wl = _workload(305)
    got, stats, _ = _run(wl.queries, wl, SVEC, mode=P.IFA_MODE_AUTO)
    mode = stats["mode"]
    assert mode in (P.IFA_MODE_BRUTE, P.IFA_MODE_INDEXED)
    exp = _expected(wl.queries, wl.ref, wl.contig_len, SVEC, mode=mode)
    assert tuples(got) == tuples(exp)


def test_change_between_segments_and_back_to_one_value():
    """Values set between two pushes apply to the second; ifa_set_max_subs
    (and a NULL array) go back to one value for every query."""
    wl = _workload(306)
    nc = len(wl.contig_len)
    cut = nc // 2
    starts = np.concatenate([[0], np.cumsum(wl.contig_len)])
    a_len, b_len = wl.contig_len[:cut], wl.contig_len[cut:]
    ref_a, ref_b = wl.ref[:starts[cut]], wl.ref[starts[cut]:]
    ids_b = np.arange(cut, nc, dtype=np.uint32)
    s1, s2 = [4, 0, 2, 1, 3, 0, 6, 1], [0, 5, 1, 4, 0, 2, 1, 8]
    h = P.ifa_create(hit_capacity=1 << 22, segment_bytes=1 << 20, brute_kernel=P.IFA_BRUTE_POPC)
    try:
        P.ifa_load_queries(h, wl.queries)
        P.ifa_set_query_max_subs(h, s1)
        for a, b, pc in P.segment_pieces(a_len, 1 << 14):
            P.ifa_push_segment(h, ref_a[a:b], pc)
        P.ifa_set_query_max_subs(h, s2)
        for a, b, pc in P.segment_pieces(b_len, 1 << 14, ids_b):
            P.ifa_push_segment(h, ref_b[a:b], pc)
        P.ifa_flush(h)
        got, over = P.ifa_drain_hits(h)
        assert not over
        exp = _cat([_expected(wl.queries, ref_a, a_len, s1),
                    _expected(wl.queries, ref_b, b_len, s2, contig_ids=ids_b)])
        assert tuples(P.sort_hits(got)) == tuples(exp)

        # back to one value: a NULL array, then ifa_set_max_subs
        P.ifa_reset_results(h)
        P.ifa_set_max_subs(h, 3)
        P.ifa_set_query_max_subs(h, s1)
        P.ifa_set_query_max_subs(h, None)
        for a, b, pc in P.segment_pieces(a_len, 1 << 14):
            P.ifa_push_segment(h, ref_a[a:b], pc)
        P.ifa_flush(h)
        got, _ = P.ifa_drain_hits(h)
        assert tuples(P.sort_hits(got)) == tuples(oracle.brute(wl.queries, ref_a, a_len, 3))
    finally:
        P.ifa_destroy(h)


def test_argument_errors():
    h = P.ifa_create(hit_capacity=1 << 16, segment_bytes=1 << 20)
    try:
        P.ifa_load_queries(h, [b"ACGTACGTAC", b"TTTTGGGGCC"])
        with pytest.raises(P.IfaError):
            P.ifa_set_query_max_subs(h, [1, 2, 3])      # one value per loaded query
        P.ifa_set_query_max_subs(h, [1, 2])
    finally:
        P.ifa_destroy(h)
    # query sets carry their own maxSubs: per-query values are refused there
    h = P.ifa_create(hit_capacity=1 << 16, segment_bytes=1 << 20)
    try:
        P.ifa_set_add(h, [b"ACGTACGTAC"], 2, P.IFA_MODE_BRUTE)
        with pytest.raises(P.IfaError):
            P.ifa_set_query_max_subs(h, [1])
    finally:
        P.ifa_destroy(h)
