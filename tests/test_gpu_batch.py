"""Many query sets against a device-resident reference (batching).

Every set -- brute force, indexed or left to the autotuner, each with its
own maxSubs -- must report exactly the oracle's hits for its queries, and
the persistent (graph-replayed) run and the one-set-at-a-time run must agree
tuple for tuple."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import tuples

pytestmark = pytest.mark.gpu

TRIALS = 20_000


def _store(h, wl, append_bytes):
    """Append the reference in chunks of append_bytes (a multiple of 32),
    cutting contigs across appends."""
    for a, b, pc in P.segment_pieces(wl.contig_len, append_bytes):
        P.ifa_ref_append(h, wl.ref[a:b], pc)


def _oracle_set(wl, queries, s, mode):
    if mode == P.IFA_MODE_BRUTE:
        return oracle.brute(queries, wl.ref, wl.contig_len, s)
    plan = [oracle.choose_k(len(q), s, trials=TRIALS) for q in queries]
    exh = [1 if st < 0 else 0 for st, _, _ in plan]
    return oracle.indexed(queries, wl.ref, wl.contig_len, s, [p[1] for p in plan],
                          [p[2] for p in plan], exh)


def _shift(h, first):
    h = h.copy()
    h["query"] += first
    return h


@pytest.mark.parametrize("append_bytes", [1 << 16, 4096])
def test_sets_match_oracle_and_kinds_agree(append_bytes):
    wl = synth.small_workload(seed=71, n_queries=2, lmin=18, lmax=50, n_contigs=30, cmin=50,
                              cmax=8000, plant_ks=[0, 1, 2, 3, 4, 5] * 3)
    specs = [  # (n queries, maxSubs, mode)
        (1, 0, P.IFA_MODE_BRUTE), (3, 4, P.IFA_MODE_INDEXED), (7, 2, P.IFA_MODE_AUTO),
        (2, 6, P.IFA_MODE_BRUTE), (40, 3, P.IFA_MODE_AUTO), (12, 5, P.IFA_MODE_INDEXED),
        (5, 1, P.IFA_MODE_AUTO),
    ]
    sets = []
    for i, (n, s, mode) in enumerate(specs):
        qs = synth.random_queries(n, 10 if i % 2 else 18, 50, 100 + i)
        sets.append((qs, s, mode))
    # the workload's planted queries go into two of the sets
    sets[1] = ([wl.queries[0]] + sets[1][0][1:], sets[1][1], sets[1][2])
    sets[4] = (sets[4][0][:-1] + [wl.queries[1]], sets[4][1], sets[4][2])
    # both kinds on one handle: the autotuner's choices (from measured rates)
    # are made once and shared
    results = {}
    h = P.ifa_create(hit_capacity=1 << 22, segment_bytes=1 << 20, minhits_trials=TRIALS)
    try:
        _store(h, wl, append_bytes)
        firsts = []
        for qs, s, mode in sets:
            sid, first = P.ifa_set_add(h, qs, s, mode)
            firsts.append(first)
        for kind in (P.IFA_BATCH_PERSISTENT, P.IFA_BATCH_PER_SET):
            P.ifa_reset_results(h)
            res = P.ifa_batch_run(h, kind, len(sets))
            hits, over = P.ifa_drain_hits(h)
            assert not over
            results[kind] = (P.sort_hits(hits), res, firsts)
            # a second run of the same batch (graph replay) gives the same hits again
            P.ifa_reset_results(h)
            P.ifa_batch_run(h, kind, len(sets))
            again, _ = P.ifa_drain_hits(h)
            assert tuples(again) == tuples(hits)
    finally:
        P.ifa_destroy(h)
    hp, rp, firsts = results[P.IFA_BATCH_PERSISTENT]
    hs, rs, _ = results[P.IFA_BATCH_PER_SET]
    assert tuples(hp) == tuples(hs)
    assert rp["mode"].tolist() == rs["mode"].tolist()
    assert rp["hits"].tolist() == rs["hits"].tolist()
    expect = []
    for (qs, s, mode), first, ran in zip(sets, firsts, rp["mode"]):
        assert mode == P.IFA_MODE_AUTO or ran == mode
        expect.extend(tuples(_shift(_oracle_set(wl, qs, s, int(ran)), first)))
    assert tuples(hp) == sorted(expect)


def test_store_errors():
    h = P.ifa_create(hit_capacity=1024, segment_bytes=1 << 16)
    try:
        ref = np.frombuffer(b"ACGT" * 20, np.uint8).copy()
        with pytest.raises(P.IfaError) as ei:
            P.ifa_batch_run(h, P.IFA_BATCH_PERSISTENT, 0)
        assert ei.value.status == P.IFA_ERR_BAD_STATE
        P.ifa_ref_append(h, ref[:40], [(0, 0, 0, 40, False)])   # 40: not a multiple of 32
        with pytest.raises(P.IfaError) as ei:
            P.ifa_ref_append(h, ref[:32], [(0, 40, 0, 32, True)])
        assert ei.value.status == P.IFA_ERR_INVALID_ARG
    finally:
        P.ifa_destroy(h)


def test_per_set_subs_at_query_length():
    """Per-set maxSubs at and above the query length on the fast path: a
    128-base query against a poly-A contig mismatches every base of every
    window (count 128), so maxSubs 128 keeps every window and 127 none;
    other sets mix 100-128 bp queries with maxSubs 60 and 200."""
    import types
    rng = np.random.default_rng(5)
    contig0 = np.full(3000, ord("A"), np.uint8)
    contig1 = np.frombuffer(bytes(rng.choice(list(b"ACGT"), 2000).astype(np.uint8)), np.uint8)
    wl = types.SimpleNamespace(ref=np.concatenate([contig0, contig1]),
                               contig_len=np.array([3000, 2000], np.int64))
    specs = [([b"C" * 128], 128), ([b"C" * 128], 127), ([b"G" * 100 + b"T" * 28], 200),
             (synth.random_queries(3, 100, 128, 9), 60), (synth.random_queries(2, 120, 128, 10), 128)]
    h = P.ifa_create(hit_capacity=1 << 20, segment_bytes=1 << 16)
    try:
        _store(h, wl, 1 << 12)
        firsts = [P.ifa_set_add(h, qs, s, P.IFA_MODE_BRUTE)[1] for qs, s in specs]
        P.ifa_batch_run(h, P.IFA_BATCH_PERSISTENT, len(specs))
        hits, over = P.ifa_drain_hits(h)
        assert not over
    finally:
        P.ifa_destroy(h)
    expect = []
    for (qs, s), first in zip(specs, firsts):
        expect.extend(tuples(_shift(oracle.brute(qs, wl.ref, wl.contig_len, s), first)))
    # maxSubs = L keeps every window of both contigs; 127 drops the poly-A contig
    assert len([x for x in expect if x[0] == firsts[0]]) == 2 * (3000 - 127) + 2 * (2000 - 127)
    assert not [x for x in expect if x[0] == firsts[1] and x[1] == 0]
    assert tuples(P.sort_hits(hits)) == sorted(expect)


def _tuples6(h):
    return sorted(zip(h["query"].tolist(), h["contig"].tolist(), h["pos"].tolist(),
                      h["strand"].tolist(), h["mismatches"].tolist(), h["clips"].tolist()))


def test_soft_clipping_in_batches():
    """Soft clipping at contig ends (25 % of the query length) in both batch
    kinds: every set, brute force or indexed, reports the clipped windows at
    its own maxSubs (exhaustively, as in streaming), with contigs cut across
    appends, exactly as the oracle."""
    wl = synth.small_workload(seed=79, n_queries=2, lmin=12, lmax=40, n_contigs=40, cmin=3,
                              cmax=3000, plant_ks=[0, 1, 2] * 4)
    sets = [(synth.random_queries(5, 6, 12, 201), 2, P.IFA_MODE_BRUTE),
            (synth.random_queries(6, 10, 16, 202), 2, P.IFA_MODE_INDEXED),
            (wl.queries + synth.random_queries(3, 8, 14, 203), 3, P.IFA_MODE_BRUTE)]
    got = {}
    h = P.ifa_create(hit_capacity=1 << 22, segment_bytes=1 << 20, minhits_trials=TRIALS, clip_pct=25)
    try:
        _store(h, wl, 1024)
        firsts = [P.ifa_set_add(h, qs, s, mode)[1] for qs, s, mode in sets]
        for kind in (P.IFA_BATCH_PERSISTENT, P.IFA_BATCH_PER_SET):
            P.ifa_reset_results(h)
            P.ifa_batch_run(h, kind, len(sets))
            hits, over = P.ifa_drain_hits(h)
            assert not over
            got[kind] = _tuples6(hits)
    finally:
        P.ifa_destroy(h)
    expect = []
    for (qs, s, mode), first in zip(sets, firsts):
        if mode == P.IFA_MODE_BRUTE:
            e = oracle.brute(qs, wl.ref, wl.contig_len, s, clip_pct=25)
        else:
            plan = [oracle.choose_k(len(q), s, trials=TRIALS) for q in qs]
            e = oracle.indexed(qs, wl.ref, wl.contig_len, s, [p[1] for p in plan], [p[2] for p in plan],
                               [1 if p[0] < 0 else 0 for p in plan], clip_pct=25)
        expect.extend(_tuples6(_shift(e, first)))
    assert any(x[5] for x in expect)                 # clipped hits are in the case
    assert got[P.IFA_BATCH_PERSISTENT] == sorted(expect)
    assert got[P.IFA_BATCH_PER_SET] == sorted(expect)


@pytest.mark.parametrize("kernel", [P.IFA_BRUTE_AUTO, P.IFA_BRUTE_TENSOR])
def test_tensor_core_sets_in_batches(kernel):
    """Brute-force sets on the tensor cores inside a batch: with the
    automatic rule a 96-query set of 24-40 bp at maxSubs 3 (sparse hits)
    goes to the tensor cores and the others stay on the popcount kernel;
    forced, every brute-force set of queries up to 64 bases does.  Sets
    share one operand (each padded to whole 128-row tiles, per-row maxSubs);
    both batch kinds must give the oracle's hits."""
    wl = synth.small_workload(seed=89, n_queries=3, lmin=24, lmax=40, n_contigs=30, cmin=50,
                              cmax=9000, plant_ks=[0, 1, 2, 3] * 4)
    sets = [(synth.random_queries(96, 24, 40, 301) + wl.queries[:1], 3, P.IFA_MODE_BRUTE),
            (synth.random_queries(5, 12, 20, 302), 2, P.IFA_MODE_BRUTE),
            (synth.random_queries(40, 18, 60, 303) + wl.queries[1:], 5, P.IFA_MODE_BRUTE),
            (synth.random_queries(8, 20, 30, 304), 2, P.IFA_MODE_INDEXED)]
    got = {}
    h = P.ifa_create(hit_capacity=1 << 22, segment_bytes=1 << 20, minhits_trials=TRIALS, brute_kernel=kernel)
    try:
        _store(h, wl, 4096)
        firsts = [P.ifa_set_add(h, qs, s, mode)[1] for qs, s, mode in sets]
        for kind in (P.IFA_BATCH_PERSISTENT, P.IFA_BATCH_PER_SET):
            P.ifa_reset_results(h)
            res = P.ifa_batch_run(h, kind, len(sets))
            hits, over = P.ifa_drain_hits(h)
            assert not over
            got[kind] = (tuples(P.sort_hits(hits)), res["hits"].tolist())
    finally:
        P.ifa_destroy(h)
    expect, per_set = [], []
    for (qs, s, mode), first in zip(sets, firsts):
        e = _oracle_set(wl, qs, s, mode)
        expect.extend(tuples(_shift(e, first)))
        per_set.append(e.size)
    assert got[P.IFA_BATCH_PERSISTENT][0] == sorted(expect)
    assert got[P.IFA_BATCH_PER_SET][0] == sorted(expect)
    assert got[P.IFA_BATCH_PERSISTENT][1] == per_set == got[P.IFA_BATCH_PER_SET][1]
