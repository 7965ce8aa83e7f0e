"""Soft clipping at contig ends in the oracle (Methods, "Algorithm Design":
alignments may overhang a contig end by up to a share of the query length),
pinned to counts and values that follow from the definition rather than to
the oracle itself."""
import numpy as np
import pytest

import oracle
import synth

COMP = bytes.maketrans(b"ACGTacgt", b"TGCAtgca")


def rc(q: bytes) -> bytes:
    return q.translate(COMP)[::-1]


def _keyset(h, with_query=True):
    return set(zip(*( ([h["query"].tolist()] if with_query else []) +
                     [h["contig"].tolist(), h["pos"].tolist(), h["strand"].tolist(),
                      h["mismatches"].tolist(), h["clips"].tolist()])))


def test_zero_clip_is_the_unclipped_scan():
    wl = synth.small_workload(seed=11, n_queries=5, lmin=6, lmax=30, n_contigs=9, cmin=1, cmax=400)
    a = oracle.brute(wl.queries, wl.ref, wl.contig_len, 3)
    b = oracle.brute(wl.queries, wl.ref, wl.contig_len, 3, clip_pct=0)
    assert a.tobytes() == b.tobytes()
    assert (a["clips"] == 0).all()


@pytest.mark.parametrize("pct", [10, 25, 50])
def test_closed_form_count_when_every_window_passes(pct):
    """With maxSubs >= L every window in range hits, so a (query, strand,
    contig) gives n - L + 1 + 2C hits when n >= L - C and none otherwise,
    C = floor(pct * L / 100)."""
    rng = np.random.default_rng(pct)
    lens = np.array([1, 3, 7, 9, 12, 15, 16, 20, 33, 64], np.int64)
    ref = np.frombuffer(bytes(rng.choice(list(b"ACGT"), int(lens.sum())).astype(np.uint8)), np.uint8).copy()
    queries = [b"ACGTACGTACGTACGT", b"TTGCA" * 4 + b"G", b"ACG" * 3]
    hits = oracle.brute(queries, ref, lens, 255, clip_pct=pct)
    for qi, q in enumerate(queries):
        L = len(q)
        C = pct * L // 100
        for ci, n in enumerate(lens.tolist()):
            expect = n - L + 1 + 2 * C if n >= L - C else 0
            for t in (0, 1):
                got = int(((hits["query"] == qi) & (hits["contig"] == ci) & (hits["strand"] == t)).sum())
                assert got == expect, (qi, ci, t, got, expect)
    # clip fields: left + right <= C, and each clipped hit keeps >= 1 aligned base
    for h in hits:
        L = len(queries[h["query"]])
        left, right = int(h["clips"]) & 0xff, int(h["clips"]) >> 8
        assert left + right <= pct * L // 100
        assert left + right < L


@pytest.mark.parametrize("side", ["start", "end"])
def test_planted_overhangs_are_found_with_their_clips(side):
    """Write the aligned part of a query (with k substitutions in it) so that
    it overhangs a contig end by o bases: the hit has clips o on that side,
    k mismatches and pos at the first aligned base."""
    rng = np.random.default_rng(3 if side == "start" else 4)
    q = bytes(rng.choice(list(b"ACGT"), 32).astype(np.uint8))
    L, pct = len(q), 25
    C = pct * L // 100     # 8
    n = 200
    for o in range(1, C + 1):
        for k in (0, 1, 3):
            contig = bytearray(rng.choice(list(b"ACGT"), n).astype(np.uint8))
            part = bytearray(q[o:] if side == "start" else q[:L - o])
            for i in rng.choice(len(part), k, replace=False):
                part[i] = [c for c in b"ACGT" if c != part[i]][int(rng.integers(0, 3))]
            if side == "start":
                contig[:len(part)] = part
                pos, clips = 0, o
            else:
                contig[n - len(part):] = part
                pos, clips = n - len(part), o << 8
            ref = np.frombuffer(bytes(contig), np.uint8)
            hits = oracle.brute([q], ref, np.array([n]), k, clip_pct=pct)
            want = (0, 0, pos, 0, k, clips)
            assert want in _keyset(hits), (side, o, k)


def test_monotone_in_clip_share_and_interior_unchanged():
    wl = synth.small_workload(seed=21, n_queries=4, lmin=10, lmax=40, n_contigs=10, cmin=5, cmax=300)
    prev = None
    base = _keyset(oracle.brute(wl.queries, wl.ref, wl.contig_len, 4))
    for pct in (0, 10, 25, 40):
        h = oracle.brute(wl.queries, wl.ref, wl.contig_len, 4, clip_pct=pct)
        cur = _keyset(h)
        assert {x for x in cur if x[5] == 0} == base
        if prev is not None:
            assert prev <= cur
        prev = cur


def test_reverse_complement_symmetry_with_clips():
    wl = synth.small_workload(seed=23, n_queries=3, lmin=12, lmax=30, n_contigs=8, cmin=5, cmax=200)
    for q in wl.queries:
        a = oracle.brute([q], wl.ref, wl.contig_len, 5, clip_pct=30)
        b = oracle.brute([rc(q)], wl.ref, wl.contig_len, 5, clip_pct=30)
        flip = {(c, p, 1 - t, m, r) for (c, p, t, m, r) in _keyset(b, with_query=False)}
        assert _keyset(a, with_query=False) == flip


def test_indexed_keeps_every_clipped_window():
    wl = synth.small_workload(seed=29, n_queries=5, lmin=16, lmax=40, n_contigs=10, cmin=5, cmax=600)
    s, pct = 3, 25
    plan = [oracle.choose_k(len(q), s, trials=5000) for q in wl.queries]
    ks = [p[1] for p in plan]
    mh = [p[2] for p in plan]
    ex = [1 if p[0] < 0 else 0 for p in plan]
    b = oracle.brute(wl.queries, wl.ref, wl.contig_len, s, clip_pct=pct)
    i = oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, ks, mh, ex, clip_pct=pct)
    bs, is_ = _keyset(b), _keyset(i)
    assert is_ <= bs
    assert {x for x in bs if x[5]} == {x for x in is_ if x[5]}


def test_digest_sees_the_clips():
    h = np.zeros(1, oracle.HIT_DTYPE)
    h[0] = (1, 2, 0, 0, 1, 0)
    d0 = oracle.digest(h)
    h["clips"] = 2
    assert oracle.digest(h) != d0


_ACGT = set(b"ACGT")


def _fold(b):
    b = int(b) & 0xDF   # upper case
    return b if b in _ACGT else ord("N")


def _brute_clipped(queries, ref, lens, s, pct):
    """The definition in plain Python loops: every window start p from -C
    to n - L + C of every contig, clips = bases outside the contig
    (left | right << 8), at most C of them and at least one base aligned,
    mismatches counted over the aligned bases only (N never matches)."""
    comp = {ord("A"): ord("T"), ord("C"): ord("G"), ord("G"): ord("C"), ord("T"): ord("A")}
    out = set()
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    for qi, q in enumerate(queries):
        L = len(q)
        C = pct * L // 100
        fwd = [_fold(b) for b in q]
        rev = [comp.get(b, ord("N")) for b in reversed(fwd)]
        for t, qq in enumerate((fwd, rev)):
            for ci, n in enumerate(lens.tolist()):
                r = [_fold(b) for b in ref[starts[ci]:starts[ci] + n]]
                for p in range(-C, n - L + C + 1):
                    left, right = max(0, -p), max(0, p + L - n)
                    if left + right > C or left + right >= L:
                        continue
                    mm = sum(1 for i in range(left, L - right)
                             if qq[i] == ord("N") or r[p + i] == ord("N") or qq[i] != r[p + i])
                    if mm <= s:
                        out.add((qi, ci, p + left, t, mm, left | (right << 8)))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_matches_plain_python_definition_on_tiny_inputs(seed):
    rng = np.random.default_rng(500 + seed)
    lens = rng.integers(1, 40, size=int(rng.integers(1, 6))).astype(np.int64)
    alphabet = np.frombuffer(b"ACGTACGTacgN", np.uint8)
    ref = rng.choice(alphabet, int(lens.sum())).astype(np.uint8)
    queries = [bytes(rng.choice(alphabet, int(rng.integers(1, 20))).astype(np.uint8)) for _ in range(4)]
    for pct in (10, 25, 50):
        for s in (0, 2, 5):
            got = _keyset(oracle.brute(queries, ref, lens, s, clip_pct=pct))
            assert got == _brute_clipped(queries, ref, lens, s, pct), (pct, s)
