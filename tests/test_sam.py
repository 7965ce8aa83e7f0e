"""SAM text (Methods, "Output Format"): the oracle against a hand-written
example, then the library's host-side formatter against the oracle.  No GPU:
the formatter is host code and the hits come from the CPU oracle."""
import json
import os

import numpy as np
import pytest

import oracle
import oracle.sam as osam
import paper_2607_27291_b300 as P
import synth

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sam_example.json")))


def _queries():
    return [q.encode() for q in GOLDEN["queries"]]


def _hit_array(tuples):
    a = np.zeros(len(tuples), dtype=P.HIT_DTYPE)
    for i, (q, c, p, t, m) in enumerate(tuples):
        a[i] = (q, c, p, t, m, 0)
    return a


def test_oracle_matches_hand_written_records():
    seen = [False] * len(GOLDEN["queries"])
    text = osam.sam_records([tuple(h) for h in GOLDEN["hits"]], _queries(), seen)
    assert text == "".join(r + "\n" for r in GOLDEN["records"])
    assert seen == [True, True]


def test_oracle_names_and_header():
    seen = [False, False]
    names = {int(k): v for k, v in GOLDEN["contig_names"].items()}
    text = osam.sam_records([tuple(h) for h in GOLDEN["hits"]], _queries(), seen,
                            query_names=GOLDEN["query_names"], contig_names=names)
    assert text.splitlines()[0] == GOLDEN["named_first_record"]
    assert osam.sam_header([tuple(c) for c in GOLDEN["header_contigs"]]) == GOLDEN["header"]


def test_library_matches_hand_written_records():
    seen = np.zeros(2, dtype=np.uint8)
    text = P.ifa_sam_records(_hit_array(GOLDEN["hits"]), _queries(), seen)
    assert text.decode() == "".join(r + "\n" for r in GOLDEN["records"])
    assert seen.tolist() == [1, 1]
    names = [None] * 6
    for k, v in GOLDEN["contig_names"].items():
        names[int(k)] = v
    seen[:] = 0
    text = P.ifa_sam_records(_hit_array(GOLDEN["hits"]), _queries(), seen,
                             query_names=GOLDEN["query_names"], contig_names=names)
    assert text.decode().splitlines()[0] == GOLDEN["named_first_record"]
    hdr = P.ifa_sam_header([c[1] for c in GOLDEN["header_contigs"]],
                           contig_names=[c[0] for c in GOLDEN["header_contigs"]])
    assert hdr.decode() == GOLDEN["header"]
    assert P.ifa_sam_header([1000, 250], contig_ids=[3, 5]).decode() == \
        "@HD\tVN:1.6\tSO:unsorted\n@SQ\tSN:c3\tLN:1000\n@SQ\tSN:c5\tLN:250\n"


def test_library_matches_oracle_across_calls():
    """Hits of a small brute-force oracle run, formatted in two calls (two
    halves of the reference in stream order) with the primary flags carried
    over: the concatenated text equals one oracle call."""
    wl = synth.small_workload(seed=3)
    hits = oracle.brute(wl.queries, wl.ref, wl.contig_len, 3)
    assert hits.size > 20
    tuples = [tuple(int(x) for x in (h["query"], h["contig"], h["pos"], h["strand"], h["mismatches"]))
              for h in hits]
    seen_o = [False] * len(wl.queries)
    expect = osam.sam_records(tuples, wl.queries, seen_o)
    split = int(np.median(hits["contig"]))
    first = hits[hits["contig"] < split]
    second = hits[hits["contig"] >= split]
    seen = np.zeros(len(wl.queries), dtype=np.uint8)
    got = P.ifa_sam_records(first.copy(), wl.queries, seen) + P.ifa_sam_records(second.copy(), wl.queries, seen)
    assert got.decode() == expect
    assert seen.astype(bool).tolist() == seen_o


def test_library_rejects_bad_hits_and_keeps_flags():
    seen = np.zeros(2, dtype=np.uint8)
    bad = _hit_array([[0, 1, 2, 0, 0], [7, 1, 2, 0, 0]])
    with pytest.raises(P.IfaError):
        P.ifa_sam_records(bad, _queries(), seen)
    assert seen.tolist() == [0, 0]
    bad = _hit_array([[0, 1, 2, 2, 0]])
    with pytest.raises(P.IfaError):
        P.ifa_sam_records(bad, _queries(), seen)
    assert P.ifa_sam_records(_hit_array([]), _queries(), seen) == b""


def test_clipped_records_match_hand_written():
    seen = [False, False]
    text = osam.sam_records([tuple(h) for h in GOLDEN["clipped_hits"]], _queries(), seen)
    assert text == "".join(r + "\n" for r in GOLDEN["clipped_records"])
    a = np.zeros(len(GOLDEN["clipped_hits"]), dtype=P.HIT_DTYPE)
    for i, (q, c, p, t, m, cl) in enumerate(GOLDEN["clipped_hits"]):
        a[i] = (q, c, p, t, m, cl)
    got = P.ifa_sam_records(a, _queries(), np.zeros(2, np.uint8))
    assert got.decode() == "".join(r + "\n" for r in GOLDEN["clipped_records"])


def _random_case(rng):
    nq = int(rng.integers(1, 8))
    alphabet = np.frombuffer(b"ACGTacgtNRY-", np.uint8)
    queries = [bytes(rng.choice(alphabet, int(rng.integers(1, 61))).astype(np.uint8)) for _ in range(nq)]
    n = int(rng.integers(0, 120))
    hits = np.zeros(n, dtype=P.HIT_DTYPE)
    for i in range(n):
        q = int(rng.integers(0, nq))
        L = len(queries[q])
        left = right = 0
        if L > 1 and rng.random() < 0.3:
            budget = int(rng.integers(1, L))          # clips < L: one base stays aligned
            left = int(rng.integers(0, budget + 1))
            right = budget - left
        hits[i] = (q, int(rng.integers(0, 6)), int(rng.integers(0, 5000)), int(rng.integers(0, 2)),
                   int(rng.integers(0, L + 1)), left | (right << 8))
    return queries, hits


@pytest.mark.parametrize("seed", range(40))
def test_library_matches_oracle_on_random_hits(seed):
    """Random query sets (IUPAC bytes, lower case, lengths 1..60) and random
    hits with clips, cut into calls at contig boundaries (reference order)
    and formatted by the library with the primary flags carried across the
    calls: the text equals one oracle call, with and without long names
    (which force the output buffer to grow)."""
    rng = np.random.default_rng(1000 + seed)
    queries, hits = _random_case(rng)
    tuples = [tuple(int(x) for x in (h["query"], h["contig"], h["pos"], h["strand"], h["mismatches"], h["clips"]))
              for h in hits]
    named = seed % 2 == 1
    qnames = ["read_%d_" % i + "x" * int(rng.integers(0, 300)) for i in range(len(queries))] if named else None
    cnames = ["contig_%d_" % c + "y" * int(rng.integers(0, 200)) for c in range(6)] if named else None
    seen_o = [False] * len(queries)
    expect = osam.sam_records(tuples, queries, seen_o, query_names=qnames,
                              contig_names=dict(enumerate(cnames)) if named else None)
    cuts = sorted(set(int(c) for c in rng.integers(0, 7, size=int(rng.integers(0, 4)))))
    bounds = [0] + cuts + [7]
    seen = np.zeros(len(queries), dtype=np.uint8)
    got = b""
    for lo, hi in zip(bounds[:-1], bounds[1:]):
        part = hits[(hits["contig"] >= lo) & (hits["contig"] < hi)].copy()
        got += P.ifa_sam_records(part, queries, seen, query_names=qnames, contig_names=cnames)
    assert got.decode() == expect
    assert seen.astype(bool).tolist() == seen_o
