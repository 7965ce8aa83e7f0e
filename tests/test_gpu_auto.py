"""IFA_MODE_AUTO on the GPU: the mode each path picks and the hits it
returns in that mode.

The paper finds that the crossover between brute force and indexed mode
depends on the workload (Results, Terabase-Scale Performance; Discussion).
By default the choice comes from rates measured on the device; a positive
auto_crossover restores the paper's count rule.  Far from the crossover the
measured choice is fixed by arithmetic: one query costs 2 entry x base
evaluations per base in brute force, against at least one k-mer table lookup
per base in indexed mode, so brute force wins; hundreds of queries cost
hundreds of evaluations per base against a handful of lookups, so indexed
mode wins.  Either way the hits equal the oracle's for the mode picked."""
import json
import os

import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import tuples

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TRIALS = 10_000


def _plan(queries, s):
    memo = {}
    out = []
    for q in queries:
        if len(q) not in memo:
            memo[len(q)] = oracle.choose_k(len(q), s, trials=TRIALS)
        out.append(memo[len(q)])
    return out


def _expected(queries, wl, s, mode):
    if mode == P.IFA_MODE_BRUTE:
        return oracle.brute(queries, wl.ref, wl.contig_len, s, threads=8)
    plan = _plan(queries, s)
    exh = [1 if st < 0 else 0 for st, _, _ in plan]
    return oracle.indexed(queries, wl.ref, wl.contig_len, s, [p[1] for p in plan], [p[2] for p in plan], exh,
                          threads=8)


def _stream(queries, wl, s, **cfg):
    h = P.ifa_create(hit_capacity=1 << 22, segment_bytes=1 << 20, minhits_trials=TRIALS, **cfg)
    try:
        P.ifa_load_queries(h, queries)
        P.ifa_set_max_subs(h, s)
        P.ifa_set_mode(h, P.IFA_MODE_AUTO)
        for a, b, pc in P.segment_pieces(wl.contig_len, 1 << 15):
            P.ifa_push_segment(h, wl.ref[a:b], pc)
        P.ifa_flush(h)
        hits, over = P.ifa_drain_hits(h)
        assert not over
        return P.sort_hits(hits), P.ifa_get_stats(h)["mode"]
    finally:
        P.ifa_destroy(h)


@pytest.mark.parametrize("n,want", [(1, P.IFA_MODE_BRUTE), (400, P.IFA_MODE_INDEXED)])
def test_streaming_auto_by_measured_rates(n, want):
    wl = synth.small_workload(seed=400 + n, n_queries=min(n, 4), lmin=28, lmax=36, n_contigs=12, cmin=500,
                              cmax=9000, plant_ks=[0, 1, 2] * 3)
    queries = (wl.queries + synth.random_queries(n, 28, 36, 401))[:n]
    got, mode = _stream(queries, wl, 2)
    assert mode == want
    exp = _expected(queries, wl, 2, mode)
    assert exp.size > 0
    assert tuples(got) == tuples(exp)


def test_streaming_auto_by_the_papers_count_rule():
    """auto_crossover from the paper's range: one query fewer runs brute
    force, the crossover count itself runs indexed."""
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_defaults.json")))["crossover_queries"]
    c = (g["low"] + g["high"]) // 2
    wl = synth.small_workload(seed=431, n_queries=3, lmin=24, lmax=32, n_contigs=6, cmin=300, cmax=3000,
                              plant_ks=[0, 1] * 2)
    for n, want in ((c - 1, P.IFA_MODE_BRUTE), (c, P.IFA_MODE_INDEXED)):
        queries = (wl.queries + synth.random_queries(n, 24, 32, 432))[:n]
        got, mode = _stream(queries, wl, 1, auto_crossover=c)
        assert mode == want
        assert tuples(got) == tuples(_expected(queries, wl, 1, mode))


def test_serving_auto_by_measured_rates():
    """Requests resolve AUTO at admission, from rates measured once on the
    store: a one-query request runs brute force, a 300-query request
    indexed, each exact for its mode."""
    wl = synth.small_workload(seed=441, n_queries=2, lmin=28, lmax=36, n_contigs=10, cmin=800, cmax=8000,
                              plant_ks=[0, 1, 2] * 3)
    reqs = [([wl.queries[0]], 2), (wl.queries[1:] + synth.random_queries(299, 28, 36, 442), 2)]
    h = P.ifa_create(hit_capacity=1024, segment_bytes=1 << 20, minhits_trials=TRIALS)
    try:
        for a, b, pc in P.segment_pieces(wl.contig_len, 1 << 14):
            P.ifa_ref_append(h, wl.ref[a:b], pc)
        P.ifa_serve_start(h, 4, 1 << 40, 1 << 20)
        ids = [P.ifa_serve_submit(h, qs, s, P.IFA_MODE_AUTO) for qs, s in reqs]
        assert all(P.ifa_serve_poll(h, i)["mode"] == P.IFA_MODE_AUTO for i in ids)   # not admitted yet
        while P.ifa_serve_step(h)[0]:
            pass
        modes = []
        for rid, (qs, s) in zip(ids, reqs):
            info = P.ifa_serve_poll(h, rid)
            assert info["state"] == 2
            modes.append(info["mode"])
            hits, over = P.ifa_serve_drain(h, rid, 1 << 20)
            assert not over
            exp = _expected(qs, wl, s, info["mode"])
            assert tuples(P.sort_hits(hits)) == tuples(exp)
            assert info["digest"] == oracle.digest(exp)
        assert modes == [P.IFA_MODE_BRUTE, P.IFA_MODE_INDEXED]
        P.ifa_serve_stop(h)
    finally:
        P.ifa_destroy(h)
