"""Continuous-batching serving over the device-resident store.

Requests arrive before and during the cyclic scan, wait for budget, join at
whatever slice the scan is on and leave after one full cycle.  Each
request's hits (request-relative query ids) and digest must equal the
oracle's for its queries and mode, and must be identical when the request
is served alone."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import tuples

pytestmark = pytest.mark.gpu

TRIALS = 20_000


def _expected(wl, queries, s, mode):
    if mode == P.IFA_MODE_BRUTE:
        return oracle.brute(queries, wl.ref, wl.contig_len, s)
    plan = [oracle.choose_k(len(q), s, trials=TRIALS) for q in queries]
    exh = [1 if st < 0 else 0 for st, _, _ in plan]
    return oracle.indexed(queries, wl.ref, wl.contig_len, s, [p[1] for p in plan],
                          [p[2] for p in plan], exh)


def _session(wl, requests, arrive_at, budget, n_slices=5):
    """Serve `requests` [(queries, s, mode)], request i submitted before
    step arrive_at[i]; returns per request (hits, info)."""
    h = P.ifa_create(hit_capacity=1024, segment_bytes=1 << 20, minhits_trials=TRIALS,
                     auto_crossover=6)
    try:
        for a, b, pc in P.segment_pieces(wl.contig_len, 1 << 14):
            P.ifa_ref_append(h, wl.ref[a:b], pc)
        P.ifa_serve_start(h, n_slices, budget, 1 << 16)
        ids = {}
        step = 0
        while True:
            for i, t in enumerate(arrive_at):
                if t == step and i not in ids:
                    qs, s, mode = requests[i]
                    ids[i] = P.ifa_serve_submit(h, qs, s, mode)
            active, _ = P.ifa_serve_step(h)
            step += 1
            infos = {i: P.ifa_serve_poll(h, r) for i, r in ids.items()}
            if len(ids) == len(requests) and all(v["state"] == 2 for v in infos.values()):
                break
            assert step < 200
        out = []
        for i in range(len(requests)):
            hits, over = P.ifa_serve_drain(h, ids[i], 1 << 16)
            assert not over
            out.append((P.sort_hits(hits), infos[i]))
        P.ifa_serve_stop(h)
        return out
    finally:
        P.ifa_destroy(h)


def test_serving_matches_oracle_alone_and_in_the_mix():
    wl = synth.small_workload(seed=81, n_queries=3, lmin=16, lmax=40, n_contigs=24, cmin=100,
                              cmax=9000, plant_ks=[0, 1, 2, 3, 4] * 4)
    requests = [
        ([wl.queries[0]] + synth.random_queries(2, 14, 40, 201), 3, P.IFA_MODE_AUTO),     # brute
        (synth.random_queries(9, 16, 44, 202) + [wl.queries[1]], 4, P.IFA_MODE_AUTO),    # indexed
        ([wl.queries[2]], 5, P.IFA_MODE_BRUTE),
        (synth.random_queries(7, 12, 30, 203), 2, P.IFA_MODE_INDEXED),
        (synth.random_queries(1, 10, 10, 204), 1, P.IFA_MODE_BRUTE),
    ]
    arrive = [0, 0, 2, 3, 7]
    budget = 3 * (1 << 16) * 16    # room for about three rings: later requests queue
    mixed = _session(wl, requests, arrive, budget)
    admits = [info["admit_s"] for _, info in mixed]
    assert max(admits) > min(admits)           # requests joined at different times
    for (qs, s, mode), (hits, info) in zip(requests, mixed):
        assert info["state"] == 2 and info["slices_done"] == 5
        exp = _expected(wl, qs, s, info["mode"])
        assert tuples(hits) == tuples(exp)
        assert info["digest"] == oracle.digest(exp)
    for i, req in enumerate(requests):
        alone = _session(wl, [req], [0], 1 << 40)[0]
        assert tuples(alone[0]) == tuples(mixed[i][0])
        assert alone[1]["digest"] == mixed[i][1]["digest"]
