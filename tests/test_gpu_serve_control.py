"""Serving control and allocation failures on the GPU.

* Cancellation: a request cancelled while queued, active or complete frees
  its ring and budget and leaves the others' hits equal to the oracle.
* An HBM budget below one request's need: requests run one at a time (one
  is always admitted when none is active), each still exact.
* Allocations that cannot succeed (a 16 TiB hit ring, a 1 TiB store, a
  16 TiB request ring) return IFA_ERR_OOM from the host call; the handle
  stays usable and later work is exact.  cudaMalloc refuses these sizes on
  the host: nothing faulting reaches the device."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import tuples

pytestmark = pytest.mark.gpu


def _wl():
    return synth.small_workload(seed=171, n_queries=4, lmin=16, lmax=40, n_contigs=16, cmin=200, cmax=6000,
                                plant_ks=[0, 1, 2, 3] * 3)


def _load(h, wl):
    for a, b, pc in P.segment_pieces(wl.contig_len, 1 << 14):
        P.ifa_ref_append(h, wl.ref[a:b], pc)


def test_cancel_queued_active_and_complete_with_budget_below_need():
    wl = _wl()
    qs = [[wl.queries[0]], [wl.queries[1]], [wl.queries[2]], [wl.queries[3]], wl.queries[:2]]
    n_slices = 4
    h = P.ifa_create(hit_capacity=1024, segment_bytes=1 << 20)
    try:
        _load(h, wl)
        P.ifa_serve_start(h, n_slices, 1, 1 << 16)     # 1 byte: below any request's need
        r = [P.ifa_serve_submit(h, q, 3, P.IFA_MODE_BRUTE) for q in qs[:3]]
        most_active = 0
        for _ in range(2):
            active, _ = P.ifa_serve_step(h)
            most_active = max(most_active, active)
        assert P.ifa_serve_poll(h, r[0])["state"] == 1
        assert P.ifa_serve_poll(h, r[2])["state"] == 0
        P.ifa_serve_cancel(h, r[0])                    # active, half scanned
        P.ifa_serve_cancel(h, r[2])                    # queued
        r.append(P.ifa_serve_submit(h, qs[3], 4, P.IFA_MODE_BRUTE))
        r.append(P.ifa_serve_submit(h, qs[4], 2, P.IFA_MODE_BRUTE))
        steps = 0
        while not all(P.ifa_serve_poll(h, i)["state"] == 2 for i in (r[1], r[3], r[4])):
            active, _ = P.ifa_serve_step(h)
            most_active = max(most_active, active)
            steps += 1
            assert steps < 40
        assert most_active == 1                        # one at a time under the budget
        # a complete request may be cancelled instead of drained
        P.ifa_serve_cancel(h, r[4])
        for i in (r[0], r[2], r[4]):
            assert P.ifa_serve_poll(h, i)["state"] == 4
            with pytest.raises(P.IfaError) as ei:
                P.ifa_serve_drain(h, i, 16)
            assert ei.value.status == P.IFA_ERR_BAD_STATE
            with pytest.raises(P.IfaError) as ei:
                P.ifa_serve_cancel(h, i)
            assert ei.value.status == P.IFA_ERR_BAD_STATE
        with pytest.raises(P.IfaError) as ei:
            P.ifa_serve_cancel(h, 99)
        assert ei.value.status == P.IFA_ERR_INVALID_ARG
        for i, q, s in ((r[1], qs[1], 3), (r[3], qs[3], 4)):
            hits, over = P.ifa_serve_drain(h, i, 1 << 16)
            exp = oracle.brute(q, wl.ref, wl.contig_len, s)
            assert not over
            assert tuples(P.sort_hits(hits)) == tuples(exp)
            assert P.ifa_serve_poll(h, i)["digest"] == oracle.digest(exp)
        P.ifa_serve_stop(h)
    finally:
        P.ifa_destroy(h)


def test_allocation_failures_return_oom_and_leave_the_handle_usable():
    with pytest.raises(P.IfaError) as ei:
        P.ifa_create(hit_capacity=1 << 40, segment_bytes=1 << 20)    # a 16 TiB hit ring
    assert ei.value.status == P.IFA_ERR_OOM
    wl = _wl()
    h = P.ifa_create(hit_capacity=1024, segment_bytes=1 << 20)
    try:
        with pytest.raises(P.IfaError) as ei:
            P.ifa_ref_reserve(h, 1 << 42)              # 1 TiB of hi/lo words
        assert ei.value.status == P.IFA_ERR_OOM
        _load(h, wl)
        P.ifa_serve_start(h, 3, 1 << 40, 1 << 40)       # every request ring is 16 TiB
        rid = P.ifa_serve_submit(h, [wl.queries[0]], 2, P.IFA_MODE_BRUTE)
        with pytest.raises(P.IfaError) as ei:
            P.ifa_serve_step(h)
        assert ei.value.status == P.IFA_ERR_OOM
        assert P.ifa_serve_poll(h, rid)["state"] == 0   # still queued, nothing held
        P.ifa_serve_cancel(h, rid)
        P.ifa_serve_stop(h)
        P.ifa_serve_start(h, 3, 1 << 40, 1 << 16)
        rid = P.ifa_serve_submit(h, wl.queries, 3, P.IFA_MODE_BRUTE)
        while P.ifa_serve_poll(h, rid)["state"] != 2:
            P.ifa_serve_step(h)
        hits, over = P.ifa_serve_drain(h, rid, 1 << 16)
        exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, 3)
        assert not over
        assert tuples(P.sort_hits(hits)) == tuples(exp)
        P.ifa_serve_stop(h)
        # the streaming path on the same handle
        P.ifa_load_queries(h, wl.queries)
        P.ifa_set_max_subs(h, 3)
        for a, b, pc in P.segment_pieces(wl.contig_len, 1 << 15):
            P.ifa_push_segment(h, wl.ref[a:b], pc)
        P.ifa_flush(h)
        got, over = P.ifa_drain_hits(h)
        assert not over
        assert tuples(P.sort_hits(got)) == tuples(exp)
    finally:
        P.ifa_destroy(h)
