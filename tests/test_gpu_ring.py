"""The device hit ring (Methods, "Output Format": hits leave as the stream
goes).

A ring far smaller than a pass's hits, drained with ifa_poll_hits between
many small segments while later segments are still being scanned, must give
exactly the oracle's tuples -- in brute force on both kernels, with soft
clipping and in indexed mode -- with ring positions wrapping many times
(capacities that are not powers of two).  Without draining, a full ring drops
hits: the digest and counts stay exact, the drained hits are exactly the
first claims, and after the drain the ring takes hits again."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import tuples

pytestmark = pytest.mark.gpu


def _tuples6(h):
    return sorted(zip(h["query"].tolist(), h["contig"].tolist(), h["pos"].tolist(),
                      h["strand"].tolist(), h["mismatches"].tolist(), h["clips"].tolist()))


def _stream_polled(wl, s, ring, seg, mode=P.IFA_MODE_BRUTE, **cfg):
    h = P.ifa_create(hit_capacity=ring, segment_bytes=1 << 16, **cfg)
    try:
        P.ifa_load_queries(h, wl.queries)
        P.ifa_set_max_subs(h, s)
        P.ifa_set_mode(h, mode)
        buf = np.zeros(ring, P.HIT_DTYPE)
        parts, polled, over_any = [], 0, False
        for a, b, pc in P.segment_pieces(wl.contig_len, seg):
            P.ifa_push_segment(h, wl.ref[a:b], pc)
            n, over, _ = P.ifa_poll_hits(h, buf)
            over_any |= over
            polled += n
            parts.append(buf[:n].copy())
        rest, over = P.ifa_drain_hits(h)
        over_any |= over
        parts.append(rest)
        dig, counts = P.ifa_get_digest(h, len(wl.queries))
        return P.sort_hits(np.concatenate(parts)), over_any, polled, dig
    finally:
        P.ifa_destroy(h)


@pytest.mark.parametrize("kernel", [P.IFA_BRUTE_POPC, P.IFA_BRUTE_TENSOR])
def test_small_ring_polled_between_segments(kernel):
    wl = synth.small_workload(seed=43, n_queries=20, lmin=10, lmax=24, n_contigs=40, cmin=10,
                              cmax=6000, plant_ks=[0, 1, 2, 3] * 20)
    s = 3
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s)
    assert exp.size > 20 * 97              # the ring wraps about 20 times
    got, over, polled, dig = _stream_polled(wl, s, 97, 512, brute_kernel=kernel)
    assert not over
    assert polled > exp.size // 2          # most hits left while the stream went on
    assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)


def test_small_ring_polled_with_clipping():
    wl = synth.small_workload(seed=47, n_queries=12, lmin=8, lmax=24, n_contigs=60, cmin=5,
                              cmax=2000, plant_ks=[0, 1, 2] * 10)
    s = 2
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s, clip_pct=25)
    assert exp.size > 10 * 61
    got, over, polled, dig = _stream_polled(wl, s, 61, 400, clip_pct=25)
    assert not over
    assert _tuples6(got) == _tuples6(exp)
    assert dig == oracle.digest(exp)


def test_small_ring_polled_indexed():
    wl = synth.small_workload(seed=53, n_queries=40, lmin=12, lmax=30, n_contigs=30, cmin=200,
                              cmax=8000, plant_ks=[0, 1, 2, 3] * 10)
    s = 4
    got, over, polled, dig = _stream_polled(wl, s, 29, 1024, mode=P.IFA_MODE_INDEXED, minhits_trials=4000)
    assert not over
    plan = [oracle.choose_k(len(q), s, trials=4000) for q in wl.queries]
    exp = oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, [p[1] for p in plan], [p[2] for p in plan],
                         [1 if p[0] < 0 else 0 for p in plan])
    assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)


def test_full_ring_drops_then_recovers():
    wl = synth.small_workload(seed=59, n_queries=4, lmin=6, lmax=10, n_contigs=8, cmax=3000)
    s = 5
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s)
    cap = exp.size // 3
    h = P.ifa_create(hit_capacity=cap, segment_bytes=1 << 16)
    try:
        P.ifa_load_queries(h, wl.queries)
        P.ifa_set_max_subs(h, s)
        for a, b, pc in P.segment_pieces(wl.contig_len, 1000):
            P.ifa_push_segment(h, wl.ref[a:b], pc)
        got, over = P.ifa_drain_hits(h)
        assert over and got.size == cap                      # the first claims, then a hole
        assert set(tuples(got)) <= set(tuples(exp))
        assert P.ifa_get_digest(h)[0] == oracle.digest(exp)  # digest still exact
        # a second pass after a reset fits the ring when drained as it goes
        P.ifa_reset_results(h)
        buf = np.zeros(cap, P.HIT_DTYPE)
        parts = []
        for a, b, pc in P.segment_pieces(wl.contig_len, 300):
            P.ifa_push_segment(h, wl.ref[a:b], pc)
            n, over, _ = P.ifa_poll_hits(h, buf)
            assert not over
            parts.append(buf[:n].copy())
        rest, over = P.ifa_drain_hits(h)
        assert not over
        parts.append(rest)
        assert tuples(P.sort_hits(np.concatenate(parts))) == tuples(exp)
    finally:
        P.ifa_destroy(h)
