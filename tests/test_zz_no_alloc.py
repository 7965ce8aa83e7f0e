"""ifa_scan_brute_noalloc against the regular handle-based entry points.

The allocation-free entry point is for callers that cannot allocate device
memory where they scan -- for example code running under a framework whose
caching allocator already holds the GPU's memory, so that any cudaMalloc
outside it fails.  Such a caller owns every buffer; here the test plays that
caller and allocates its buffers with torch before the calls.  Two calls in
a row (different queries, reference and maxSubs, so the second one starts
from the first one's leftovers in the library's scratch array) must each
give exactly the hits, digest and per-query counts of the handle API on the
same input.  This file is collected last so that a failure here cannot hide
any other test."""
import numpy as np
import pytest

import paper_2607_27291_b300 as P
import synth
from gpu_helpers import gpu_scan, tuples

pytestmark = pytest.mark.gpu


def _noalloc(queries, ref, lens, s, cap=1 << 18):
    import torch
    ref_dev = torch.from_numpy(np.ascontiguousarray(ref)).cuda()
    hits = torch.zeros(cap * 16, dtype=torch.uint8, device="cuda")
    counters = torch.zeros(5, dtype=torch.int64, device="cuda")
    counts = torch.zeros(len(queries), dtype=torch.int64, device="cuda")
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    pieces = [(i, 0, int(a), int(n), True) for i, (a, n) in enumerate(zip(starts, lens))]
    torch.cuda.synchronize()
    P.ifa_scan_brute_noalloc(0, queries, ref_dev.data_ptr(), ref.size, pieces, s, hits.data_ptr(),
                             cap, counters.data_ptr(), counts.data_ptr(), None)
    torch.cuda.synchronize()
    c = counters.cpu().numpy().astype(np.uint64)
    head = int(c[0])
    assert int(c[1]) == 0 and head <= cap, "hit buffer too small for this test"
    got = hits[:head * 16].cpu().numpy().view(P.HIT_DTYPE)
    return P.sort_hits(got), (int(c[2]), int(c[3]), int(c[4])), counts.cpu().numpy().astype(np.uint64)


def test_noalloc_matches_handle_api_on_two_calls():
    wl = synth.small_workload(seed=61, n_queries=12, lmin=5, lmax=70, n_contigs=40, cmin=1,
                              cmax=20000, lowercase_frac=0.05)
    calls = [
        (wl.queries, wl.ref, wl.contig_len, 3),
        (wl.queries[3:8], wl.ref[:int(wl.contig_len[:25].sum())], wl.contig_len[:25], 6),
    ]
    for queries, ref, lens, s in calls:
        got, dig, counts = _noalloc(queries, ref, lens, s)
        exp, over, edig, ecounts, _ = gpu_scan(queries, ref, lens, s)
        assert not over
        assert tuples(got) == tuples(exp)
        assert dig == edig
        assert counts.tolist() == ecounts.tolist()


def test_noalloc_many_long_queries_several_launches():
    """256 queries of up to 255 bases: 8 words per entry, so the 512 entries
    need several scan launches (each launch holds what fits its shared
    memory); maxSubs 2^32 - 1 must report every window."""
    wl = synth.small_workload(seed=67, n_queries=256, lmin=18, lmax=255, n_contigs=30, cmin=1,
                              cmax=60000, plant_ks=[0, 1, 2, 3])
    for s in (3, 6):
        got, dig, counts = _noalloc(wl.queries, wl.ref, wl.contig_len, s, cap=1 << 20)
        exp, over, edig, ecounts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, hit_capacity=1 << 20)
        assert not over
        assert tuples(got) == tuples(exp)
        assert dig == edig
        assert counts.tolist() == ecounts.tolist()
    # maxSubs 2^32 - 1 (no upper limit): every window of every contig, both strands
    q = wl.queries[:4]
    lens = wl.contig_len[:5]
    got, dig, _ = _noalloc(q, wl.ref[:int(lens.sum())], lens, 0xFFFFFFFF, cap=1 << 22)
    n_win = sum(2 * int(np.maximum(lens - len(x) + 1, 0).sum()) for x in q)
    assert got.size == n_win == dig[0]


def test_noalloc_call_under_memory_pressure_allocates_nothing():
    """The caller this entry point is for has handed nearly all device memory
    to its own allocator.  After the set-up call (nq = 0) and one warm call,
    a call made while torch holds all but a few hundred MB of the free memory
    must succeed, give the handle API's hits, and change neither the device's
    free bytes nor torch's reserved bytes."""
    import torch
    wl = synth.small_workload(seed=71, n_queries=40, lmin=18, lmax=50, n_contigs=20, cmin=100,
                              cmax=50000, plant_ks=[0, 1, 2])
    exp, over, edig, ecounts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, 4)
    assert not over
    P.ifa_scan_brute_noalloc(0, [], 0, 0, [], 0, 0, 0, 0)   # set-up only
    cap = 1 << 18
    ref_dev = torch.from_numpy(np.ascontiguousarray(wl.ref)).cuda()
    hits = torch.zeros(cap * 16, dtype=torch.uint8, device="cuda")
    counters = torch.zeros(5, dtype=torch.int64, device="cuda")
    counts = torch.zeros(len(wl.queries), dtype=torch.int64, device="cuda")
    starts = np.concatenate([[0], np.cumsum(wl.contig_len)[:-1]])
    pieces = [(i, 0, int(a), int(n), True) for i, (a, n) in enumerate(zip(starts, wl.contig_len))]

    def call():
        P.ifa_scan_brute_noalloc(0, wl.queries, ref_dev.data_ptr(), wl.ref.size, pieces, 4,
                                 hits.data_ptr(), cap, counters.data_ptr(), counts.data_ptr(), None)
        torch.cuda.synchronize()

    call()   # warm: the kernels' first launches happen here
    free, _ = torch.cuda.mem_get_info()
    hog = torch.empty(max(0, free - (384 << 20)), dtype=torch.uint8, device="cuda")
    try:
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        res0 = torch.cuda.memory_reserved()
        counters.zero_()
        call()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        assert torch.cuda.memory_reserved() == res0
    finally:
        del hog
        torch.cuda.empty_cache()
    c = counters.cpu().numpy().astype(np.uint64)
    head = int(c[0])
    assert int(c[1]) == 0 and head <= cap
    got = P.sort_hits(hits[:head * 16].cpu().numpy().view(P.HIT_DTYPE))
    assert tuples(got) == tuples(exp)
    assert (int(c[2]), int(c[3]), int(c[4])) == edig
    assert counts.cpu().numpy().astype(np.uint64).tolist() == ecounts.tolist()


def test_noalloc_refuses_a_capturing_stream():
    """The call reads host memory freed on return, so capture is refused
    before anything is enqueued (the capture itself stays valid)."""
    import torch
    wl = synth.small_workload(seed=73, n_queries=3, lmin=18, lmax=30, n_contigs=4, cmin=100, cmax=1000)
    ref_dev = torch.from_numpy(np.ascontiguousarray(wl.ref)).cuda()
    hits = torch.zeros(1024 * 16, dtype=torch.uint8, device="cuda")
    counters = torch.zeros(5, dtype=torch.int64, device="cuda")
    starts = np.concatenate([[0], np.cumsum(wl.contig_len)[:-1]])
    pieces = [(i, 0, int(a), int(n), True) for i, (a, n) in enumerate(zip(starts, wl.contig_len))]
    P.ifa_scan_brute_noalloc(0, [], 0, 0, [], 0, 0, 0, 0)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            counters.add_(1)
            try:
                P.ifa_scan_brute_noalloc(0, wl.queries, ref_dev.data_ptr(), wl.ref.size, pieces, 2,
                                         hits.data_ptr(), 1024, counters.data_ptr(), 0, s)
            except P.IfaError as e:
                err = e
    assert err is not None and err.status == P.IFA_ERR_INVALID_ARG and "captured" in str(err)
    g.replay()
    torch.cuda.synchronize()
    assert counters.cpu().tolist() == [1, 1, 1, 1, 1]


def test_noalloc_rejects_sizes_beyond_its_limits():
    q = [b"ACGTACGT"]
    with pytest.raises(P.IfaError) as ei:
        P.ifa_scan_brute_noalloc(0, q, 16, (32 << 20) + 1, [(0, 0, 0, (32 << 20) + 1, True)], 1,
                                 16, 16, 16)
    assert ei.value.status == P.IFA_ERR_INVALID_ARG and "32 MiB" in str(ei.value)
    with pytest.raises(P.IfaError) as ei:
        P.ifa_scan_brute_noalloc(0, [b"ACGT"] * 257, 16, 100, [(0, 0, 0, 100, True)], 1, 16, 16, 16)
    assert ei.value.status == P.IFA_ERR_INVALID_ARG and "256 queries" in str(ei.value)
