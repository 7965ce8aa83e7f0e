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


def test_noalloc_rejects_sizes_beyond_its_limits():
    q = [b"ACGTACGT"]
    with pytest.raises(P.IfaError) as ei:
        P.ifa_scan_brute_noalloc(0, q, 16, (32 << 20) + 1, [(0, 0, 0, (32 << 20) + 1, True)], 1,
                                 16, 16, 16)
    assert ei.value.status == P.IFA_ERR_INVALID_ARG and "32 MiB" in str(ei.value)
    with pytest.raises(P.IfaError) as ei:
        P.ifa_scan_brute_noalloc(0, [b"ACGT"] * 257, 16, 100, [(0, 0, 0, 100, True)], 1, 16, 16, 16)
    assert ei.value.status == P.IFA_ERR_INVALID_ARG and "256 queries" in str(ei.value)
