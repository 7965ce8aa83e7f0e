"""The tensor-core brute-force kernel (one-hot e4m3 GEMM on tcgen05) against
the CPU oracle: the same hit tuples, digest and per-query counts as the
plain definition, on ragged references with N runs, IUPAC bytes and lower
case, with query sets spanning several 128-entry tiles."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import gpu_scan, tuples

pytestmark = pytest.mark.gpu


def _queries(n, lmin, lmax, seed, n_frac=0.05):
    rng = np.random.default_rng(seed)
    qs = []
    for i in range(n):
        L = int(rng.integers(lmin, lmax + 1))
        b = rng.choice(np.frombuffer(b"ACGTacgt", np.uint8), L)
        b[rng.random(L) < n_frac] = ord("N")
        qs.append(bytes(b.astype(np.uint8)))
    return qs


@pytest.mark.parametrize("s,nq,seg", [(0, 3, 1 << 20), (3, 70, 4000), (6, 150, 1 << 20), (12, 40, 2500)])
def test_tensor_matches_oracle(s, nq, seg):
    wl = synth.small_workload(seed=90 + s, n_queries=2, lmin=10, lmax=60, n_contigs=14, cmin=1, cmax=6000,
                              plant_ks=[0, 1, 2, 3, 4, 5, 6] * 3, lowercase_frac=0.1)
    qs = wl.queries + _queries(nq, 5, 64, 1000 + s)
    got, over, dig, counts, _ = gpu_scan(qs, wl.ref, wl.contig_len, s, seg_bytes=seg,
                                         brute_kernel=P.IFA_BRUTE_TENSOR)
    exp = oracle.brute(qs, wl.ref, wl.contig_len, s)
    assert not over
    assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(qs)).tolist()


def test_tensor_equals_popcount_kernel_high_subs():
    """maxSubs at and above the query length: every window of every contig
    that fits the query is a hit."""
    wl = synth.small_workload(seed=97, n_queries=4, lmin=8, lmax=24, n_contigs=6, cmin=20, cmax=700)
    qs = wl.queries + _queries(130, 8, 32, 77)
    for s in (20, 40):
        a, *_ = gpu_scan(qs, wl.ref, wl.contig_len, s, brute_kernel=P.IFA_BRUTE_TENSOR, hit_capacity=1 << 24)
        b, *_ = gpu_scan(qs, wl.ref, wl.contig_len, s, brute_kernel=P.IFA_BRUTE_POPC, hit_capacity=1 << 24)
        assert tuples(a) == tuples(b)
    exp = oracle.brute(qs, wl.ref, wl.contig_len, 40)
    assert tuples(a) == tuples(exp)


def test_tensor_count_only_digest():
    wl = synth.small_workload(seed=98, n_queries=3, lmin=20, lmax=40, n_contigs=8, cmin=500, cmax=4000)
    qs = wl.queries + _queries(200, 20, 40, 5)
    _, _, dig, counts, _ = gpu_scan(qs, wl.ref, wl.contig_len, 7, count_only=1, brute_kernel=P.IFA_BRUTE_TENSOR)
    exp = oracle.brute(qs, wl.ref, wl.contig_len, 7)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(qs)).tolist()


def test_tensor_rejects_long_queries():
    ref = np.frombuffer(b"ACGT" * 100, np.uint8).copy()
    with pytest.raises(P.IfaError) as ei:
        gpu_scan([b"A" * 65], ref, np.array([400]), 2, brute_kernel=P.IFA_BRUTE_TENSOR)
    assert ei.value.status == P.IFA_ERR_INVALID_ARG


def test_tensor_wait_timeout_is_reported_and_context_survives():
    """Each tensor-core CTA withholds its first tile (a flag nothing else
    sets): the MMA's bounded wait runs out, ifa_flush reports TIMEOUT, and
    the same process then scans correctly again (the context is intact)."""
    wl = synth.small_workload(seed=99, n_queries=4, lmin=20, lmax=40, n_contigs=4, cmin=500, cmax=3000)
    qs = wl.queries + _queries(60, 20, 40, 8)
    with pytest.raises(P.IfaError) as ei:
        gpu_scan(qs, wl.ref, wl.contig_len, 3, brute_kernel=P.IFA_BRUTE_TENSOR, test_stall=1)
    assert ei.value.status == P.IFA_ERR_TIMEOUT
    got, over, dig, counts, _ = gpu_scan(qs, wl.ref, wl.contig_len, 3, brute_kernel=P.IFA_BRUTE_TENSOR)
    exp = oracle.brute(qs, wl.ref, wl.contig_len, 3)
    assert tuples(got) == tuples(exp)


@pytest.mark.parametrize("s,seg", [(5, 1 << 20), (6, 70_000)])
def test_tensor_dense_hits_in_long_contigs(s, seg):
    """Contigs much longer than a 1024-window tile, so most tiles lie inside
    one piece, and short queries at a high maxSubs, so that many windows of
    such tiles are hits (the per-tile fast path), with segments cutting the
    contigs (halo tiles take the checked path)."""
    wl = synth.small_workload(seed=150 + s, n_queries=4, lmin=10, lmax=30, n_contigs=7, cmin=15_000,
                              cmax=45_000, plant_ks=[0, 1, 2, 3] * 2)
    qs = wl.queries + _queries(70, 10, 30, 2000 + s, n_frac=0.02)
    got, over, dig, counts, _ = gpu_scan(qs, wl.ref, wl.contig_len, s, seg_bytes=seg,
                                         brute_kernel=P.IFA_BRUTE_TENSOR, hit_capacity=1 << 23)
    exp = oracle.brute(qs, wl.ref, wl.contig_len, s)
    assert not over
    assert exp.size > 100_000
    assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(qs)).tolist()


def test_tensor_pieces_starting_on_tile_boundaries():
    """Contig boundaries exactly at multiples of the 1024-window tile (a
    tile whose first window is a piece's first base is still one piece) and
    one base either side of them."""
    rng = np.random.default_rng(160)
    lens = np.array([1024 * 9, 1024 * 3, 1024 * 5 + 1, 1024 * 4 - 2, 1024 * 6, 1, 1024 * 2 + 1023, 1024 * 8],
                    np.int64)
    ref = rng.choice(np.frombuffer(b"ACGT", np.uint8), int(lens.sum()))
    qs = _queries(90, 8, 24, 161, n_frac=0.0)
    for i, q in enumerate(qs[:40]):
        # copies of the queries across and beside the boundaries
        a = int(np.cumsum(lens)[i % 7]) - len(q) // 2 + (i % 3) - 1
        ref[a:a + len(q)] = np.frombuffer(q, np.uint8)
    _, _, dig, counts, _ = gpu_scan(qs, ref, lens, 5, count_only=1, brute_kernel=P.IFA_BRUTE_TENSOR)
    exp = oracle.brute(qs, ref, lens, 5)
    assert exp.size > 50_000
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(qs)).tolist()
