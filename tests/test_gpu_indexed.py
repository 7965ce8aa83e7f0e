"""MinHitsCalculator and indexed mode on the GPU against the oracle.

MinHits runs on counter-based Philox on both sides, so thresholds must be
bit-identical; the indexed hit set must equal the oracle's seed-filtered
brute-force set exactly."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import gpu_scan, tuples

pytestmark = pytest.mark.gpu


def test_minhits_bit_exact_grid():
    L, S, K = [], [], []
    for l in range(18, 51, 4):
        for s in (0, 1, 2, 4, 8, 16):
            for k in (8, 9, 10, 12, 14):
                if k <= l:
                    L.append(l), S.append(s), K.append(k)
    got = P.ifa_minhits(0, L, S, K, trials=100_000, seed=1)
    exp = [oracle.minhits(l, s, k, trials=100_000, seed=1) for l, s, k in zip(L, S, K)]
    assert got.tolist() == exp


@pytest.mark.parametrize("step,mask_w,num,den,seed", [(2, 0, 9, 10, 3), (1, 3, 99, 100, 5),
                                                      (3, 1, 1, 2, 7), (1, 0, 1, 1, 1)])
def test_minhits_options_bit_exact(step, mask_w, num, den, seed):
    L, S, K = [], [], []
    for l in (20, 33, 47, 64, 100):
        for s in (0, 2, 5):
            for k in (8, 11, 14):
                L.append(l), S.append(s), K.append(k)
    got = P.ifa_minhits(0, L, S, K, step=step, mask_width=mask_w, num=num, den=den,
                        trials=20_000, seed=seed)
    exp = [oracle.minhits(l, s, k, step, mask_w, 0, num, den, 20_000, seed)
           for l, s, k in zip(L, S, K)]
    assert got.tolist() == exp


def test_query_plan_matches_oracle_choice():
    queries = synth.random_queries(40, 18, 50, 11) + [b"ACGTNACGTACGTACGTACG"]
    for s in (0, 2, 4, 8):
        h = P.ifa_create(minhits_trials=50_000, segment_bytes=1 << 16, hit_capacity=1024)
        try:
            P.ifa_load_queries(h, queries)
            P.ifa_set_max_subs(h, s)
            k, m, ex = P.ifa_get_query_plan(h, len(queries))
        finally:
            P.ifa_destroy(h)
        for i, q in enumerate(queries):
            st, kk, mm = oracle.choose_k(len(q), s, trials=50_000)
            assert (k[i], m[i]) == (kk, mm), (i, s)
            assert ex[i] == (1 if (st < 0 or b"N" in q) else 0)


@pytest.mark.parametrize("s", [0, 2, 4, 8])
@pytest.mark.parametrize("seg_bytes", [None, 1601])
def test_indexed_matches_oracle(s, seg_bytes):
    wl = synth.small_workload(seed=41, n_queries=12, lmin=12, lmax=45, n_contigs=12, cmin=50,
                              cmax=4000, plant_ks=[0, 1, 2, 3, 4, 5, 6, 8] * 3)
    trials = 20_000
    got, over, dig, counts, stats = gpu_scan(wl.queries, wl.ref, wl.contig_len, s,
                                             mode=P.IFA_MODE_INDEXED, seg_bytes=seg_bytes,
                                             minhits_trials=trials)
    plan = [oracle.choose_k(len(q), s, trials=trials) for q in wl.queries]
    exh = [1 if (st < 0 or any(c not in b"ACGTacgt" for c in q)) else 0
           for (st, _, _), q in zip(plan, wl.queries)]
    exp = oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, [p[1] for p in plan],
                         [p[2] for p in plan], exh)
    assert not over
    assert tuples(got) == tuples(exp)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(wl.queries)).tolist()
    brute = set(tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, s)))
    assert set(tuples(got)) <= brute


@pytest.mark.parametrize("step,mask_w,klist", [(2, 0, (8, 10)), (1, 2, (9, 11)), (3, 1, (6, 7)),
                                                (1, 0, (13, 15)), (2, 1, (14, 16))])
def test_indexed_step_and_mask(step, mask_w, klist):
    wl = synth.small_workload(seed=43, n_queries=8, lmin=14, lmax=40, n_contigs=10, cmin=100,
                              cmax=3000, plant_ks=[0, 1, 2, 3] * 4)
    s, trials = 3, 10_000
    got, *_ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, mode=P.IFA_MODE_INDEXED,
                       seg_bytes=2500, minhits_trials=trials, kmer_step=step, mask_width=mask_w,
                       k_list=list(klist))
    plan = [oracle.choose_k(len(q), s, klist, step, mask_w, trials=trials) for q in wl.queries]
    exh = [1 if (st < 0 or any(c not in b"ACGTacgt" for c in q)) else 0
           for (st, _, _), q in zip(plan, wl.queries)]
    exp = oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, [p[1] for p in plan],
                         [p[2] for p in plan], exh, step, mask_w)
    assert tuples(got) == tuples(exp)


def test_indexed_exact_bound_finds_all_seeded_hits():
    """P = 100% (deterministic bound): every brute hit with >= 1 error-free
    k-mer is reported (Methods, indexed mode)."""
    wl = synth.small_workload(seed=47, n_queries=10, lmin=20, lmax=40, n_contigs=10, cmin=200,
                              cmax=3000, plant_ks=[0, 1, 2, 3, 4] * 4)
    s = 4
    got, *_ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, mode=P.IFA_MODE_INDEXED,
                       minhits_num=1, minhits_den=1)
    plan = [oracle.choose_k(len(q), s, num=1, den=1) for q in wl.queries]
    brute = oracle.brute(wl.queries, wl.ref, wl.contig_len, s)
    seeded = []
    for h in tuples(brute):
        q = wl.queries[h[0]]
        if oracle.window_seeds(q, h[3], wl.contig(h[1]), h[2], plan[h[0]][1]) >= 1:
            seeded.append(h)
    assert set(seeded) <= set(tuples(got))
