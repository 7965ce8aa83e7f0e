"""Pins for the oracle's indexed-mode filter, MinHitsCalculator and Philox.

* Philox4x32-10 against the known-answer vectors published with Salmon et
  al. (SC'11) in the Random123 distribution.
* MinHits Monte Carlo against the exact survivor distribution obtained by
  enumerating every set of substitution positions (itertools), the
  closed forms at subs = 0 and subs >= L, and the P = 100% bound of
  Methods, indexed mode (validKmers - kEffective * maxSubs - maxClips),
  which must never exceed the true minimum survivor count.
* The seed-count filter against plain substring comparison, the
  one-mismatch closed form and its subset / equality relations to brute
  force."""
import itertools
import math
import re

import numpy as np
import pytest

import oracle
import synth

_RC = bytes.maketrans(b"ACGTacgt", b"TGCAtgca")


def _rc(q):
    return q.translate(_RC)[::-1]


def tuples(h):
    return sorted(zip(h["query"].tolist(), h["contig"].tolist(), h["pos"].tolist(),
                      h["strand"].tolist(), h["mismatches"].tolist()))


# ------------------------------------------------------------------ Philox

@pytest.mark.parametrize("ctr,key,expect", [
    ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
    ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
    ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
     [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
])
def test_philox_known_answers(ctr, key, expect):
    assert oracle.philox4x32_10(ctr, key).tolist() == expect


def test_philox_bits_balanced():
    words = np.array([oracle.philox4x32_10([i, 0, 7, 1], [1, 0]) for i in range(4096)],
                     dtype=np.uint32).ravel()
    bits = np.unpackbits(words.view(np.uint8))
    # 131072 fair bits: mean 0.5 +- 5 sigma
    assert abs(bits.mean() - 0.5) < 5 * 0.5 / math.sqrt(bits.size)


# ------------------------------------------------------------------ MinHits

def exact_survivors(L, s, k, step=1, mask_w=0):
    """Exact distribution of surviving k-mers over all C(L, s) position sets."""
    offs = list(range(0, L - k + 1, step))
    mlo = (k - mask_w) // 2
    cover = []
    for o in offs:
        cover.append({o + j for j in range(k) if not (mask_w and mlo <= j < mlo + mask_w)})
    counts = np.zeros(len(offs) + 1, dtype=np.int64)
    total = 0
    for pos in itertools.combinations(range(L), min(s, L)):
        ps = set(pos)
        counts[sum(1 for cv in cover if not (cv & ps))] += 1
        total += 1
    return counts / total, counts


def exact_threshold(p, num, den):
    tail = np.cumsum(p[::-1])[::-1]
    ok = [m for m in range(len(p)) if tail[m] * den >= num - 1e-12 * den]
    return max(ok), tail


@pytest.mark.parametrize("L,s,k,step,mask_w,num,den", [
    (12, 2, 4, 1, 0, 999, 1000),
    (12, 2, 4, 1, 0, 1, 2),
    (16, 3, 4, 1, 0, 9, 10),
    (14, 2, 5, 1, 1, 3, 4),
    (12, 3, 3, 2, 0, 1, 2),
    (20, 4, 8, 1, 0, 99, 100),
    (20, 1, 8, 1, 0, 999, 1000),
])
def test_minhits_matches_exact_enumeration(L, s, k, step, mask_w, num, den):
    T = 200_000
    m, hist = oracle.minhits(L, s, k, step, mask_w, 0, num, den, T, 1, with_hist=True)
    p, _ = exact_survivors(L, s, k, step, mask_w)
    assert hist.sum() == T
    freq = hist / T
    sigma = np.sqrt(np.maximum(p * (1 - p), 1e-12) / T)
    assert np.all(np.abs(freq - p) <= 5 * sigma + 1e-9), (freq, p)
    # cells the exact law forbids never occur
    assert np.all(hist[p == 0] == 0)
    m_exact, tail = exact_threshold(p, num, den)
    # compare thresholds unless the exact tail sits within 5 sigma of P
    P = num / den
    near = [abs(tail[j] - P) < 5 * math.sqrt(P * (1 - P) / T) for j in (m_exact, min(m_exact + 1, len(p) - 1))]
    if not any(near):
        assert m == m_exact


def test_quantile_rule_on_hand_histograms():
    # "found with probability P": a threshold met by exactly P of the trials counts
    assert oracle.minhits_quantile([50, 50], 1, 2) == 1
    assert oracle.minhits_quantile([51, 49], 1, 2) == 0
    assert oracle.minhits_quantile([0, 1, 998, 1], 999, 1000) == 2
    assert oracle.minhits_quantile([0, 2, 997, 1], 999, 1000) == 1
    assert oracle.minhits_quantile([0, 0, 0, 10], 999, 1000) == 3
    assert oracle.minhits_quantile([10, 0, 0, 0], 1, 1000) == 0


@pytest.mark.parametrize("L,k,step", [(20, 8, 1), (33, 14, 1), (40, 10, 3)])
def test_minhits_closed_forms(L, k, step):
    K = len(range(0, L - k + 1, step))
    m0, h0 = oracle.minhits(L, 0, k, step, trials=1000, with_hist=True)
    assert m0 == K and h0[K] == 1000
    mL, hL = oracle.minhits(L, L + 3, k, step, trials=1000, with_hist=True)
    assert mL == 0 and hL[0] == 1000


@pytest.mark.parametrize("L,s,k,mask_w,clips", [(20, 1, 8, 0, 0), (20, 2, 5, 0, 0),
                                                  (30, 2, 8, 2, 1), (40, 1, 14, 0, 3)])
def test_deterministic_bound(L, s, k, mask_w, clips):
    K = L - k + 1
    bound = oracle.minhits(L, s, k, 1, mask_w, clips, 1, 1)
    assert bound == max(0, K - (k - mask_w) * s - clips)
    # the bound never exceeds the true worst case (without clips)
    _, counts = exact_survivors(L, s, k, 1, mask_w)
    worst = min(c for c in range(len(counts)) if counts[c] > 0)
    assert oracle.minhits(L, s, k, 1, mask_w, 0, 1, 1) <= worst


def test_minhits_deterministic_and_seeded():
    a = oracle.minhits(30, 4, 8, trials=50_000, seed=1, with_hist=True)
    b = oracle.minhits(30, 4, 8, trials=50_000, seed=1, with_hist=True)
    c = oracle.minhits(30, 4, 8, trials=50_000, seed=2, with_hist=True)
    assert a[0] == b[0] and (a[1] == b[1]).all()
    assert not (a[1] == c[1]).all()


def test_choose_k_closed_forms():
    kl = (8, 9, 10, 12, 14)
    # no substitutions: every k qualifies, the longest that fits is taken
    for L in (8, 11, 13, 20, 40):
        st, k, m = oracle.choose_k(L, 0, kl, trials=2000)
        kk = max(x for x in kl if x <= L)
        assert (st, k, m) == (1, kk, L - kk + 1)
    # all positions substituted: nothing survives, smallest k clamped to 1
    st, k, m = oracle.choose_k(20, 20, kl, trials=2000)
    assert (st, k, m) == (0, 8, 1)
    # too short for any listed k
    assert oracle.choose_k(7, 1, kl, trials=2000)[0] == -1
    # P = 100%: longest k whose bound K - k*s is at least 1
    for L, s in ((40, 1), (40, 2), (30, 2), (25, 3)):
        st, k, m = oracle.choose_k(L, s, kl, num=1, den=1)
        good = [x for x in kl if x <= L and (L - x + 1) - x * s >= 1]
        if good:
            assert (st, k, m) == (1, max(good), (L - max(good) + 1) - max(good) * s)
        else:
            assert (st, k, m) == (0, 8, 1)


# ------------------------------------------------------------------ seed filter

def _text_seeded(q, ctg, p, k, step, mask_w):
    """Plain-text seed test: some offset's unmasked bases equal, all ACGT."""
    L = len(q)
    mlo = (k - mask_w) // 2
    qs = q.upper()
    rs = bytes(ctg[p:p + L]).upper()
    n = 0
    for o in range(0, L - k + 1, step):
        keep = [j for j in range(k) if not (mask_w and mlo <= j < mlo + mask_w)]
        a = bytes(qs[o + j] for j in keep)
        b = bytes(rs[o + j] for j in keep)
        if a == b and not re.search(rb"[^ACGT]", a):
            n += 1
    return n


@pytest.fixture(scope="module")
def wl_idx():
    return synth.small_workload(seed=31, n_queries=5, lmin=14, lmax=36, n_contigs=8,
                                cmin=100, cmax=1500, plant_ks=[0, 1, 1, 2, 2, 3, 4, 6] * 2)


@pytest.mark.parametrize("k,step,mask_w", [(5, 1, 0), (6, 2, 0), (7, 1, 3)])
def test_minhits_one_equals_text_seed_test(wl_idx, k, step, mask_w):
    wl = wl_idx
    s = 6
    nq = len(wl.queries)
    got = tuples(oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, [k] * nq, [1] * nq,
                                [0] * nq, step, mask_w))
    brute = tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, s))
    expect = []
    for h in brute:
        q = wl.queries[h[0]]
        qq = q if h[3] == 0 else _rc(q)
        if _text_seeded(qq, wl.contig(h[1]), h[2], k, step, mask_w) >= 1:
            expect.append(h)
    assert got == expect


@pytest.mark.parametrize("step,mask_w", [(1, 0), (2, 0), (1, 2), (3, 1)])
def test_thresholds_above_one_equal_text_seed_counts(wl_idx, step, mask_w):
    """Per-query k and minHits (2..6): a brute-force hit is kept exactly when
    its plain-text seed count reaches the query's threshold."""
    wl = wl_idx
    s = 5
    nq = len(wl.queries)
    ks = [(5, 6, 7, 8, 6)[i % 5] for i in range(nq)]
    mh = [(2, 3, 4, 6, 2)[i % 5] for i in range(nq)]
    got = tuples(oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, ks, mh, [0] * nq, step, mask_w))
    brute = tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, s))
    expect = []
    for h in brute:
        q = wl.queries[h[0]]
        qq = q if h[3] == 0 else _rc(q)
        if _text_seeded(qq, wl.contig(h[1]), h[2], ks[h[0]], step, mask_w) >= mh[h[0]]:
            expect.append(h)
    assert len(expect) < len(brute)       # the thresholds filter something
    assert got == expect


def test_n_is_never_part_of_a_seed():
    # an N opposite an N is still a mismatch: no k-mer holding it is a seed
    ctg = np.frombuffer(b"ACGTNACGTA", np.uint8).copy()
    assert oracle.window_seeds(b"ACGTNACGTA", 0, ctg, 0, 10) == 0
    assert oracle.window_seeds(b"ACGTNACGTA", 0, ctg, 0, 4) == 3      # ACGT, ACGT, CGTA
    assert oracle.window_seeds(b"ACGTNACGTA", 0, ctg, 0, 5) == 1      # ACGTA only
    assert oracle.window_mismatches(b"ACGTNACGTA", 0, ctg, 0) == 1


def test_indexed_subset_and_degenerate_cases(wl_idx):
    wl = wl_idx
    nq = len(wl.queries)
    s = 4
    brute = tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, s))
    idx = tuples(oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, [8] * nq, [3] * nq,
                                [0] * nq))
    assert set(idx) <= set(brute)
    # exhaustive queries and a zero threshold keep every brute hit
    assert tuples(oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, [8] * nq, [3] * nq,
                                 [1] * nq)) == brute
    assert tuples(oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, [8] * nq, [0] * nq,
                                 [0] * nq)) == brute
    # k = L with threshold 1 keeps exactly the error-free windows
    kq = [len(q) for q in wl.queries]
    full = tuples(oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, kq, [1] * nq, [0] * nq))
    assert full == [h for h in brute if h[4] == 0]


def test_seed_counts_closed_forms(wl_idx):
    wl = wl_idx
    k = 6
    hits = oracle.brute(wl.queries, wl.ref, wl.contig_len, 3)
    for h in hits:
        q = wl.queries[h["query"]]
        L = len(q)
        K = L - k + 1
        ctg = wl.contig(int(h["contig"]))
        sd = oracle.window_seeds(q, int(h["strand"]), ctg, int(h["pos"]), k)
        mm = int(h["mismatches"])
        assert K - k * mm <= sd <= K
        if mm == 0:
            assert sd == K
        if mm == 1:
            qq = (q if h["strand"] == 0 else _rc(q)).upper()
            rr = bytes(ctg[h["pos"]:h["pos"] + L]).upper()
            i = next(j for j in range(L) if qq[j] != rr[j])
            killed = min(i, L - k) - max(0, i - k + 1) + 1
            assert sd == K - killed
