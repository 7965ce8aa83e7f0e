"""Soft clipping at contig ends (Methods, Algorithm Design) on the GPU: the
clipped windows of every contig end, in brute-force and indexed mode, with
either brute-force kernel and in the serving loop, match the oracle tuple
for tuple (clips included), with contigs cut across segments and contigs
shorter than the queries."""
import numpy as np
import pytest

import oracle
import paper_2607_27291_b300 as P
import synth
from gpu_helpers import gpu_scan

pytestmark = pytest.mark.gpu


def tuples6(h):
    return sorted(zip(h["query"].tolist(), h["contig"].tolist(), h["pos"].tolist(),
                      h["strand"].tolist(), h["mismatches"].tolist(), h["clips"].tolist()))


def _workload(seed, pct=25):
    """A ragged small workload with overhanging copies of the queries planted
    at contig starts and ends (the aligned part only, overhang 1..C bases,
    one substitution in every other copy)."""
    wl = synth.small_workload(seed=seed, n_queries=6, lmin=8, lmax=60, n_contigs=24, cmin=1, cmax=900,
                              plant_ks=[0, 1, 2, 3] * 3, lowercase_frac=0.1)
    rng = np.random.default_rng(seed)
    starts = np.concatenate([[0], np.cumsum(wl.contig_len)[:-1]])
    ref = wl.ref
    for qi, q in enumerate(wl.queries):
        L = len(q)
        C = max(1, pct * L // 100)
        for rep in range(4):
            c = int(rng.integers(0, len(wl.contig_len)))
            n = int(wl.contig_len[c])
            o = int(rng.integers(1, C + 1))
            part = bytearray(q[o:] if rep % 2 == 0 else q[:L - o])
            if rep >= 2 and len(part) > 1:
                i = int(rng.integers(0, len(part)))
                part[i] = b"ACGT"[(b"ACGT".find(bytes([part[i]]).upper()) + 1) % 4]
            if len(part) > n:
                continue
            a = starts[c] if rep % 2 == 0 else starts[c] + n - len(part)
            ref[a:a + len(part)] = np.frombuffer(bytes(part), np.uint8)
    return wl


@pytest.mark.parametrize("pct,s,seg,mem", [(25, 3, 1 << 20, "host"), (10, 0, 700, "host"),
                                           (50, 6, 333, "device"), (25, 12, 2048, "pinned")])
def test_brute_clipped_windows_match_oracle(pct, s, seg, mem):
    wl = _workload(100 + pct + s, pct)
    got, over, dig, counts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, seg_bytes=seg, mem=mem,
                                         clip_pct=pct, brute_kernel=P.IFA_BRUTE_POPC)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s, clip_pct=pct)
    assert not over
    assert (exp["clips"] != 0).any()
    assert tuples6(got) == tuples6(exp)
    assert dig == oracle.digest(exp)
    assert counts.tolist() == np.bincount(exp["query"], minlength=len(wl.queries)).tolist()


def test_indexed_keeps_clipped_windows():
    wl = synth.small_workload(seed=131, n_queries=7, lmin=18, lmax=44, n_contigs=20, cmin=5, cmax=1200,
                              plant_ks=[0, 1, 2, 3] * 3)
    s, pct, trials = 3, 25, 10_000
    got, over, dig, _, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, mode=P.IFA_MODE_INDEXED, seg_bytes=1500,
                                    clip_pct=pct, minhits_trials=trials)
    plan = [oracle.choose_k(len(q), s, trials=trials) for q in wl.queries]
    exh = [1 if (st < 0 or any(c not in b"ACGTacgt" for c in q)) else 0 for (st, _, _), q in zip(plan, wl.queries)]
    exp = oracle.indexed(wl.queries, wl.ref, wl.contig_len, s, [p[1] for p in plan], [p[2] for p in plan], exh,
                         clip_pct=pct)
    assert not over
    assert tuples6(got) == tuples6(exp)
    assert dig == oracle.digest(exp)


def test_tensor_kernel_with_clipping():
    wl = _workload(141, 30)
    rng = np.random.default_rng(7)
    qs = wl.queries + [bytes(rng.choice(list(b"ACGT"), int(rng.integers(12, 50))).astype(np.uint8))
                       for _ in range(60)]
    got, *_ = gpu_scan(qs, wl.ref, wl.contig_len, 4, seg_bytes=1000, clip_pct=30,
                       brute_kernel=P.IFA_BRUTE_TENSOR, hit_capacity=1 << 22)
    exp = oracle.brute(qs, wl.ref, wl.contig_len, 4, clip_pct=30)
    assert tuples6(got) == tuples6(exp)


def _serve(wl, requests, n_slices, pct, arrive):
    """Serve requests [(queries, s, mode)], request i submitted before step
    arrive[i]; returns each request's (sorted hits, info)."""
    h = P.ifa_create(hit_capacity=1024, segment_bytes=1 << 20, minhits_trials=10_000, clip_pct=pct)
    try:
        for a, b, pc in P.segment_pieces(wl.contig_len, 1 << 12):
            P.ifa_ref_append(h, wl.ref[a:b], pc)
        P.ifa_serve_start(h, n_slices, 1 << 40, 1 << 16)
        ids, step = {}, 0
        while True:
            for i, t in enumerate(arrive):
                if t == step:
                    ids[i] = P.ifa_serve_submit(h, *requests[i])
            P.ifa_serve_step(h)
            step += 1
            infos = {i: P.ifa_serve_poll(h, r) for i, r in ids.items()}
            if len(ids) == len(requests) and all(v["state"] == 2 for v in infos.values()):
                break
            assert step < 100
        out = []
        for i in range(len(requests)):
            hits, over = P.ifa_serve_drain(h, ids[i], 1 << 16)
            assert not over
            out.append((P.sort_hits(hits), infos[i]))
        P.ifa_serve_stop(h)
        return out
    finally:
        P.ifa_destroy(h)


@pytest.mark.parametrize("n_slices,pct", [(1, 25), (7, 25), (13, 50)])
def test_serving_clipped_windows_match_oracle(n_slices, pct):
    """Requests joining at different slices, in both modes, each find every
    clipped window once: contigs cut across appends (pieces continued) and
    contigs shorter than the queries included."""
    wl = _workload(160 + n_slices, pct)
    trials = 10_000
    requests = [(wl.queries[:3], 3, P.IFA_MODE_BRUTE), (wl.queries[3:], 5, P.IFA_MODE_INDEXED),
                (wl.queries, 2, P.IFA_MODE_BRUTE)]
    got = _serve(wl, requests, n_slices, pct, [0, 1, 3])
    clipped = 0
    for (qs, s, mode), (hits, info) in zip(requests, got):
        if mode == P.IFA_MODE_BRUTE:
            exp = oracle.brute(qs, wl.ref, wl.contig_len, s, clip_pct=pct)
        else:
            plan = [oracle.choose_k(len(q), s, trials=trials) for q in qs]
            exh = [1 if (st < 0 or any(c not in b"ACGTacgt" for c in q)) else 0
                   for (st, _, _), q in zip(plan, qs)]
            exp = oracle.indexed(qs, wl.ref, wl.contig_len, s, [p[1] for p in plan], [p[2] for p in plan], exh,
                                 clip_pct=pct)
        clipped += int((exp["clips"] != 0).sum())
        assert tuples6(hits) == tuples6(exp)
        assert info["digest"] == oracle.digest(exp)
    assert clipped > 0
