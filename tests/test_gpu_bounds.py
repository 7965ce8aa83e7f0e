"""The bounds-checked build (libifa_bc.so, -DIFA_BOUNDS_CHECK) on the GPU.

Every read of the packed reference checks its index against its
allocation and records the first one out of range in a device word; no
read traps.  In a child process that loads that build, passes over a
ragged workload (Ns, contigs shorter than the queries, segments of a few
hundred bases, soft clipping) in brute force with both kernels, indexed
mode, a batch of sets and a serving request must equal the oracle with the
word still zero.  The default build reports that it checks nothing.

No test here makes a read go out of range on purpose: the checks are
there to catch a fault in the index arithmetic, not to be driven into."""
import os
import subprocess
import sys

import pytest

import paper_2607_27291_b300 as P
from paper_2607_27291_b300 import build as B

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import os, sys
sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
import numpy as np
import oracle, synth
import paper_2607_27291_b300 as P
from gpu_helpers import gpu_scan, tuples
assert os.path.basename(P.LIB_PATH) == "libifa_bc.so", P.LIB_PATH
enabled, first = P.ifa_bounds_check(0, reset=True)
assert enabled and first == 0

def t6(h):
    return sorted(zip(*(h[f].tolist() for f in ("query", "contig", "pos", "strand", "mismatches", "clips"))))

wl = synth.small_workload(seed=501, n_queries=6, lmin=12, lmax=60, n_contigs=30, cmin=1, cmax=5000,
                          n_frac=0.01, plant_ks=[0, 1, 2, 3] * 3, lowercase_frac=0.1)
for s, seg, kern in ((3, 777, P.IFA_BRUTE_POPC), (7, 1 << 16, P.IFA_BRUTE_POPC), (4, 1500, P.IFA_BRUTE_TENSOR)):
    got, over, dig, counts, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, s, seg_bytes=seg,
                                         brute_kernel=kern, clip_pct=25)
    exp = oracle.brute(wl.queries, wl.ref, wl.contig_len, s, clip_pct=25)
    assert not over and t6(got) == t6(exp), (s, seg, kern)
    assert dig == oracle.digest(exp)

trials = 10_000
plan = [oracle.choose_k(len(q), 3, trials=trials) for q in wl.queries]
exh = [1 if (st < 0 or any(c not in b"ACGTacgt" for c in q)) else 0 for (st, _, _), q in zip(plan, wl.queries)]
got, over, dig, _, _ = gpu_scan(wl.queries, wl.ref, wl.contig_len, 3, mode=P.IFA_MODE_INDEXED, seg_bytes=999,
                                minhits_trials=trials)
exp = oracle.indexed(wl.queries, wl.ref, wl.contig_len, 3, [p[1] for p in plan], [p[2] for p in plan], exh)
assert not over and tuples(got) == tuples(exp)

# a batch of two brute-force sets and a serving request on the store
h = P.ifa_create(hit_capacity=1 << 20, segment_bytes=1 << 16)
try:
    for a, b, pc in P.segment_pieces(wl.contig_len, 4096):
        P.ifa_ref_append(h, wl.ref[a:b], pc)
    sets = [(wl.queries[:3], 2), (wl.queries[3:], 5)]
    firsts = [P.ifa_set_add(h, qs, s, P.IFA_MODE_BRUTE)[1] for qs, s in sets]
    P.ifa_batch_run(h, P.IFA_BATCH_PERSISTENT, len(sets))
    hits, over = P.ifa_drain_hits(h)
    assert not over
    want = []
    for (qs, s), f in zip(sets, firsts):
        e = oracle.brute(qs, wl.ref, wl.contig_len, s)
        want += [(q + f,) + t[1:] for t in tuples(e) for q in [t[0]]]
    assert tuples(P.sort_hits(hits)) == sorted(want)
    P.ifa_serve_start(h, 5, 1 << 40, 1 << 16)
    rid = P.ifa_serve_submit(h, wl.queries, 4, P.IFA_MODE_BRUTE)
    while P.ifa_serve_step(h)[0]:
        pass
    hits, over = P.ifa_serve_drain(h, rid, 1 << 16)
    assert not over and tuples(P.sort_hits(hits)) == tuples(oracle.brute(wl.queries, wl.ref, wl.contig_len, 4))
    P.ifa_serve_stop(h)
finally:
    P.ifa_destroy(h)

enabled, first = P.ifa_bounds_check(0)
assert enabled and first == 0, hex(first)
print("BOUNDS-CHECKED OK")
"""


def test_default_build_checks_nothing():
    assert P.ifa_bounds_check(0) == (False, 0)


def test_bounds_checked_build_is_exact_and_reads_in_range():
    assert os.path.exists(B.BC_LIB_PATH)
    env = dict(os.environ, IFA_LIB=B.BC_LIB_PATH)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "BOUNDS-CHECKED OK" in r.stdout
