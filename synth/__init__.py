"""Seeded synthetic inputs for the indel-free (Hamming) scan.

This module only draws inputs: query sequences, reference contigs (ASCII),
N-runs and planted hits, and it cuts the reference into streamed segments.
It holds none of the method's arithmetic (no mismatch counting, no seeds,
no Monte Carlo thresholds); both the CUDA path's tests and the CPU oracle
read the same arrays from here.

Recipe (the paper's datasets are not available, so these stand in for them;
the paper's own test reads are simulated in the same spirit, Methods,
"Benchmarking"):

* bases are i.i.d. with P(G) = P(C) = gc/2 and P(A) = P(T) = (1 - gc)/2,
  drawn per 64 Mbp chunk from its own generator so any chunk can be
  regenerated alone;
* contig lengths are log-normal (mu = ln sqrt(ab), sigma = ln(b/a)/6,
  resampled into [a, b]) or log-uniform in [a, b]; contigs are drawn until
  the total reaches the target and the last one is cut (never below a);
* N-runs have lengths uniform in [10, 1000] and are dropped at uniform
  positions of the concatenated reference until the N fraction is reached;
* a plant picks a query, a contig long enough, a position and a strand
  uniformly, avoiding N-runs and other plants, and writes the query (or its
  reverse complement for strand 1) with exactly k distinct positions changed,
  each to one of the three other bases uniformly.
"""
from __future__ import annotations

import bisect
import concurrent.futures as _cf
import dataclasses
import os
from typing import List, Optional, Sequence

import numpy as np

CHUNK = 1 << 26          # bases per independently seeded chunk
_ACGT = np.frombuffer(b"ACGT", dtype=np.uint8)
# complement used only to write minus-strand plants
_PLANT_COMP = {ord("A"): ord("T"), ord("C"): ord("G"), ord("G"): ord("C"), ord("T"): ord("A")}

# stream ids inside one seed
_S_QUERIES, _S_LENGTHS, _S_BASES, _S_NRUNS, _S_PLANTS, _S_GC = 0, 1, 2, 3, 4, 5


def _rng(seed: int, stream: int, sub: int = 0) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream), int(sub)])


def random_queries(n: int, lmin: int, lmax: int, seed: int) -> List[bytes]:
    """n queries of uniform ACGT with lengths uniform in [lmin, lmax]."""
    rng = _rng(seed, _S_QUERIES)
    lens = rng.integers(lmin, lmax + 1, size=n)
    out = []
    for L in lens:
        out.append(_ACGT[rng.integers(0, 4, size=int(L))].tobytes())
    return out


def contig_lengths(total: int, a: int, b: int, dist: str, seed: int,
                   fixed: Optional[int] = None) -> np.ndarray:
    """Contig lengths summing to about `total` (the last one cut, minimum a)."""
    if fixed is not None:
        n = total // fixed
        return np.full(n, fixed, dtype=np.int64)
    rng = _rng(seed, _S_LENGTHS)
    out = []
    acc = 0
    mu = np.log(np.sqrt(float(a) * float(b)))
    sigma = np.log(float(b) / float(a)) / 6.0
    while acc < total:
        draws = (np.exp(rng.normal(mu, sigma, size=4096)) if dist == "lognormal"
                 else np.exp(rng.uniform(np.log(a), np.log(b), size=4096)))
        draws = draws[(draws >= a) & (draws <= b)].astype(np.int64)
        for L in draws:
            L = int(L)
            if acc + L >= total:
                L = max(a, total - acc)
                out.append(L)
                acc += L
                break
            out.append(L)
            acc += L
        # loop re-checks acc
    return np.asarray(out, dtype=np.int64)


def _fill_chunk(out: np.ndarray, start: int, n: int, gc_of, seed: int, ci: int):
    rng = _rng(seed, _S_BASES, ci)
    r = rng.random(n, dtype=np.float32)
    gc = gc_of(start, n)
    if np.isscalar(gc):
        t1 = np.float32((1.0 - gc) / 2.0)
        t2 = np.float32(0.5)
        t3 = np.float32((1.0 + gc) / 2.0)
    else:
        t1 = ((1.0 - gc) / 2.0).astype(np.float32)
        t2 = np.float32(0.5)
        t3 = ((1.0 + gc) / 2.0).astype(np.float32)
    # order A, C, G, T with cumulative (1-gc)/2, 1/2, (1+gc)/2
    code = (r >= t1).astype(np.uint8)
    code += (r >= t2)
    code += (r >= t3)
    out[start:start + n] = _ACGT[code]


def random_bases(total: int, gc, seed: int, threads: Optional[int] = None,
                 contig_len: Optional[np.ndarray] = None,
                 contig_gc: Optional[np.ndarray] = None, window=None) -> np.ndarray:
    """ASCII bases (uint8) with the GC model above.

    `gc` is a float, or None together with per-contig `contig_gc` values
    (then `contig_len` gives the contig layout).  `window` = (a, b) returns
    only bases [a, b) of the `total`, equal to that slice of the whole."""
    if window is not None:
        a, b = int(window[0]), int(window[1])
        if contig_gc is not None:
            raise ValueError("window needs a fixed gc")
        out = np.empty(b - a, dtype=np.uint8)
        tmp = np.empty(CHUNK, dtype=np.uint8)
        for ci in range(a // CHUNK, (b + CHUNK - 1) // CHUNK):
            c0 = ci * CHUNK
            n = min(CHUNK, total - c0)
            _fill_chunk(tmp, 0, n, lambda st, k: float(gc), seed, ci)
            lo, hi = max(a, c0), min(b, c0 + n)
            out[lo - a:hi - a] = tmp[lo - c0:hi - c0]
        return out
    out = np.empty(total, dtype=np.uint8)
    if contig_gc is not None:
        starts = np.concatenate([[0], np.cumsum(contig_len)[:-1]])

        def gc_of(start, n):
            pos = np.arange(start, start + n, dtype=np.int64)
            idx = np.searchsorted(starts, pos, side="right") - 1
            return contig_gc[idx]
    else:
        def gc_of(start, n):
            return float(gc)
    nchunks = (total + CHUNK - 1) // CHUNK
    threads = threads or min(32, os.cpu_count() or 1)
    with _cf.ThreadPoolExecutor(threads) as ex:
        futs = [ex.submit(_fill_chunk, out, i * CHUNK, min(CHUNK, total - i * CHUNK),
                          gc_of, seed, i) for i in range(nchunks)]
        for f in futs:
            f.result()
    return out


class _Occupied:
    """Sorted disjoint half-open intervals of the concatenated reference."""

    def __init__(self):
        self.starts: List[int] = []
        self.ends: List[int] = []

    def free(self, a: int, b: int) -> bool:
        i = bisect.bisect_right(self.starts, a)
        if i > 0 and self.ends[i - 1] > a:
            return False
        if i < len(self.starts) and self.starts[i] < b:
            return False
        return True

    def add(self, a: int, b: int):
        i = bisect.bisect_right(self.starts, a)
        self.starts.insert(i, a)
        self.ends.insert(i, b)


def _write(ref: np.ndarray, offset: int, a: int, data) -> None:
    """ref holds bases [offset, offset + ref.size) of the whole reference:
    write `data` (a byte value or bytes) at whole-reference position a, only
    where it overlaps."""
    n = 1 if isinstance(data, int) else len(data)
    lo, hi = max(a, offset), min(a + n, offset + ref.size)
    if lo >= hi:
        return
    if isinstance(data, int):
        ref[lo - offset:hi - offset] = data
    else:
        ref[lo - offset:hi - offset] = np.frombuffer(bytes(data), dtype=np.uint8)[lo - a:hi - a]


def add_n_runs(ref: np.ndarray, frac: float, seed: int, occ: _Occupied, total: Optional[int] = None,
               offset: int = 0) -> int:
    """Overwrite runs of 'N' (length uniform in [10, 1000]) until `frac` of
    the bases are N.  Returns the number of N bases written.  With `total`,
    ref is the window [offset, offset + ref.size) of a reference of `total`
    bases: the runs are drawn for the whole and written where they overlap."""
    if frac <= 0:
        return 0
    total = ref.size if total is None else int(total)
    rng = _rng(seed, _S_NRUNS)
    target = int(frac * total)
    done = 0
    while done < target:
        L = int(rng.integers(10, 1001))
        L = min(L, target - done) if target - done >= 10 else L
        a = int(rng.integers(0, max(1, total - L)))
        if not occ.free(a, a + L):
            continue
        if offset == 0 and total == ref.size:
            ref[a:a + L] = ord("N")
        else:
            _write(ref, offset, a, b"N" * L)
        occ.add(a, a + L)
        done += L
    return done


@dataclasses.dataclass
class Plant:
    query: int
    contig: int       # contig index (0-based, dense)
    pos: int          # leftmost forward coordinate inside the contig
    strand: int       # 0 = '+', 1 = '-'
    k: int            # exact number of substitutions written


def plant_hits(ref: np.ndarray, starts: np.ndarray, lens: np.ndarray,
               queries: Sequence[bytes], ks: Sequence[int], seed: int,
               occ: _Occupied, offset: int = 0) -> List[Plant]:
    """Write one plant per entry of `ks` (its substitution count); ref holds
    the whole reference, or its window from `offset` on (plants are drawn
    for the whole and written where they overlap)."""
    rng = _rng(seed, _S_PLANTS)
    plants = []
    for k in ks:
        for _ in range(100000):
            qi = int(rng.integers(0, len(queries)))
            q = queries[qi]
            L = len(q)
            ci = int(rng.integers(0, len(lens)))
            if lens[ci] < L:
                continue
            p = int(rng.integers(0, lens[ci] - L + 1))
            t = int(rng.integers(0, 2))
            a = int(starts[ci]) + p
            if not occ.free(a, a + L):
                continue
            seq = bytearray(q)
            if t == 1:
                seq = bytearray(_PLANT_COMP[c] for c in reversed(seq))
            k_eff = min(int(k), L)
            pos = rng.choice(L, size=k_eff, replace=False)
            for j in pos:
                cur = seq[j]
                others = [c for c in b"ACGT" if c != cur]
                seq[j] = others[int(rng.integers(0, 3))]
            _write(ref, offset, a, seq)
            occ.add(a, a + L)
            plants.append(Plant(qi, ci, p, t, k_eff))
            break
        else:
            raise RuntimeError("could not place a plant")
    return plants


@dataclasses.dataclass
class Workload:
    """One synthetic problem: queries, a concatenated reference and plants."""
    name: str
    queries: List[bytes]
    ref: np.ndarray            # uint8 ASCII, all contigs concatenated
    contig_len: np.ndarray     # int64 per contig
    max_subs: List[int]
    plants: List[Plant]
    n_bases_N: int = 0
    ref_offset: int = 0        # ref holds bases [ref_offset, ref_offset + ref.size) of the whole

    @property
    def contig_start(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.contig_len)[:-1]]).astype(np.int64)

    def contig(self, i: int) -> np.ndarray:
        s = int(self.contig_start[i])
        return self.ref[s:s + int(self.contig_len[i])]


def segments(contig_len: np.ndarray, seg_bytes: int):
    """Cut the concatenated reference into segments of at most `seg_bytes`.

    Yields (begin, end, pieces) with pieces = list of
    (contig, offset_in_contig, start_in_segment, length, is_last_piece)."""
    starts = np.concatenate([[0], np.cumsum(contig_len)]).astype(np.int64)
    total = int(starts[-1])
    ci = 0
    pos = 0
    while pos < total:
        end = min(total, pos + seg_bytes)
        pieces = []
        cur = pos
        while cur < end:
            while starts[ci + 1] <= cur:
                ci += 1
            cend = int(starts[ci + 1])
            take = min(end, cend) - cur
            off = cur - int(starts[ci])
            pieces.append((ci, off, cur - pos, take, cur + take == cend))
            cur += take
        yield pos, end, pieces
        pos = end


# ---------------------------------------------------------------- presets

def small_workload(seed: int = 7, n_queries: int = 6, lmin: int = 5, lmax: int = 40,
                   n_contigs: int = 12, cmin: int = 1, cmax: int = 3000,
                   gc: float = 0.5, n_frac: float = 0.01,
                   plant_ks: Sequence[int] = (0, 1, 2, 3, 4),
                   max_subs: Sequence[int] = (0, 2, 4),
                   lowercase_frac: float = 0.0) -> Workload:
    """Small mixed case for parity tests: ragged contig lengths (some shorter
    than the queries), N-runs, lower-case bases and other IUPAC bytes."""
    rng = _rng(seed, 9)
    lens = rng.integers(cmin, cmax + 1, size=n_contigs).astype(np.int64)
    queries = random_queries(n_queries, lmin, lmax, seed)
    total = int(lens.sum())
    ref = random_bases(total, gc, seed, threads=1)
    occ = _Occupied()
    nN = 0
    if n_frac > 0:
        # short N-runs so a small reference still gets several
        nrng = _rng(seed, _S_NRUNS)
        target = int(n_frac * total)
        while nN < target:
            L = int(nrng.integers(1, 12))
            a = int(nrng.integers(0, max(1, total - L)))
            if occ.free(a, a + L):
                ref[a:a + L] = np.frombuffer(b"NRYKMSWBDHV-*."[:L] if L <= 14 else b"N" * L,
                                             dtype=np.uint8)[:L]
                occ.add(a, a + L)
                nN += L
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    plants = plant_hits(ref, starts, lens, queries, list(plant_ks), seed, occ)
    if lowercase_frac > 0:
        m = rng.random(total) < lowercase_frac
        sel = ref[m]
        isb = np.isin(sel, np.frombuffer(b"ACGT", np.uint8))
        sel[isb] = sel[isb] + 32
        ref[m] = sel
    return Workload("small", queries, ref, lens, list(max_subs), plants, nN)


def workload_1mbp_x10() -> Workload:
    """1 query of 20 bp (seed 0) against 10 contigs of 1 Mbp of uniform ACGT,
    maxSubs 2, 20 plants with 0, 1, 2 substitutions cycling."""
    queries = random_queries(1, 20, 20, 0)
    lens = np.full(10, 1_000_000, dtype=np.int64)
    ref = random_bases(int(lens.sum()), 0.5, 0)
    occ = _Occupied()
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    plants = plant_hits(ref, starts, lens, queries, [i % 3 for i in range(20)], 0, occ)
    return Workload("1q20bp_10x1Mbp_s2", queries, ref, lens, [2], plants)


def workload_4gbp(total: int = 4_000_000_000, plants_per_k: int = 1000,
                  max_subs: Sequence[int] = (0, 4, 8, 16), seed: int = 2, window=None) -> Workload:
    """10 queries of 30-40 bp against a GC-40% reference of log-normal
    contigs (1 kbp - 5 Mbp) with 0.1% N in runs of 10-1000, and
    `plants_per_k` plants for every k <= max(max_subs).  `total` can be
    lowered to build a scaled-down instance of the same recipe.  The queries
    are always drawn from seed 2; `seed` draws the reference and plants.
    `window` = (a, b): build only bases [a, b) of the reference (ref_offset
    = a), byte for byte that slice of the whole -- one rank's range of a
    reference too large for one host."""
    queries = random_queries(10, 30, 40, 2)
    lens = contig_lengths(total, 1000, 5_000_000, "lognormal", seed)
    tot = int(lens.sum())
    a, b = (0, tot) if window is None else (max(0, int(window[0])), min(tot, int(window[1])))
    ref = random_bases(tot, 0.40, seed, window=None if window is None else (a, b))
    occ = _Occupied()
    nN = add_n_runs(ref, 0.001, seed, occ, total=tot, offset=a)
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    ks = [k for k in range(max(max_subs) + 1) for _ in range(plants_per_k)]
    plants = plant_hits(ref, starts, lens, queries, ks, seed, occ, offset=a)
    wl = Workload("10q30-40bp_4Gbp", queries, ref, lens, list(max_subs), plants, nN)
    wl.ref_offset = a
    return wl


def workload_1gbp_indexed(total: int = 1_000_000_000, n_queries: int = 10_000,
                          max_subs: Sequence[int] = (4, 8, 16), planted_frac: float = 0.05,
                          plant_subs: int = 4) -> Workload:
    """Queries of 20-40 bp against a GC-50% reference of log-uniform contigs
    (10 kbp - 2 Mbp); `planted_frac` of the queries are planted once with
    exactly `plant_subs` substitutions."""
    seed = 3
    queries = random_queries(n_queries, 20, 40, seed)
    lens = contig_lengths(total, 10_000, 2_000_000, "loguniform", seed)
    tot = int(lens.sum())
    ref = random_bases(tot, 0.50, seed)
    occ = _Occupied()
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
    n_pl = int(round(planted_frac * n_queries))
    plants = _plant_queries(ref, starts, lens, queries, list(range(n_pl)),
                            plant_subs, seed, occ)
    return Workload("10kq20-40bp_1Gbp", queries, ref, lens, list(max_subs), plants)


def _plant_queries(ref, starts, lens, queries, qids, k, seed, occ) -> List[Plant]:
    """Plant each query in `qids` once with exactly k substitutions."""
    rng = _rng(seed, _S_PLANTS, 1)
    out = []
    for qi in qids:
        q = queries[qi]
        L = len(q)
        for _ in range(100000):
            ci = int(rng.integers(0, len(lens)))
            if lens[ci] < L:
                continue
            p = int(rng.integers(0, lens[ci] - L + 1))
            t = int(rng.integers(0, 2))
            a = int(starts[ci]) + p
            if not occ.free(a, a + L):
                continue
            seq = bytearray(q)
            if t == 1:
                seq = bytearray(_PLANT_COMP[c] for c in reversed(seq))
            k_eff = min(k, L)
            for j in rng.choice(L, size=k_eff, replace=False):
                others = [c for c in b"ACGT" if c != seq[j]]
                seq[j] = others[int(rng.integers(0, 3))]
            ref[a:a + L] = np.frombuffer(bytes(seq), dtype=np.uint8)
            occ.add(a, a + L)
            out.append(Plant(qi, ci, p, t, k_eff))
            break
    return out


# ------------------------------------------------- many sets / serving inputs

def per_contig_reference(lens: np.ndarray, gc_lo: float, gc_hi: float, seed: int,
                         n_frac: float = 0.0, threads: Optional[int] = None):
    """Reference whose contig i has its own GC drawn uniform in [gc_lo, gc_hi]
    (a fixed GC when gc_lo == gc_hi); each contig comes from its own
    generator, so contigs can be regenerated alone.  Returns (ref, gc)."""
    rng = _rng(seed, _S_GC)
    gc = rng.uniform(gc_lo, gc_hi, size=len(lens)) if gc_hi > gc_lo else np.full(len(lens), gc_lo)
    starts = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    ref = np.empty(int(starts[-1]), dtype=np.uint8)

    def fill(i):
        r = _rng(seed, _S_BASES, 1_000_000 + i).random(int(lens[i]), dtype=np.float32)
        g = gc[i]
        code = (r >= np.float32((1 - g) / 2)).astype(np.uint8)
        code += r >= np.float32(0.5)
        code += r >= np.float32((1 + g) / 2)
        ref[starts[i]:starts[i + 1]] = _ACGT[code]

    threads = threads or min(32, os.cpu_count() or 1)
    with _cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(fill, range(len(lens))))
    if n_frac > 0:
        add_n_runs(ref, n_frac, seed, _Occupied())
    return ref, gc


def log_uniform_int(rng, lo: int, hi: int, size: int) -> np.ndarray:
    return np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi + 1), size=size))).astype(np.int64)


def query_sets(n_sets: int, size_lo: int, size_hi: int, lmin: int, lmax: int, smax: int,
               seed: int):
    """n_sets sets of uniform-ACGT queries: sizes log-uniform in
    [size_lo, size_hi], lengths uniform in [lmin, lmax], each set's maxSubs
    uniform in {0..smax}.  Returns [(queries, max_subs)]."""
    rng = _rng(seed, _S_QUERIES, 7)
    sizes = log_uniform_int(rng, size_lo, size_hi, n_sets)
    subs = rng.integers(0, smax + 1, size=n_sets)
    out = []
    for i in range(n_sets):
        out.append((random_queries(int(sizes[i]), lmin, lmax, seed * 100_000 + i), int(subs[i])))
    return out


def workload_sets_16gbp(total: int = 16_000_000_000, n_sets: int = 256):
    """Query sets of log-uniform sizes 1-5000, lengths 18-50 bp, maxSubs
    0-12, against a reference of log-uniform contigs 1 kbp - 10 Mbp with
    per-contig GC uniform in [0.30, 0.65].  Returns (ref, lens, sets)."""
    seed = 4
    lens = contig_lengths(total, 1000, 10_000_000, "loguniform", seed)
    ref, _ = per_contig_reference(lens, 0.30, 0.65, seed)
    return ref, lens, query_sets(n_sets, 1, 5000, 18, 50, 12, seed)


def workload_serving(total: int, rate: float, duration: float, seed: int = 5):
    """Poisson arrivals (mean `rate` per second over `duration` seconds) of
    query sets of log-uniform sizes 1-2000, lengths 18-50 bp, maxSubs 0-8,
    against a reference (GC 45%, 0.05% N, log-uniform contigs 1 kbp -
    10 Mbp).  Returns (ref, lens, [(arrival_s, queries, max_subs)])."""
    lens = contig_lengths(total, 1000, 10_000_000, "loguniform", seed)
    ref, _ = per_contig_reference(lens, 0.45, 0.45, seed, n_frac=0.0005)
    return ref, lens, serving_requests(rate, duration, seed)


def serving_requests(rate: float, duration: float, seed: int = 5):
    """The serving workload's requests alone: [(arrival_s, queries, max_subs)]."""
    rng = _rng(seed, _S_QUERIES, 8)
    t = 0.0
    arrivals = []
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            break
        arrivals.append(t)
    sets = query_sets(len(arrivals), 1, 2000, 18, 50, 8, seed)
    return [(a, qs, s) for a, (qs, s) in zip(arrivals, sets)]


# ------------------------------------------- counter-based reference (any size)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _splitmix_out(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def gc_thresholds(gc: float):
    """(t1, t2, t3) of the counter-based generator for a GC fraction."""
    return (int((1.0 - gc) / 2.0 * 2 ** 32), 1 << 31, min(int((1.0 + gc) / 2.0 * 2 ** 32), 2 ** 32 - 1))


def counter_bases(first: int, n: int, seed: int, gc: float) -> np.ndarray:
    """Bases [first, first + n) of a reference whose base i is drawn from the
    high 32 bits u of splitmix64's output function at i + seed * 0x9E3779B97F4A7C15
    (A below t1, C below t2, G below t3, else T; see gc_thresholds).  Any
    slice is regenerated alone; synth/devgen.cu writes the same bytes on the
    device."""
    with np.errstate(over="ignore"):
        key = np.uint64(seed) * _GOLDEN
        i = np.arange(first, first + n, dtype=np.uint64) + key
        u = (_splitmix_out(i) >> np.uint64(32)).astype(np.uint32)
    t1, t2, t3 = gc_thresholds(gc)
    code = (u >= np.uint32(t1)).astype(np.uint8)
    code += u >= np.uint32(t2)
    code += u >= np.uint32(t3)
    return _ACGT[code]


def n_run_list(total: int, frac: float, seed: int):
    """Disjoint N-runs (lengths uniform in [10, 1000], uniform positions)
    covering `frac` of `total` bases: sorted (starts, lengths) arrays."""
    rng = _rng(seed, _S_NRUNS, 2)
    target = int(frac * total)
    starts, lens_ = [], []
    done = 0
    occ = _Occupied()
    while done < target:
        m = max(64, (target - done) // 400)
        L = rng.integers(10, 1001, size=m)
        A = rng.integers(0, max(1, total - 1000), size=m)
        for a, l in zip(A.tolist(), L.tolist()):
            if done >= target:
                break
            if occ.free(a, a + l):
                occ.add(a, a + l)
                starts.append(a)
                lens_.append(l)
                done += l
    order = np.argsort(np.asarray(starts, np.int64))
    return np.asarray(starts, np.uint64)[order], np.asarray(lens_, np.uint32)[order]


@dataclasses.dataclass
class CounterReference:
    """A reference defined by counters rather than stored: contig lengths,
    the GC fraction, the base seed and the N-runs; bases(a, b) gives any
    slice (host), and synth.devgen fills a device buffer with the same
    bytes."""
    contig_len: np.ndarray
    gc: object                 # a float, or one GC fraction per contig
    seed: int
    run_start: np.ndarray
    run_len: np.ndarray

    @property
    def total(self) -> int:
        return int(self.contig_len.sum())

    @property
    def contig_start(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.contig_len)[:-1]]).astype(np.int64)

    def gc_spans(self, a: int, b: int):
        """[(lo, hi, gc)] covering [a, b): one span, or one per contig."""
        if np.isscalar(self.gc):
            return [(a, b, float(self.gc))]
        st = self.contig_start
        i = int(np.searchsorted(st, a, side="right")) - 1
        out = []
        while a < b:
            end = min(b, int(st[i] + self.contig_len[i]))
            out.append((a, end, float(self.gc[i])))
            a = end
            i += 1
        return out

    def bases(self, a: int, b: int) -> np.ndarray:
        out = np.concatenate([counter_bases(lo, hi - lo, self.seed, g) for lo, hi, g in self.gc_spans(a, b)])
        i0 = int(np.searchsorted(self.run_start, a, side="left"))
        i0 = max(0, i0 - 1)
        for s_, l_ in zip(self.run_start[i0:].tolist(), self.run_len[i0:].tolist()):
            if s_ >= b:
                break
            lo, hi = max(a, s_), min(b, s_ + l_)
            if lo < hi:
                out[lo - a:hi - a] = ord("N")
        return out


def sets_reference(total: int = 16_000_000_000, seed: int = 4) -> CounterReference:
    """The batched workload's reference recipe, counter-based: log-uniform
    contigs of 1 kbp - 10 Mbp, each with its own GC drawn uniform in
    [0.30, 0.65], no N."""
    lens = contig_lengths(total, 1000, 10_000_000, "loguniform", seed)
    gc = _rng(seed, _S_GC, 2).uniform(0.30, 0.65, size=len(lens))
    return CounterReference(lens, gc, seed, np.zeros(0, np.uint64), np.zeros(0, np.uint32))


def serving_reference(total: int = 200_000_000_000, seed: int = 5) -> CounterReference:
    """The serving workload's reference at any size: log-uniform contigs of
    1 kbp - 10 Mbp, GC 45%, 0.05% N in runs of 10-1000 -- counter-based so
    that 200 Gbp is built on the device and any slice regenerated on the
    host."""
    lens = contig_lengths(total, 1000, 10_000_000, "loguniform", seed)
    rs, rl = n_run_list(int(lens.sum()), 0.0005, seed)
    return CounterReference(lens, 0.45, seed, rs, rl)
