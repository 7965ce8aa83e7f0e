"""CPU oracle for the indel-free scan -- TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the benchmark's timed CPU
baseline may import this package.  The product path never does.

The arithmetic lives in plain C (`ifa_oracle.c`, built with gcc by
`build.py`); this wrapper only marshals numpy arrays and splits the
contigs across host threads (results do not depend on the thread count).
Each C function cites the passage of the paper it follows.
"""
from __future__ import annotations

import concurrent.futures as _cf
import ctypes as C
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from .build import build as _build, LIB_PATH

HIT_DTYPE = np.dtype([("query", "<u4"), ("contig", "<u4"), ("pos", "<u4"),
                      ("strand", "u1"), ("mismatches", "u1"), ("clips", "<u2")])

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            _build()
        L = C.CDLL(LIB_PATH)
        u8p = C.POINTER(C.c_uint8)
        u32p = C.POINTER(C.c_uint32)
        u64p = C.POINTER(C.c_uint64)
        L.oracle_brute.restype = C.c_int64
        L.oracle_brute.argtypes = [u8p, u64p, u32p, C.c_uint32, u8p, u64p, u64p, u32p,
                                   C.c_uint32, C.c_uint32, C.c_uint32, C.c_void_p, C.c_int64]
        L.oracle_indexed.restype = C.c_int64
        L.oracle_indexed.argtypes = [u8p, u64p, u32p, C.c_uint32, u8p, u64p, u64p, u32p,
                                     C.c_uint32, C.c_uint32, u32p, u32p, u8p, C.c_uint32,
                                     C.c_uint32, C.c_uint32, C.c_void_p, C.c_int64]
        L.oracle_minhits.restype = C.c_uint32
        L.oracle_minhits.argtypes = [C.c_uint32] * 9 + [C.c_uint64, u64p]
        L.oracle_choose_k.restype = C.c_int
        L.oracle_choose_k.argtypes = [C.c_uint32, C.c_uint32, u32p, C.c_uint32, C.c_uint32,
                                      C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_uint32, C.c_uint64, u32p, u32p]
        L.oracle_philox4x32_10.restype = None
        L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.oracle_digest.restype = None
        L.oracle_digest.argtypes = [C.c_void_p, C.c_int64, u64p]
        L.oracle_window_mismatches.restype = C.c_uint32
        L.oracle_window_mismatches.argtypes = [u8p, C.c_uint32, C.c_uint8, u8p, C.c_uint64]
        L.oracle_window_seeds.restype = C.c_uint32
        L.oracle_window_seeds.argtypes = [u8p, C.c_uint32, C.c_uint8, u8p, C.c_uint64,
                                          C.c_uint32, C.c_uint32, C.c_uint32]
        L.oracle_revcomp.restype = None
        L.oracle_revcomp.argtypes = [u8p, C.c_uint32, u8p]
        L.oracle_minhits_quantile.restype = C.c_uint32
        L.oracle_minhits_quantile.argtypes = [u64p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64]
        L.oracle_kmer_count.restype = C.c_uint32
        L.oracle_kmer_count.argtypes = [C.c_uint32] * 3
        _lib = L
    return _lib


class use_library:
    """Context manager: route every oracle call to another build of the same
    C source (the pin tests use it to check that planted mistakes fail)."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib, LIB_PATH
        self.saved, self._orig = _lib, LIB_PATH
        _lib, LIB_PATH = None, self.path
        lib()
        return self

    def __exit__(self, *a):
        global _lib, LIB_PATH
        _lib, LIB_PATH = self.saved, self._orig


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _pack_queries(queries: Sequence[bytes]):
    qlen = np.array([len(q) for q in queries], dtype=np.uint32)
    qoff = np.concatenate([[0], np.cumsum(qlen, dtype=np.uint64)[:-1]]).astype(np.uint64)
    qcat = np.frombuffer(b"".join(queries) or b"\0", dtype=np.uint8).copy()
    return qcat, qoff, qlen


def sort_hits(h: np.ndarray) -> np.ndarray:
    """Sort by (query, contig, pos, strand, mismatches, clips)."""
    if h.size == 0:
        return h
    order = np.lexsort((h["clips"], h["mismatches"], h["strand"], h["pos"], h["contig"], h["query"]))
    return h[order]


def _run_chunks(fn, ref, contig_len, contig_ids, threads):
    contig_len = np.asarray(contig_len, dtype=np.uint64)
    nc = contig_len.size
    roff = np.concatenate([[0], np.cumsum(contig_len)[:-1]]).astype(np.uint64)
    rid = (np.arange(nc, dtype=np.uint32) if contig_ids is None
           else np.asarray(contig_ids, dtype=np.uint32))
    ref = np.ascontiguousarray(ref, dtype=np.uint8)
    if nc == 0:
        return np.zeros(0, HIT_DTYPE)
    threads = max(1, min(threads, nc))
    # contiguous contig ranges of about equal base count
    csum = np.cumsum(contig_len.astype(np.float64))
    bounds = [0] + [int(np.searchsorted(csum, csum[-1] * i / threads)) + 1
                    for i in range(1, threads)] + [nc]
    bounds = sorted(set(min(nc, b) for b in bounds))

    def work(a, b):
        if a >= b:
            return np.zeros(0, HIT_DTYPE)
        sl_off = roff[a:b].copy()
        sl_len = contig_len[a:b].copy()
        sl_id = rid[a:b].copy()
        cap = 1024
        while True:
            out = np.zeros(cap, HIT_DTYPE)
            n = fn(ref, sl_off, sl_len, sl_id, b - a, out, cap)
            if n <= cap:
                return out[:n]
            cap = int(n)

    if len(bounds) <= 2:
        parts = [work(bounds[0], bounds[-1])]
    else:
        with _cf.ThreadPoolExecutor(len(bounds) - 1) as ex:
            parts = list(ex.map(lambda ab: work(*ab), zip(bounds[:-1], bounds[1:])))
    return sort_hits(np.concatenate(parts))


def brute(queries: Sequence[bytes], ref: np.ndarray, contig_len, max_subs: int,
          contig_ids=None, threads: int = 1, clip_pct: int = 0) -> np.ndarray:
    """All (query, contig, pos, strand, mismatches) with Hamming <= max_subs;
    with clip_pct > 0 also the windows overhanging a contig end by up to
    floor(clip_pct * L / 100) bases (clips = left | right << 8)."""
    qcat, qoff, qlen = _pack_queries(queries)
    L = lib()

    def fn(ref_, off, ln, ids, nc, out, cap):
        return L.oracle_brute(_ptr(qcat, C.c_uint8), _ptr(qoff, C.c_uint64), _ptr(qlen, C.c_uint32),
                              len(queries), _ptr(ref_, C.c_uint8), _ptr(off, C.c_uint64),
                              _ptr(ln, C.c_uint64), _ptr(ids, C.c_uint32), nc, int(max_subs),
                              int(clip_pct), out.ctypes.data, cap)
    return _run_chunks(fn, ref, contig_len, contig_ids, threads)


def indexed(queries: Sequence[bytes], ref: np.ndarray, contig_len, max_subs: int,
            k_per_query, minhits_per_query, exhaustive_per_query, step: int = 1,
            mask_w: int = 0, contig_ids=None, threads: int = 1, clip_pct: int = 0) -> np.ndarray:
    """Brute hits whose seed count reaches the per-query threshold (clipped
    windows, clip_pct > 0, are kept exhaustively)."""
    qcat, qoff, qlen = _pack_queries(queries)
    kq = np.ascontiguousarray(k_per_query, dtype=np.uint32)
    mh = np.ascontiguousarray(minhits_per_query, dtype=np.uint32)
    ex = np.ascontiguousarray(exhaustive_per_query, dtype=np.uint8)
    L = lib()

    def fn(ref_, off, ln, ids, nc, out, cap):
        return L.oracle_indexed(_ptr(qcat, C.c_uint8), _ptr(qoff, C.c_uint64), _ptr(qlen, C.c_uint32),
                                len(queries), _ptr(ref_, C.c_uint8), _ptr(off, C.c_uint64),
                                _ptr(ln, C.c_uint64), _ptr(ids, C.c_uint32), nc, int(max_subs),
                                _ptr(kq, C.c_uint32), _ptr(mh, C.c_uint32), _ptr(ex, C.c_uint8),
                                int(step), int(mask_w), int(clip_pct), out.ctypes.data, cap)
    return _run_chunks(fn, ref, contig_len, contig_ids, threads)


def minhits(L: int, subs: int, k: int, step: int = 1, mask_w: int = 0, max_clips: int = 0,
            num: int = 999, den: int = 1000, trials: int = 100_000, seed: int = 1,
            with_hist: bool = False):
    K = int(lib().oracle_kmer_count(L, k, step))
    hist = np.zeros(K + 1, dtype=np.uint64)
    m = lib().oracle_minhits(L, subs, k, step, mask_w, max_clips, num, den, trials, seed,
                             _ptr(hist, C.c_uint64))
    return (int(m), hist) if with_hist else int(m)


def choose_k(L: int, subs: int, klist=(8, 9, 10, 12, 14), step: int = 1, mask_w: int = 0,
             max_clips: int = 0, num: int = 999, den: int = 1000, trials: int = 100_000,
             seed: int = 1) -> Tuple[int, int, int]:
    """(status, k, minhits); status 1 = qualified, 0 = clamped, -1 = none."""
    kl = np.asarray(klist, dtype=np.uint32)
    ko = np.zeros(1, np.uint32)
    mo = np.zeros(1, np.uint32)
    st = lib().oracle_choose_k(L, subs, _ptr(kl, C.c_uint32), kl.size, step, mask_w, max_clips,
                               num, den, trials, seed, _ptr(ko, C.c_uint32), _ptr(mo, C.c_uint32))
    return int(st), int(ko[0]), int(mo[0])


def minhits_quantile(hist, num: int, den: int) -> int:
    h = np.ascontiguousarray(hist, dtype=np.uint64)
    return int(lib().oracle_minhits_quantile(_ptr(h, C.c_uint64), h.size - 1, num, den,
                                             int(h.sum())))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(o, C.c_uint32))
    return o


def digest(hits: np.ndarray) -> Tuple[int, int, int]:
    h = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
    o = np.zeros(3, np.uint64)
    lib().oracle_digest(h.ctypes.data if h.size else None, h.size, _ptr(o, C.c_uint64))
    return int(o[0]), int(o[1]), int(o[2])


def window_mismatches(query: bytes, strand: int, contig: np.ndarray, pos: int) -> int:
    q = np.frombuffer(query, dtype=np.uint8).copy()
    c = np.ascontiguousarray(contig, dtype=np.uint8)
    return int(lib().oracle_window_mismatches(_ptr(q, C.c_uint8), len(query), strand,
                                               _ptr(c, C.c_uint8), pos))


def window_seeds(query: bytes, strand: int, contig: np.ndarray, pos: int, k: int,
                 step: int = 1, mask_w: int = 0) -> int:
    q = np.frombuffer(query, dtype=np.uint8).copy()
    c = np.ascontiguousarray(contig, dtype=np.uint8)
    return int(lib().oracle_window_seeds(_ptr(q, C.c_uint8), len(query), strand,
                                          _ptr(c, C.c_uint8), pos, k, step, mask_w))


def revcomp(query: bytes) -> bytes:
    q = np.frombuffer(query, dtype=np.uint8).copy()
    o = np.zeros(len(query), np.uint8)
    lib().oracle_revcomp(_ptr(q, C.c_uint8), len(query), _ptr(o, C.c_uint8))
    return o.tobytes()


def kmer_count(L: int, k: int, step: int = 1) -> int:
    return int(lib().oracle_kmer_count(L, k, step))
