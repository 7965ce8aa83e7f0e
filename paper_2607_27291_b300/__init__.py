"""B300-native indel-free (Hamming) aligner: thin ctypes binding over libifa.so.

The functions below carry the names of the C ABI in ``include/ifa.h`` and
only marshal arguments; every step of the scan runs in the library's CUDA
kernels.  Importing this package does not need a GPU; calling into the
library does, and a missing library raises at once (there is no CPU
fallback).  PyTorch is optional: it may supply device buffers and streams.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# IFA_LIB selects another build of the library (tuning experiments)
LIB_PATH = os.environ.get("IFA_LIB") or os.path.join(_HERE, "libifa.so")

IFA_OK = 0
IFA_ERR_INVALID_ARG = 1
IFA_ERR_OOM = 2
IFA_ERR_CUDA = 3
IFA_ERR_BAD_STATE = 4
IFA_ERR_HIT_OVERFLOW = 5
IFA_ERR_TIMEOUT = 6

IFA_MODE_AUTO, IFA_MODE_BRUTE, IFA_MODE_INDEXED = 0, 1, 2
IFA_MEM_HOST, IFA_MEM_HOST_PINNED, IFA_MEM_DEVICE, IFA_MEM_HOST_PINNED_ASYNC = 0, 1, 2, 3
IFA_BRUTE_AUTO, IFA_BRUTE_POPC, IFA_BRUTE_TENSOR = 0, 1, 2
IFA_MAX_QUERY_LEN = 255

HIT_DTYPE = np.dtype([("query", "<u4"), ("contig", "<u4"), ("pos", "<u4"),
                      ("strand", "u1"), ("mismatches", "u1"), ("clips", "<u2")])
PIECE_DTYPE = np.dtype([("contig", "<u4"), ("last", "<u4"), ("offset_in_contig", "<u8"),
                        ("start", "<u8"), ("len", "<u8")])


class ifa_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("count_only", C.c_uint32), ("hit_capacity", C.c_uint64),
                ("segment_bytes", C.c_uint64), ("k_list", C.c_uint32 * 8), ("n_k", C.c_uint32),
                ("kmer_step", C.c_uint32), ("mask_width", C.c_uint32), ("minhits_num", C.c_uint32),
                ("minhits_den", C.c_uint32), ("minhits_trials", C.c_uint32),
                ("minhits_seed", C.c_uint64), ("clip_pct", C.c_uint32),
                ("exhaustive_fallback", C.c_uint32), ("auto_crossover", C.c_uint32),
                ("profile", C.c_uint32), ("brute_kernel", C.c_uint32), ("test_stall", C.c_uint32),
                ("event_capacity", C.c_uint32), ("reserved", C.c_uint32 * 3)]


class ifa_digest(C.Structure):
    _fields_ = [("count", C.c_uint64), ("sum", C.c_uint64), ("xr", C.c_uint64)]


class ifa_stats(C.Structure):
    _fields_ = [("segments", C.c_uint64), ("bases", C.c_uint64), ("h2d_bytes", C.c_uint64),
                ("windows", C.c_uint64), ("query_bases", C.c_uint64),
                ("kernel_launches", C.c_uint64), ("candidates", C.c_uint64),
                ("scan_launches", C.c_uint64), ("scan_ns", C.c_uint64),
                ("mode", C.c_uint32), ("reserved", C.c_uint32)]


class ifa_sam_info(C.Structure):
    _fields_ = [("query_seqs", C.POINTER(C.c_void_p)), ("query_lens", C.POINTER(C.c_uint32)),
                ("query_names", C.POINTER(C.c_char_p)), ("n_queries", C.c_uint32),
                ("contig_names", C.POINTER(C.c_char_p)), ("n_contig_names", C.c_uint32)]


class IfaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("ifa status %d: %s" % (status, msg))
        self.status = status


_lib = None
_SYMBOLS = {
    "ifa_config_default": (C.c_int, [C.POINTER(ifa_config)]),
    "ifa_create": (C.c_int, [C.POINTER(ifa_config), C.POINTER(C.c_void_p)]),
    "ifa_destroy": (None, [C.c_void_p]),
    "ifa_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ifa_load_queries": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_uint32),
                                   C.c_uint32, C.POINTER(C.c_uint32)]),
    "ifa_set_max_subs": (C.c_int, [C.c_void_p, C.c_uint32]),
    "ifa_set_query_max_subs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32]),
    "ifa_set_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "ifa_push_segment": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint32,
                                   C.c_int]),
    "ifa_prime_halo": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint64, C.c_void_p, C.c_uint64, C.c_int]),
    "ifa_flush": (C.c_int, [C.c_void_p]),
    "ifa_drain_hits": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.POINTER(C.c_uint64),
                                 C.POINTER(C.c_int)]),
    "ifa_poll_hits": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.POINTER(C.c_uint64),
                                C.POINTER(C.c_int)]),
    "ifa_get_digest": (C.c_int, [C.c_void_p, C.POINTER(ifa_digest), C.c_void_p]),
    "ifa_reset_results": (C.c_int, [C.c_void_p]),
    "ifa_get_stats": (C.c_int, [C.c_void_p, C.POINTER(ifa_stats)]),
    "ifa_get_query_plan": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ifa_minhits": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint32,
                              C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                              C.c_uint32, C.c_uint64, C.c_void_p]),
    "ifa_last_error": (C.c_char_p, [C.c_void_p]),
    "ifa_ref_append": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint32, C.c_int]),
    "ifa_ref_reserve": (C.c_int, [C.c_void_p, C.c_uint64]),
    "ifa_ref_reset": (C.c_int, [C.c_void_p]),
    "ifa_set_add": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_uint32), C.c_uint32,
                              C.c_uint32, C.c_int, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "ifa_batch_run": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "ifa_serve_start": (C.c_int, [C.c_void_p, C.c_uint32, C.c_uint64, C.c_uint64]),
    "ifa_serve_submit": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_uint32), C.c_uint32,
                                   C.c_uint32, C.c_int, C.POINTER(C.c_uint32)]),
    "ifa_serve_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "ifa_serve_poll": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p]),
    "ifa_serve_drain": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_uint64, C.POINTER(C.c_uint64)]),
    "ifa_serve_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "ifa_serve_stop": (C.c_int, [C.c_void_p]),
    "ifa_serve_cancel": (C.c_int, [C.c_void_p, C.c_uint32]),
    "ifa_bounds_check": (C.c_int, [C.c_int, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32), C.c_int]),
    "ifa_scan_brute_noalloc": (C.c_int, [C.c_int32, C.POINTER(C.c_void_p), C.POINTER(C.c_uint32),
                                         C.c_uint32, C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint32,
                                         C.c_uint32, C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p,
                                         C.c_void_p]),
    "ifa_sam_records": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(ifa_sam_info), C.c_void_p,
                                  C.c_void_p, C.c_uint64, C.POINTER(C.c_uint64)]),
    "ifa_sam_header": (C.c_int, [C.POINTER(C.c_char_p), C.c_void_p, C.c_void_p, C.c_uint32,
                                 C.c_void_p, C.c_uint64, C.POINTER(C.c_uint64)]),
}


def lib():
    """The loaded libifa.so (raises if it was never built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libifa.so is not built; run `python -m paper_2607_27291_b300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SYMBOLS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> List[str]:
    return list(_SYMBOLS)


def _check(st: int, h=None, allow=(IFA_OK,)):
    if st not in allow:
        raise IfaError(st, lib().ifa_last_error(h).decode(errors="replace"))
    return st


# ------------------------------------------------------------ C ABI by name

def ifa_config_default() -> ifa_config:
    cfg = ifa_config()
    _check(lib().ifa_config_default(C.byref(cfg)))
    return cfg


def ifa_create(cfg: Optional[ifa_config] = None, **overrides) -> C.c_void_p:
    cfg = cfg or ifa_config_default()
    for k, v in overrides.items():
        if k == "k_list":
            for i, x in enumerate(v):
                cfg.k_list[i] = x
            cfg.n_k = len(v)
        else:
            setattr(cfg, k, v)
    h = C.c_void_p()
    _check(lib().ifa_create(C.byref(cfg), C.byref(h)))
    return h


def ifa_destroy(h) -> None:
    if h is not None and h.value is not None:
        _PINNED.pop(h.value, None)
    lib().ifa_destroy(h)


def ifa_set_stream(h, stream) -> None:
    """`stream`: a torch.cuda.Stream, a raw cudaStream_t as int, or None."""
    ptr = getattr(stream, "cuda_stream", stream)
    _check(lib().ifa_set_stream(h, C.c_void_p(ptr or None)), h)


def ifa_load_queries(h, queries: Sequence[bytes]) -> int:
    n = len(queries)
    bufs = [C.create_string_buffer(bytes(q), len(q)) for q in queries]
    ptrs = (C.c_void_p * max(1, n))(*[C.cast(b, C.c_void_p) for b in bufs])
    lens = (C.c_uint32 * max(1, n))(*[len(q) for q in queries])
    first = C.c_uint32()
    _check(lib().ifa_load_queries(h, ptrs, lens, n, C.byref(first)), h)
    return first.value


def ifa_set_max_subs(h, s: int) -> None:
    _check(lib().ifa_set_max_subs(h, int(s)), h)


def ifa_set_query_max_subs(h, max_subs: Optional[Sequence[int]]) -> None:
    """Each loaded query's own maxSubs (None: back to the single value)."""
    if max_subs is None:
        _check(lib().ifa_set_query_max_subs(h, None, 0), h)
        return
    a = np.ascontiguousarray(np.asarray(max_subs, dtype=np.uint32))
    _check(lib().ifa_set_query_max_subs(h, a.ctypes.data if a.size else None, a.size), h)


def ifa_set_mode(h, mode: int) -> None:
    _check(lib().ifa_set_mode(h, int(mode)), h)


def _as_pieces(pieces) -> np.ndarray:
    if isinstance(pieces, np.ndarray) and pieces.dtype == PIECE_DTYPE:
        return np.ascontiguousarray(pieces)
    arr = np.zeros(len(pieces), PIECE_DTYPE)
    for i, (contig, off, start, ln, last) in enumerate(pieces):
        arr[i] = (contig, 1 if last else 0, off, start, ln)
    return arr


def _buffer(data, mem: Optional[int]):
    """(pointer, length, memory kind) of a numpy uint8 array (pageable host),
    a torch uint8 tensor (CUDA, or pinned CPU) or a (pointer, length, mem)
    tuple."""
    if isinstance(data, tuple):
        return data
    if isinstance(data, np.ndarray):
        assert data.dtype == np.uint8 and data.flags.c_contiguous
        return data.ctypes.data, data.size, IFA_MEM_HOST if mem is None else mem
    assert data.is_contiguous()  # torch tensor
    if mem is None:
        mem = IFA_MEM_DEVICE if data.is_cuda else (IFA_MEM_HOST_PINNED if data.is_pinned() else IFA_MEM_HOST)
    return data.data_ptr(), data.numel(), mem


def ifa_push_segment(h, data, pieces, mem: Optional[int] = None) -> None:
    """Push one segment.  `data`: a numpy uint8 array (pageable host), a torch
    uint8 tensor (CUDA, or pinned CPU), or a (pointer, length, mem) tuple.
    `pieces`: PIECE_DTYPE array or (contig, offset_in_contig, start, len,
    last) tuples."""
    pa = _as_pieces(pieces)
    ptr, ln, mem = _buffer(data, mem)
    _check(lib().ifa_push_segment(h, C.c_void_p(ptr), ln, pa.ctypes.data, pa.size, mem), h)


def ifa_prime_halo(h, contig: int, offset_in_contig: int, data, mem: Optional[int] = None) -> None:
    """Start the stream inside contig `contig`: `data` holds its bases from
    offset_in_contig up to where the next pushed segment begins."""
    ptr, ln, mem = _buffer(data, mem)
    _check(lib().ifa_prime_halo(h, int(contig), int(offset_in_contig), C.c_void_p(ptr), ln, mem), h)


def ifa_flush(h) -> int:
    """Returns IFA_OK or IFA_ERR_HIT_OVERFLOW; raises on other errors."""
    return _check(lib().ifa_flush(h), h, allow=(IFA_OK, IFA_ERR_HIT_OVERFLOW))


_PINNED = {}


def _pinned_hits(h, n: int):
    """A page-locked hit array of at least n entries kept per handle (the
    device-to-host copy of hits runs at full PCIe speed only into pinned
    memory).  None when torch is unavailable."""
    try:
        import torch
    except ImportError:
        return None
    key = h.value
    buf = _PINNED.get(key)
    if buf is None or buf[1].size < n:
        t = torch.empty(max(n, 1) * HIT_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        buf = (t, t.numpy().view(HIT_DTYPE))
        _PINNED[key] = buf
    return buf[1]


def ifa_drain_hits(h, cap: Optional[int] = None, copy: bool = True) -> Tuple[np.ndarray, bool]:
    """Drain buffered hits; returns (hits, overflowed).  The hits are copied
    from the device into a page-locked buffer owned by the handle; with
    copy=False the returned array is a view of that buffer, valid until the
    next drain on the handle."""
    d = ifa_digest()
    st = lib().ifa_get_digest(h, C.byref(d), None)
    _check(st, h)
    want = int(d.count) if cap is None else int(cap)
    pinned = _pinned_hits(h, want) if want else None
    parts = []
    overflowed = False
    while True:
        if pinned is not None and want:
            out, chunk = pinned, pinned.size
        else:
            chunk = cap or (1 << 22)
            out = np.zeros(chunk, HIT_DTYPE)
        n = C.c_uint64()
        more = C.c_int()
        st = _check(lib().ifa_drain_hits(h, out.ctypes.data, chunk, C.byref(n), C.byref(more)), h,
                    allow=(IFA_OK, IFA_ERR_HIT_OVERFLOW))
        overflowed |= st == IFA_ERR_HIT_OVERFLOW
        got = out[:n.value]
        parts.append(got.copy() if (copy or more.value) and out is pinned else got)
        if cap is not None or not more.value:
            break
    if len(parts) == 1:
        return parts[0], overflowed
    return (np.concatenate(parts) if parts else np.zeros(0, HIT_DTYPE)), overflowed


def ifa_poll_hits(h, out: np.ndarray) -> Tuple[int, bool, bool]:
    """Copy the hits of already finished segments into `out` (a HIT_DTYPE
    array; pinned memory copies fastest) without waiting for the device;
    returns (hits copied, overflowed, more finished hits waiting)."""
    assert out.dtype == HIT_DTYPE and out.flags.c_contiguous
    n = C.c_uint64()
    more = C.c_int()
    st = _check(lib().ifa_poll_hits(h, out.ctypes.data, out.size, C.byref(n), C.byref(more)), h,
                allow=(IFA_OK, IFA_ERR_HIT_OVERFLOW))
    return n.value, st == IFA_ERR_HIT_OVERFLOW, bool(more.value)


def ifa_drain_into(h, out: np.ndarray) -> Tuple[int, bool, bool]:
    """ifa_drain_hits into the caller's HIT_DTYPE array `out` (waits for the
    device); returns (hits copied, overflowed, more hits waiting)."""
    assert out.dtype == HIT_DTYPE and out.flags.c_contiguous
    n = C.c_uint64()
    more = C.c_int()
    st = _check(lib().ifa_drain_hits(h, out.ctypes.data, out.size, C.byref(n), C.byref(more)), h,
                allow=(IFA_OK, IFA_ERR_HIT_OVERFLOW))
    return n.value, st == IFA_ERR_HIT_OVERFLOW, bool(more.value)


def ifa_get_digest(h, nq: Optional[int] = None):
    d = ifa_digest()
    counts = np.zeros(max(1, nq or 0), np.uint64)
    _check(lib().ifa_get_digest(h, C.byref(d), counts.ctypes.data if nq else None), h)
    return (int(d.count), int(d.sum), int(d.xr)), (counts[:nq] if nq else None)


def ifa_reset_results(h) -> None:
    _check(lib().ifa_reset_results(h), h)


def ifa_get_stats(h) -> dict:
    s = ifa_stats()
    _check(lib().ifa_get_stats(h, C.byref(s)), h)
    return {f: int(getattr(s, f)) for f, _ in ifa_stats._fields_}


def ifa_get_query_plan(h, nq: int):
    k = np.zeros(nq, np.uint32)
    m = np.zeros(nq, np.uint32)
    ex = np.zeros(nq, np.uint8)
    _check(lib().ifa_get_query_plan(h, k.ctypes.data, m.ctypes.data, ex.ctypes.data), h)
    return k, m, ex


def ifa_minhits(device: int, L, subs, k, step: int = 1, mask_width: int = 0, max_clips: int = 0,
                num: int = 999, den: int = 1000, trials: int = 200_000, seed: int = 1) -> np.ndarray:
    L = np.ascontiguousarray(L, np.uint32)
    subs = np.ascontiguousarray(subs, np.uint32)
    k = np.ascontiguousarray(k, np.uint32)
    out = np.zeros(L.size, np.uint32)
    _check(lib().ifa_minhits(device, L.ctypes.data, subs.ctypes.data, k.ctypes.data, L.size, step,
                             mask_width, max_clips, num, den, trials, seed, out.ctypes.data))
    return out


IFA_BATCH_PERSISTENT, IFA_BATCH_PER_SET = 0, 1
SET_RESULT_DTYPE = np.dtype([("mode", "<u4"), ("queries", "<u4"), ("hits", "<u8"),
                             ("done_ms", "<f4"), ("pad", "<f4")])


def ifa_ref_append(h, data, pieces, mem: Optional[int] = None) -> None:
    """Append to the device-resident reference store (same data/pieces forms
    as ifa_push_segment)."""
    pa = _as_pieces(pieces)
    if isinstance(data, tuple):
        ptr, ln, mem = data
    elif isinstance(data, np.ndarray):
        ptr, ln = data.ctypes.data, data.size
        mem = IFA_MEM_HOST if mem is None else mem
    else:
        ptr, ln = data.data_ptr(), data.numel()
        if mem is None:
            mem = IFA_MEM_DEVICE if data.is_cuda else (
                IFA_MEM_HOST_PINNED if data.is_pinned() else IFA_MEM_HOST)
    _check(lib().ifa_ref_append(h, C.c_void_p(ptr), ln, pa.ctypes.data, pa.size, mem), h)


def ifa_ref_reserve(h, bases: int) -> None:
    _check(lib().ifa_ref_reserve(h, int(bases)), h)


def ifa_ref_reset(h) -> None:
    _check(lib().ifa_ref_reset(h), h)


def ifa_set_add(h, queries: Sequence[bytes], max_subs: int, mode: int = IFA_MODE_AUTO) -> Tuple[int, int]:
    """Register a query set; returns (set_id, first_query)."""
    n = len(queries)
    bufs = [C.create_string_buffer(bytes(q), len(q)) for q in queries]
    ptrs = (C.c_void_p * max(1, n))(*[C.cast(b, C.c_void_p) for b in bufs])
    lens = (C.c_uint32 * max(1, n))(*[len(q) for q in queries])
    sid = C.c_uint32()
    first = C.c_uint32()
    _check(lib().ifa_set_add(h, ptrs, lens, n, int(max_subs), int(mode), C.byref(sid), C.byref(first)), h)
    return sid.value, first.value


def ifa_batch_run(h, kind: int, n_sets: int) -> np.ndarray:
    """Scan all sets against the store; returns one SET_RESULT_DTYPE row per set."""
    out = np.zeros(max(1, n_sets), SET_RESULT_DTYPE)
    _check(lib().ifa_batch_run(h, int(kind), out.ctypes.data), h)
    return out[:n_sets]


class ifa_request_info(C.Structure):
    _fields_ = [("state", C.c_uint32), ("mode", C.c_uint32), ("queries", C.c_uint32),
                ("slices_done", C.c_uint32), ("hits", C.c_uint64), ("overflowed", C.c_uint64),
                ("submit_s", C.c_double), ("admit_s", C.c_double), ("done_s", C.c_double),
                ("digest", ifa_digest)]


def ifa_serve_start(h, n_slices: int, hbm_budget_bytes: int, ring_hits: int) -> None:
    _check(lib().ifa_serve_start(h, n_slices, hbm_budget_bytes, ring_hits), h)


def ifa_serve_submit(h, queries: Sequence[bytes], max_subs: int, mode: int = IFA_MODE_AUTO) -> int:
    n = len(queries)
    bufs = [C.create_string_buffer(bytes(q), len(q)) for q in queries]
    ptrs = (C.c_void_p * max(1, n))(*[C.cast(b, C.c_void_p) for b in bufs])
    lens = (C.c_uint32 * max(1, n))(*[len(q) for q in queries])
    rid = C.c_uint32()
    _check(lib().ifa_serve_submit(h, ptrs, lens, n, int(max_subs), int(mode), C.byref(rid)), h)
    return rid.value


def ifa_serve_step(h) -> Tuple[int, int]:
    a = C.c_uint32()
    d = C.c_uint32()
    _check(lib().ifa_serve_step(h, C.byref(a), C.byref(d)), h)
    return a.value, d.value


def ifa_serve_poll(h, rid: int) -> dict:
    info = ifa_request_info()
    _check(lib().ifa_serve_poll(h, rid, C.byref(info)), h)
    out = {f: getattr(info, f) for f, _ in ifa_request_info._fields_ if f != "digest"}
    out["digest"] = (int(info.digest.count), int(info.digest.sum), int(info.digest.xr))
    return out


def ifa_serve_drain(h, rid: int, cap: int) -> Tuple[np.ndarray, bool]:
    out = np.zeros(max(1, cap), HIT_DTYPE)
    n = C.c_uint64()
    st = _check(lib().ifa_serve_drain(h, rid, out.ctypes.data, cap, C.byref(n)), h,
                allow=(IFA_OK, IFA_ERR_HIT_OVERFLOW))
    return out[:n.value], st == IFA_ERR_HIT_OVERFLOW


def ifa_serve_stats(h) -> dict:
    n = C.c_uint64()
    qb = C.c_double()
    ps = C.c_double()
    ss = C.c_double()
    _check(lib().ifa_serve_stats(h, C.byref(n), C.byref(qb), C.byref(ps), C.byref(ss)), h)
    return {"slices": n.value, "query_bases": qb.value, "plan_s": ps.value, "scan_s": ss.value}


def ifa_bounds_check(device: int = 0, reset: bool = False) -> Tuple[bool, int]:
    """(built with bounds checks, first out-of-range read as kind << 56 |
    index or 0)."""
    first = C.c_uint64()
    enabled = C.c_uint32()
    _check(lib().ifa_bounds_check(int(device), C.byref(first), C.byref(enabled), 1 if reset else 0))
    return bool(enabled.value), int(first.value)


def ifa_serve_cancel(h, rid: int) -> None:
    _check(lib().ifa_serve_cancel(h, rid), h)


def ifa_serve_stop(h) -> None:
    _check(lib().ifa_serve_stop(h), h)


def ifa_scan_brute_noalloc(device: int, queries: Sequence[bytes], ref_ptr: int, length: int,
                           pieces, max_subs: int, hits_ptr: int, hit_capacity: int,
                           counters_ptr: int, per_query_counts_ptr: int = 0, stream=None) -> None:
    """Allocation-free brute-force scan of one chunk of whole contigs; every
    buffer is the caller's (device pointers as ints).  With no queries the
    call only places the library's scratch array on `device` (set-up)."""
    n = len(queries)
    bufs = [C.create_string_buffer(bytes(q), len(q)) for q in queries]
    ptrs = (C.c_void_p * max(1, n))(*[C.cast(b, C.c_void_p) for b in bufs])
    lens = (C.c_uint32 * max(1, n))(*[len(q) for q in queries])
    pa = _as_pieces(pieces)
    sptr = getattr(stream, "cuda_stream", stream)
    _check(lib().ifa_scan_brute_noalloc(device, ptrs, lens, n, C.c_void_p(ref_ptr), length,
                                        pa.ctypes.data, pa.size, max_subs, C.c_void_p(hits_ptr),
                                        hit_capacity, C.c_void_p(counters_ptr),
                                        C.c_void_p(per_query_counts_ptr or None),
                                        C.c_void_p(sptr or None)))


def _names(names, n):
    if names is None:
        return None
    arr = (C.c_char_p * max(1, n))()
    for i, x in enumerate(names):
        arr[i] = x.encode() if isinstance(x, str) else x
    return arr


def ifa_sam_records(hits: np.ndarray, queries: Sequence[bytes], primary_seen: np.ndarray,
                    query_names=None, contig_names=None) -> bytes:
    """Headerless SAM records for `hits` (sorted in place into reference
    order); `primary_seen` (uint8, one per query) carries the primary flags
    across calls of one pass over the reference."""
    hits = np.ascontiguousarray(hits, dtype=HIT_DTYPE)
    if primary_seen.dtype != np.uint8 or primary_seen.size != len(queries) or \
            not primary_seen.flags.c_contiguous:
        raise ValueError("primary_seen must be a contiguous uint8 array, one byte per query")
    nq = len(queries)
    bufs = [C.create_string_buffer(bytes(q), max(1, len(q))) for q in queries]
    info = ifa_sam_info()
    seqs = (C.c_void_p * max(1, nq))(*[C.cast(b, C.c_void_p) for b in bufs])
    lens = (C.c_uint32 * max(1, nq))(*[len(q) for q in queries])
    info.query_seqs = C.cast(seqs, C.POINTER(C.c_void_p))
    info.query_lens = C.cast(lens, C.POINTER(C.c_uint32))
    qn = _names(query_names, nq)
    info.query_names = C.cast(qn, C.POINTER(C.c_char_p)) if qn is not None else None
    info.n_queries = nq
    cn = _names(contig_names, len(contig_names) if contig_names is not None else 0)
    info.contig_names = C.cast(cn, C.POINTER(C.c_char_p)) if cn is not None else None
    info.n_contig_names = len(contig_names) if contig_names is not None else 0
    need = C.c_uint64()
    cap = max(1, hits.size) * 128
    while True:
        out = C.create_string_buffer(cap)
        st = lib().ifa_sam_records(hits.ctypes.data, hits.size, C.byref(info), primary_seen.ctypes.data,
                                   out, cap, C.byref(need))
        if st == IFA_ERR_INVALID_ARG and need.value > cap:
            cap = need.value
            continue
        _check(st)
        return out.raw[:need.value]


def ifa_sam_header(contig_lens, contig_ids=None, contig_names=None) -> bytes:
    """The separate SAM header (@HD, then one @SQ per contig)."""
    lens = np.ascontiguousarray(contig_lens, dtype=np.uint64)
    n = lens.size
    ids = None if contig_ids is None else np.ascontiguousarray(contig_ids, dtype=np.uint32)
    cn = _names(contig_names, n)
    need = C.c_uint64()
    cap = 64 + 64 * n
    while True:
        out = C.create_string_buffer(cap)
        st = lib().ifa_sam_header(cn, ids.ctypes.data if ids is not None else None, lens.ctypes.data, n,
                                  out, cap, C.byref(need))
        if st == IFA_ERR_INVALID_ARG and need.value > cap:
            cap = need.value
            continue
        _check(st)
        return out.raw[:need.value]


def ifa_last_error(h=None) -> str:
    return lib().ifa_last_error(h).decode(errors="replace")


# ------------------------------------------------------------ convenience

def sort_hits(h: np.ndarray) -> np.ndarray:
    if h.size == 0:
        return h
    order = np.lexsort((h["clips"], h["mismatches"], h["strand"], h["pos"], h["contig"], h["query"]))
    return h[order]


def segment_pieces(contig_len: np.ndarray, seg_bytes: int, contig_ids=None, lo: int = 0,
                   hi: Optional[int] = None):
    """Cut the range [lo, hi) (default: all) of a concatenated reference into
    (begin, end, PIECE_DTYPE array); begin/end are offsets into the whole
    reference.  A range starting inside a contig gives a first piece with
    offset_in_contig > 0 (prime the handle with ifa_prime_halo first, see
    shard_halo); one ending inside a contig gives a last piece with last = 0."""
    starts = np.concatenate([[0], np.cumsum(np.asarray(contig_len, np.int64))]).astype(np.int64)
    total = int(starts[-1]) if hi is None else min(int(hi), int(starts[-1]))
    ids = np.arange(len(contig_len), dtype=np.int64) if contig_ids is None else np.asarray(contig_ids)
    pos = int(lo)
    while pos < total:
        end = min(total, pos + seg_bytes)
        a = int(np.searchsorted(starts, pos, side="right")) - 1
        b = int(np.searchsorted(starts, end, side="left"))
        cs = starts[a:b]
        ce = starts[a + 1:b + 1]
        ps = np.maximum(cs, pos)
        pe = np.minimum(ce, end)
        arr = np.zeros(b - a, PIECE_DTYPE)
        arr["contig"] = ids[a:b]
        arr["offset_in_contig"] = ps - cs
        arr["start"] = ps - pos
        arr["len"] = pe - ps
        arr["last"] = (pe == ce).astype(np.uint32)
        keep = arr["len"] > 0
        yield pos, end, arr[keep]
        pos = end


def shard_range(total: int, world: int, rank: int) -> Tuple[int, int]:
    """Rank `rank`'s share [lo, hi) of a reference of `total` bases split into
    `world` contiguous ranges of (nearly) equal length.  Ranges may cut
    contigs; the scans need no exchange step (each window belongs to the
    range holding its last base), so hits concatenate and digests add."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return total * rank // world, total * (rank + 1) // world


def shard_halo(contig_len: np.ndarray, lo: int, lmax: int, contig_ids=None):
    """The halo a range starting at `lo` needs: (contig id, offset_in_contig,
    begin, end) of the up to lmax - 1 bases of lo's contig just before lo
    (begin/end are offsets into the whole reference), or None when lo is a
    contig start.  Pass ref[begin:end] to ifa_prime_halo."""
    starts = np.concatenate([[0], np.cumsum(np.asarray(contig_len, np.int64))]).astype(np.int64)
    if lo <= 0 or lo >= int(starts[-1]):
        return None
    ci = int(np.searchsorted(starts, lo, side="right")) - 1
    off = lo - int(starts[ci])
    if off == 0 or lmax <= 1:
        return None
    h = min(off, lmax - 1)
    cid = ci if contig_ids is None else int(np.asarray(contig_ids)[ci])
    return cid, off - h, lo - h, lo


class Aligner:
    """One handle: load queries once, stream the reference, drain hits."""

    def __init__(self, queries: Sequence[bytes] = (), max_subs=0,
                 mode: int = IFA_MODE_BRUTE, **cfg):
        """max_subs: one value for every query, or a sequence of one per query."""
        self.h = ifa_create(**cfg)
        self.nq = 0
        if queries:
            self.load_queries(queries)
        if np.ndim(max_subs) == 0:
            ifa_set_max_subs(self.h, int(max_subs))
        else:
            ifa_set_query_max_subs(self.h, max_subs)
        ifa_set_mode(self.h, mode)

    def close(self):
        if self.h:
            ifa_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def load_queries(self, queries):
        ifa_load_queries(self.h, queries)
        self.nq += len(queries)

    def scan(self, ref, contig_len, seg_bytes: Optional[int] = None, contig_ids=None,
             drain: bool = True):
        """Push a concatenated reference (numpy or torch) through in segments."""
        seg = seg_bytes or 256 << 20
        for a, b, pieces in segment_pieces(contig_len, seg, contig_ids):
            ifa_push_segment(self.h, ref[a:b], pieces)
        if drain:
            return ifa_drain_hits(self.h)
        return ifa_flush(self.h)
