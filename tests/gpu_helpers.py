"""Shared helpers for the GPU tests: run the CUDA path through the C ABI and
turn hit arrays into comparable tuple lists."""
import numpy as np

import paper_2607_27291_b300 as P


def tuples(h):
    return sorted(zip(h["query"].tolist(), h["contig"].tolist(), h["pos"].tolist(),
                      h["strand"].tolist(), h["mismatches"].tolist()))


def to_mem(arr: np.ndarray, kind: str):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(arr))
    if kind == "device":
        return t.cuda()
    if kind in ("pinned", "pinned_async"):
        return t.pin_memory()
    return np.ascontiguousarray(arr)


def gpu_scan(queries, ref, contig_len, max_subs, mode=P.IFA_MODE_BRUTE, seg_bytes=None,
             mem="host", contig_ids=None, **cfg):
    """Run one pass; returns (sorted hits, overflowed, digest, per-query counts, stats)."""
    cfg.setdefault("hit_capacity", 1 << 22)
    cfg.setdefault("segment_bytes", max(int(seg_bytes or 0), 1 << 20))
    h = P.ifa_create(**cfg)
    try:
        P.ifa_load_queries(h, queries)
        P.ifa_set_max_subs(h, max_subs)
        P.ifa_set_mode(h, mode)
        seg = seg_bytes or cfg["segment_bytes"]
        keep = []
        for a, b, pieces in P.segment_pieces(contig_len, seg, contig_ids):
            buf = to_mem(ref[a:b], mem)
            keep.append(buf)   # (pinned_async: unchanged until the flush below)
            P.ifa_push_segment(h, buf, pieces, P.IFA_MEM_HOST_PINNED_ASYNC if mem == "pinned_async" else None)
        P.ifa_flush(h)
        hits, over = P.ifa_drain_hits(h)
        dig, counts = P.ifa_get_digest(h, len(queries))
        stats = P.ifa_get_stats(h)
        return P.sort_hits(hits), over, dig, counts, stats
    finally:
        P.ifa_destroy(h)
