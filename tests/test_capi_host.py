"""Host-side checks of the C ABI: no GPU needed.

The library must load, export every function include/ifa.h declares, lay
out its structs as the header says (checked with gcc against the header
itself), carry the paper's defaults, and refuse bad arguments before
touching a device."""
import ctypes as C
import json
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import paper_2607_27291_b300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ifa.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ifa_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = P.lib()
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(P.exported_symbols()) == names


def test_bounds_checked_library_exports_the_same_symbols():
    """libifa_bc.so (-DIFA_BOUNDS_CHECK) is the same ABI: every declared
    function, nothing else of the ifa_ prefix."""
    from paper_2607_27291_b300 import build as b
    assert os.path.exists(b.BC_LIB_PATH)
    lib = C.CDLL(b.BC_LIB_PATH)
    for n in _declared():
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", b.BC_LIB_PATH], capture_output=True, text=True).stdout
    exported = sorted({w for w in re.findall(r"\b(ifa_[a-z_]+)\b", out)})
    assert exported == _declared()


def test_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "ifa.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(ifa_hit), sizeof(ifa_digest), sizeof(ifa_piece),
         sizeof(ifa_config), sizeof(ifa_stats));
  printf("%zu %zu %zu %zu\n", offsetof(ifa_hit, strand), offsetof(ifa_hit, mismatches),
         offsetof(ifa_config, minhits_seed), offsetof(ifa_config, auto_crossover));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe])
        out = subprocess.check_output([exe]).decode().split()
    sizes = list(map(int, out[:5]))
    offs = list(map(int, out[5:]))
    assert sizes == [16, 24, 32, C.sizeof(P.ifa_config), C.sizeof(P.ifa_stats)]
    assert P.HIT_DTYPE.itemsize == 16 and P.PIECE_DTYPE.itemsize == 32
    assert offs == [12, 13, P.ifa_config.minhits_seed.offset, P.ifa_config.auto_crossover.offset]


def test_defaults_are_the_papers():
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_defaults.json")))
    cfg = P.ifa_config_default()
    assert list(cfg.k_list)[:cfg.n_k] == g["k_list"]["value"]
    assert (cfg.minhits_num, cfg.minhits_den) == (g["minhits_probability"]["num"],
                                                  g["minhits_probability"]["den"])
    assert cfg.minhits_trials == g["minhits_trials"]["value"]
    # IFA_MODE_AUTO defaults to measured rates; the paper's count rule is
    # the configured alternative (tests/test_gpu_auto.py sets it from the
    # paper's 100-200 range)
    assert cfg.auto_crossover == 0
    assert cfg.clip_pct == 0 and cfg.kmer_step == 1 and cfg.mask_width == 0


def test_bad_config_rejected_before_device():
    for kw in ({"clip_pct": 51}, {"n_k": 0}, {"kmer_step": 0}, {"minhits_den": 0},
               {"k_list": [40]}, {"segment_bytes": 0}):
        with pytest.raises(P.IfaError) as ei:
            P.ifa_create(**kw)
        assert ei.value.status == P.IFA_ERR_INVALID_ARG, kw
    # NULL pointers return a status, they do not crash
    assert P.lib().ifa_create(None, None) == P.IFA_ERR_INVALID_ARG
    assert P.lib().ifa_flush(None) == P.IFA_ERR_INVALID_ARG
    assert P.lib().ifa_push_segment(None, None, 0, None, 0, 0) == P.IFA_ERR_INVALID_ARG
    assert P.ifa_last_error(None)


def test_minhits_entry_point_validates():
    with pytest.raises(P.IfaError):
        P.ifa_minhits(0, [20], [2], [0])          # k = 0
    with pytest.raises(P.IfaError):
        P.ifa_minhits(0, [300], [2], [8])         # L > 255
    with pytest.raises(P.IfaError):
        P.ifa_minhits(0, [20], [2], [8], step=0)


def test_segment_pieces_cover_reference():
    lens = np.array([5, 1, 17, 3, 40, 2], np.int64)
    for seg in (1, 4, 7, 16, 100):
        covered = []
        prev_open = None
        for a, b, pc in P.segment_pieces(lens, seg):
            assert pc["start"][0] == 0
            assert (np.diff(pc["start"].astype(np.int64)) == pc["len"][:-1].astype(np.int64)).all()
            assert int(pc["len"].sum()) == b - a
            assert (pc["last"][:-1] == 1).all()
            if prev_open is not None:
                assert pc["contig"][0] == prev_open[0] and pc["offset_in_contig"][0] == prev_open[1]
            prev_open = None if pc["last"][-1] else (pc["contig"][-1],
                                                     pc["offset_in_contig"][-1] + pc["len"][-1])
            for r in pc:
                covered.append((int(r["contig"]), int(r["offset_in_contig"]), int(r["len"])))
        per = {}
        for c, o, ln in covered:
            assert per.get(c, 0) == o
            per[c] = o + ln
        assert [per[i] for i in range(len(lens))] == lens.tolist()


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(P.IfaError) as ei:
        P.ifa_create()
    assert ei.value.status == P.IFA_ERR_CUDA


def test_noalloc_rejects_misaligned_buffers_before_device():
    """The allocation-free scan stores hits 16 bytes at a time and updates
    its counters with 64-bit atomics, so misaligned caller buffers are
    refused on the host.  The pointers below are never dereferenced: the
    check comes before any CUDA call, so this runs without a GPU."""
    pieces = [(0, 0, 0, 64, True)]
    q = [b"ACGTACGTAC"]
    cases = [(0x10004, 0x20000, 0), (0x10008, 0x20000, 0), (0x10000, 0x20004, 0), (0x10000, 0x20000, 0x30004)]
    for hits, counters, per_query in cases:
        with pytest.raises(P.IfaError) as ei:
            P.ifa_scan_brute_noalloc(0, q, 0x40000, 64, pieces, 1, hits, 16, counters, per_query)
        assert ei.value.status == P.IFA_ERR_INVALID_ARG
        assert "aligned" in str(ei.value)


HANDLE_CALLS = ["ifa_set_stream", "ifa_load_queries", "ifa_set_max_subs", "ifa_set_query_max_subs",
                "ifa_set_mode", "ifa_push_segment", "ifa_prime_halo", "ifa_flush", "ifa_drain_hits",
                "ifa_poll_hits", "ifa_get_digest", "ifa_reset_results", "ifa_get_stats", "ifa_get_query_plan",
                "ifa_ref_append", "ifa_ref_reserve", "ifa_ref_reset", "ifa_set_add", "ifa_batch_run",
                "ifa_serve_start", "ifa_serve_submit", "ifa_serve_step", "ifa_serve_poll", "ifa_serve_drain",
                "ifa_serve_stats", "ifa_serve_stop", "ifa_serve_cancel"]


def test_every_handle_call_rejects_a_null_handle():
    """Each entry point that takes a handle returns INVALID_ARG for NULL (no
    device is touched), whatever its other arguments."""
    import ctypes as C
    for name in HANDLE_CALLS:
        fn = getattr(P.lib(), name)
        args = []
        for t in fn.argtypes:
            args.append(None if (t is C.c_void_p or t is C.c_char_p or hasattr(t, "contents")) else t(0))
        assert fn(*args) == P.IFA_ERR_INVALID_ARG, name
    P.lib().ifa_destroy(None)   # a no-op
