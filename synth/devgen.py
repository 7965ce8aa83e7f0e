"""ctypes wrapper of libsynth_dev.so: fill device memory with a slice of a
synth.CounterReference (the same bytes CounterReference.bases gives on the
host)."""
import ctypes as C
import os

import numpy as np

from . import gc_thresholds
from .build import LIB, build

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        L = C.CDLL(LIB)
        L.synth_dev_bases.restype = C.c_int
        L.synth_dev_bases.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_uint64, C.c_uint32, C.c_uint32,
                                      C.c_uint32, C.c_void_p, C.c_void_p, C.c_uint32, C.c_void_p]
        _lib = L
    return _lib


class DeviceFiller:
    """Fills torch uint8 CUDA tensors with slices of `ref`."""

    def __init__(self, ref, device="cuda"):
        import torch
        self.ref = ref
        # (one padding entry each, so that an empty run list still has an address)
        rs = np.concatenate([np.ascontiguousarray(ref.run_start, np.uint64), np.zeros(1, np.uint64)])
        rl = np.concatenate([np.ascontiguousarray(ref.run_len, np.uint32), np.zeros(1, np.uint32)])
        self.rs = torch.from_numpy(rs.view(np.int64)).to(device)
        self.rl = torch.from_numpy(rl.view(np.int32)).to(device)

    def fill(self, out, a: int, stream=None) -> None:
        """out[:] = bases [a, a + out.numel()) of the reference (one launch
        per GC span: the whole range, or each contig piece)."""
        n = out.numel()
        sptr = getattr(stream, "cuda_stream", stream) or None
        for lo, hi, g in self.ref.gc_spans(a, a + n):
            i0 = int(np.searchsorted(self.ref.run_start, lo, side="left"))
            i0 = max(0, i0 - 1)
            i1 = int(np.searchsorted(self.ref.run_start, hi, side="left"))
            t1, t2, t3 = gc_thresholds(g)
            rc = lib().synth_dev_bases(C.c_void_p(out.data_ptr() + (lo - a)), lo, hi - lo, self.ref.seed, t1, t2,
                                       t3, C.c_void_p(self.rs.data_ptr() + 8 * i0),
                                       C.c_void_p(self.rl.data_ptr() + 4 * i0), max(0, i1 - i0), C.c_void_p(sptr))
            if rc:
                raise RuntimeError("synth_dev_bases failed: %d" % rc)
