"""The device twin of the counter-based reference generator writes exactly
the bytes synth.CounterReference.bases gives on the host -- for slices at
unaligned offsets and lengths, across contigs with their own GC, and over
N-runs -- so that a reference too large for the host (200 Gbp) can be built
on the device and any slice of it regenerated on the host for the oracle."""
import numpy as np
import pytest

import synth
from synth.devgen import DeviceFiller

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", ["serving", "sets"])
def test_device_bytes_equal_host_bytes(which):
    import torch
    ref = synth.serving_reference(3_000_000_000) if which == "serving" else synth.sets_reference(60_000_000)
    fill = DeviceFiller(ref)
    rng = np.random.default_rng(3)
    cases = [(0, 1), (0, 4097), (ref.total - 777, 777)]
    cases += [(int(a), int(n)) for a, n in zip(rng.integers(0, ref.total - 3_000_000, size=12),
                                               rng.integers(1, 3_000_000, size=12))]
    if which == "serving":   # slices over N-runs
        for r in rng.choice(len(ref.run_start), size=6, replace=False):
            cases.append((int(ref.run_start[r]) - 37, int(ref.run_len[r]) + 91))
    for a, n in cases:
        out = torch.empty(n, dtype=torch.uint8, device="cuda")
        fill.fill(out, a)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        exp = ref.bases(a, a + n)
        assert np.array_equal(got, exp), (a, n)
    # base frequencies follow the GC model (45 % for the serving reference)
    if which == "serving":
        b = ref.bases(10_000_000, 12_000_000)
        gc = np.isin(b, np.frombuffer(b"GC", np.uint8)).sum() / np.isin(b, np.frombuffer(b"ACGT", np.uint8)).sum()
        assert abs(gc - 0.45) < 0.003
