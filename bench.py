"""Benchmark of the indel-free scan on the B300.

Workload (one step): 10 queries of 30-40 bp against a 4 Gbp synthetic
reference (GC 40%, log-normal contigs of 1 kbp - 5 Mbp, 0.1% N in runs of
10-1000, 1000 planted hits per substitution count k <= 16), scanned on both
strands in brute-force mode at maxSubs 0, 4, 8 and 16 -- one full pass of
the reference per maxSubs value, streamed as 256 MB segments.

* value: query-base comparisons per second (nominal: sum over windows of the
  query length, both strands) with the ASCII reference already resident in
  HBM; pack + scan + hit compaction run inside the timed region.
* e2e: the same metric through the C ABI from pinned host memory, with the
  host-to-device segment copies and the device-to-host hit drain inside
  the timed region.
* roofline: the brute-force scan kernel against the POPC pipe (one POPC per
  window evaluation of the first 32-base word), launch durations from CUDA
  events inside the library on the compute stream.
* cpu_baseline: the CPU oracle on a bounded sample of the same workload.

`--impl reference` times the CPU oracle instead (the reference arm).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "query-base comparisons/s and ref Gbp/s scanned (% of roofline); p50/p99 latency"
UNIT = "query-base comparisons/s"
SUBS = (0, 4, 8, 16)
SEG = 256 << 20
PIPE_RATES_MD = os.path.join(ROOT, "profiles", "int_pipe_rates.md")
PIPE_KINDS = ("popc", "lop3", "shf", "imad")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--total", type=float, default=4e9, help="reference bases (default 4 Gbp)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "batched", "serving", "indexed", "latency", "brute-kernels", "pipe-rates"],
                    help="sweep: the 4 Gbp maxSubs sweep (default); batched: many query sets "
                         "in one persistent launch vs one launch per set; serving: Poisson "
                         "arrivals with continuous batching")
    ap.add_argument("--sets", type=int, default=256, help="batched: number of query sets")
    ap.add_argument("--rate", type=float, default=50.0, help="serving: arrivals per second")
    ap.add_argument("--duration", type=float, default=20.0, help="serving: seconds of arrivals")
    ap.add_argument("--slices", type=int, default=16, help="serving: slices per cycle")
    ap.add_argument("--no-solo", action="store_true", help="serving: skip the one-request-at-a-time baseline")
    ap.add_argument("--sizes", default="16,32,64,512,10000", help="brute-kernels: query-set sizes")
    ap.add_argument("--subs", default="4", help="brute-kernels: maxSubs values")
    ap.add_argument("--solo-max-s", type=float, default=180.0,
                    help="serving: wall-time cap of the one-request-at-a-time baseline")
    ap.add_argument("--max-wall", type=float, default=float("inf"),
                    help="serving: wall-time cap of the continuous-batching run")
    ap.add_argument("--burst", type=int, default=0,
                    help="serving: first serve this many requests arriving at once (capacity)")
    ap.add_argument("--no-extras", action="store_true",
                    help="sweep: skip the other workloads' keys (latency, indexed, batched, serving)")
    return ap.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def make_workload(total, rank=0, world=1):
    """The 4 Gbp recipe.  Under N ranks it is one reference of N x `total`
    bases split by range: rank r builds only its range [lo, hi) (plus the
    bases its halo needs) and scans it; the ranges' hits together are one
    pass's hits (weak scaling: every rank scans `total` bases).  Returns
    (workload, lo, hi, halo) with halo as from P.shard_halo."""
    import synth
    import paper_2607_27291_b300 as P
    if world <= 1:
        wl = synth.workload_4gbp(total=int(total))
        return wl, 0, int(wl.ref.size), None
    lens = synth.contig_lengths(int(world * total), 1000, 5_000_000, "lognormal", 2)
    lo, hi = P.shard_range(int(lens.sum()), world, rank)
    lmax = max(len(q) for q in synth.random_queries(10, 30, 40, 2))
    halo = P.shard_halo(lens, lo, lmax)
    wl = synth.workload_4gbp(total=int(world * total), window=(halo[2] if halo else lo, hi))
    return wl, lo, hi, halo


def nominal_work(wl, contig_sel=None, lo=0, hi=None):
    """(windows, query-base comparisons) for one maxSubs pass, both strands:
    the windows whose last base lies in [lo, hi) (default: all)."""
    lens = wl.contig_len if contig_sel is None else wl.contig_len[contig_sel]
    starts = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64)
    hi = int(lens.sum()) if hi is None else hi
    win = 0
    qb = 0
    for q in wl.queries:
        L = len(q)
        first = np.maximum(starts + L - 1, lo)           # last base of the contig's first window
        last = np.minimum(starts + lens - 1, hi - 1)     # last base of its last window
        w = int(np.maximum(last - first + 1, 0).sum())
        win += 2 * w
        qb += 2 * w * L
    return win, qb


class Clocks:
    """nvidia-smi sampler for the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
            return
        # the timed region starts once the sampler has written its first row
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.p.poll() is None and os.path.getsize(self.f.name) == 0:
            time.sleep(0.01)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def popc_rate():
    """POPC results per SM per clock, from the committed microbenchmark
    record (bench.py --workload pipe-rates, kept in profiles/)."""
    for line in open(PIPE_RATES_MD):
        if line.strip().startswith("popc_per_clk_sm:"):
            return float(line.split(":", 1)[1])
    raise RuntimeError("no popc_per_clk_sm line in " + PIPE_RATES_MD)


def gather_rate():
    """Random 32-bit gathers per second from an L2-resident table, from the
    committed microbenchmark record (bench.py --workload pipe-rates)."""
    for line in open(PIPE_RATES_MD):
        if line.strip().startswith("random_gather_l2_per_s:"):
            return float(line.split(":", 1)[1])
    raise RuntimeError("no random_gather_l2_per_s line in " + PIPE_RATES_MD)


def pcie_peaks(dev, mb=256, reps=10):
    """Pinned host <-> device copy rates of `mb` MiB (GB/s): the best of `reps`
    single cudaMemcpyAsync copies from cudaHostAlloc memory and `reps` copies
    back to back on one stream (the streamed segments' pattern), from the
    probe library; torch's copy_ between pinned and device tensors beside
    them, for reference."""
    import ctypes as C
    import torch
    lib = C.CDLL(os.path.join(ROOT, "paper_2607_27291_b300", "libifa_probe.so"))
    f = lib.ifa_probe_copy_rate
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_uint64, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    native = {}
    for name, to_dev in (("h2d", 1), ("d2h", 0)):
        best, b2b = C.c_double(), C.c_double()
        rc = f(dev, mb << 20, to_dev, reps, C.byref(best), C.byref(b2b))
        if rc:
            raise RuntimeError("copy probe failed: %d" % rc)
        native[name + "_gbps"] = best.value
        native[name + "_gbps_back_to_back"] = b2b.value
    n = mb << 20
    host = torch.empty(n, dtype=torch.uint8).pin_memory()
    devb = torch.empty(n, dtype=torch.uint8, device=f"cuda:{dev}")
    st = torch.cuda.Stream(device=dev)
    out = {}
    for name, fn in (("h2d_gbps", lambda: devb.copy_(host, non_blocking=True)),
                     ("d2h_gbps", lambda: host.copy_(devb, non_blocking=True))):
        best = None
        with torch.cuda.stream(st):
            fn()
            for _ in range(reps):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(st)
                fn()
                b.record(st)
                b.synchronize()
                ms = a.elapsed_time(b)
                best = ms if best is None else min(best, ms)
        out[name] = n / (best * 1e-3) / 1e9
        with torch.cuda.stream(st):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(8):
                fn()
            b.record(st)
            b.synchronize()
        out[name + "_back_to_back"] = 8 * n / (a.elapsed_time(b) * 1e-3) / 1e9
    del host, devb
    native["torch_copy"] = out
    native["bytes"] = n
    native["how"] = ("cudaMemcpyAsync of %d MiB between cudaHostAlloc and device memory: best of %d single "
                     "copies, and %d back to back; CUDA events" % (mb, reps, reps))
    return native


def run_pipe_rates(args):
    """Integer-pipe issue rates per SM per clock (POPC, LOP3, SHF, IMAD) from
    the probe library, with the SM clock sampled meanwhile, and the pinned
    PCIe copy peaks."""
    import ctypes as C
    import torch
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    lib = C.CDLL(os.path.join(ROOT, "paper_2607_27291_b300", "libifa_probe.so"))
    f = lib.ifa_probe_pipe_rate
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double),
                  C.POINTER(C.c_double)]
    clocks = Clocks(dev)
    clocks.start()
    rates = {}
    for kind, name in enumerate(PIPE_KINDS):
        rows = []
        for _ in range(max(1, args.steps)):
            r, ms, mhz = C.c_double(), C.c_double(), C.c_double()
            rc = f(dev, kind, 4, 2000, C.byref(r), C.byref(ms), C.byref(mhz))
            if rc:
                raise RuntimeError("probe failed for %s: %d" % (name, rc))
            rows.append((r.value, ms.value, mhz.value))
        rows.sort()
        med = rows[len(rows) // 2]
        rates[name] = {"per_clk_sm": med[0], "ms": med[1], "sm_mhz_from_cycles": med[2],
                       "min": rows[0][0], "max": rows[-1][0]}
    g = lib.ifa_probe_gather_rate
    g.restype = C.c_int
    g.argtypes = [C.c_int, C.c_uint64, C.c_uint32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    gathers = {}
    for mb in (16, 64, 1024):
        best = None
        for _ in range(max(1, args.steps)):
            r, ms = C.c_double(), C.c_double()
            rc = g(dev, mb << 20, 512, C.byref(r), C.byref(ms))
            if rc:
                raise RuntimeError("gather probe failed: %d" % rc)
            best = r.value if best is None else max(best, r.value)
        gathers["%d MiB table" % mb] = best
    clk = clocks.stop()
    pcie = pcie_peaks(dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    line = {"workload": "pipe-rates", "metric": "results per SM per clock", "unit": "ops/clk/SM",
            "rates": rates, "random_gather_loads_per_s": gathers, "sms": sms, "clocks": clk, "pcie": pcie,
            "config": {"blocks_per_sm": 4, "threads": 256, "chains_per_thread": 8,
                       "instructions_per_thread": 2000 * 16 * 8, "runs": max(1, args.steps)}}
    print(json.dumps(line), flush=True)


def kernel_source_digest():
    """sha256 (first 16 hex digits) of the scan kernel's sources."""
    import hashlib
    h = hashlib.sha256()
    for f in ("scan_brute.cu", "scan_brute.cuh", "hits.cuh", "ifa_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2607_27291_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_record():
    """DRAM bytes per scan launch pair (scan + hit expansion) from the
    committed ncu summary, if it was taken on the current kernel source
    (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "scan_brute_4gbp_traffic.txt")
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        digest = kernel_source_digest()
        if kv.get("kernel_source_sha256_16") != digest:
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


# ---------------------------------------------------------------- CPU oracle

def cpu_sample(wl, target_bases):
    """First contigs covering about `target_bases` (the oracle's sample)."""
    c = np.cumsum(wl.contig_len)
    n = int(np.searchsorted(c, target_bases)) + 1
    n = min(n, len(wl.contig_len))
    return np.arange(n)


def time_oracle(wl, sel, subs=SUBS, threads=None):
    import oracle
    threads = threads or os.cpu_count() or 1
    end = int(wl.contig_len[sel].sum())
    ref = wl.ref[:end]
    lens = wl.contig_len[sel]
    t0 = time.perf_counter()
    for s in subs:
        oracle.brute(wl.queries, ref, lens, s, threads=threads)
    dt = time.perf_counter() - t0
    _, qb = nominal_work(wl, sel)
    return qb * len(subs) / dt, threads, dt, end


def run_reference(args, rank, world):
    if rank != 0:
        return
    import synth
    wl = synth.workload_4gbp(total=int(args.total), window=(0, 16_000_000))   # the sample's contigs
    sel = cpu_sample(wl, 4_000_000)
    for _ in range(max(0, args.warmup)):
        time_oracle(wl, sel[:1])
    vals = []
    dts = []
    for _ in range(args.steps):
        v, threads, dt, nb = time_oracle(wl, sel)
        vals.append(v)
        dts.append(dt)
    value = float(np.mean(vals))
    sample = "first %d contigs (%d bases) of the 4 Gbp reference, maxSubs %s" % (
        len(sel), nb, "/".join(map(str, SUBS)))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(dts)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": "10q30-40bp_4Gbp_GC40_sweep0-4-8-16", "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm

def run_ours(args, rank, world):
    import torch
    import paper_2607_27291_b300 as P

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    t_gen = time.perf_counter()
    wl, lo, hi, halo = make_workload(args.total, rank, world)
    t_gen = time.perf_counter() - t_gen
    off = wl.ref_offset
    segs = list(P.segment_pieces(wl.contig_len, SEG, lo=lo, hi=hi))
    ref_dev = torch.from_numpy(wl.ref).to(f"cuda:{dev}")
    stream = torch.cuda.Stream(device=dev)
    # hit buffer sized to the reference: the 4 Gbp sweep's maxSubs-16 pass emits
    # about 8.3e7 hits, a 256 Mbp profiling case about 5e6
    hcap = min(1 << 28, max(1 << 22, int(args.total) // 16))
    h = P.ifa_create(device=dev, hit_capacity=hcap, segment_bytes=SEG, profile=1)
    P.ifa_set_stream(h, stream)
    P.ifa_load_queries(h, wl.queries)
    P.ifa_set_mode(h, P.IFA_MODE_BRUTE)
    win_pass, qb_pass = nominal_work(wl, lo=lo, hi=hi)

    def one_pass(s, source, drain):
        P.ifa_reset_results(h)
        P.ifa_set_max_subs(h, s)
        if halo:
            P.ifa_prime_halo(h, halo[0], halo[1], source[halo[2] - off:halo[3] - off])
        for a, b, pc in segs:
            P.ifa_push_segment(h, source[a - off:b - off], pc)
        if drain:
            hits, _ = P.ifa_drain_hits(h, copy=False)
            return hits.size
        return 0

    # ---- device-resident timed region
    for _ in range(args.warmup):
        for s in SUBS:
            one_pass(s, ref_dev, False)
    torch.cuda.synchronize()
    barrier(world)
    clocks = Clocks(dev)
    clocks.start()
    step_ms = []
    per_s = {s: [] for s in SUBS}
    scan_ns = 0
    scan_launches = 0
    launches = 0
    hits_per_s = {}
    ev_all0 = torch.cuda.Event(enable_timing=True)
    ev_all1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev_all0.record(stream)
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in SUBS:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            one_pass(s, ref_dev, False)
            b.record(stream)
            st = P.ifa_get_stats(h)
            scan_ns += st["scan_ns"]
            scan_launches += st["scan_launches"]
            launches += st["kernel_launches"]
            dg, _ = P.ifa_get_digest(h)
            hits_per_s[s] = dg[0]
            per_s[s].append(a.elapsed_time(b))
        e1 = torch.cuda.Event(enable_timing=True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    ev_all1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    total_ms = ev_all0.elapsed_time(ev_all1)
    total_ms = allmax(total_ms, world)
    steps = args.steps
    qb_step = qb_pass * len(SUBS)
    qb_all = allsum(qb_step, world)            # every rank's windows: one pass over the whole reference
    bases_all = allsum(hi - lo, world)
    value = qb_all * steps / (total_ms * 1e-3)
    gbps = bases_all * len(SUBS) * steps / (total_ms * 1e-3) / 1e9

    # ---- roofline of the scan kernel (POPC pipe)
    peaks = measured_peaks()
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2032.0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # each brute-force chunk launch is a pair: the scan, which writes window
    # events, and the kernel that expands them into hits; the library times
    # the pair as one span, so a "launch" below is one pair
    pairs = max(1, scan_launches // 2)
    avg_launch_s = (scan_ns * 1e-9) / pairs
    evals_per_launch = win_pass * len(SUBS) * steps / pairs
    popc_clk = popc_rate()
    achieved = evals_per_launch / avg_launch_s / 1e9           # G popc / s
    peak = sms * popc_clk * sm_mhz * 1e6 / 1e9                 # G popc / s
    traffic = traffic_record()

    # ---- end to end through pinned host memory
    e2e = None
    if not args.no_e2e:
        P.ifa_destroy(h)
        del ref_dev
        torch.cuda.empty_cache()
        # end to end: pinned host ASCII in, every hit out to pinned host
        # memory through a fixed ring of 64 Mi hits (1 GiB) polled after each
        # segment, so hits leave while later segments are scanned
        ring = 1 << 26
        h = P.ifa_create(device=dev, hit_capacity=ring, segment_bytes=SEG)
        P.ifa_set_stream(h, stream)
        P.ifa_load_queries(h, wl.queries)
        P.ifa_set_mode(h, P.IFA_MODE_BRUTE)
        ref_pin = torch.from_numpy(wl.ref).pin_memory()
        dg_hits = max(int(v) for v in hits_per_s.values())
        out_t = torch.empty((dg_hits + ring) * 16, dtype=torch.uint8).pin_memory()
        out = out_t.numpy().view(P.HIT_DTYPE)

        def e2e_pass(s):
            P.ifa_reset_results(h)
            P.ifa_set_max_subs(h, s)
            if halo:
                P.ifa_prime_halo(h, halo[0], halo[1], ref_pin[halo[2] - off:halo[3] - off])
            got, over_any = 0, False
            for a, b, pc in segs:
                # the pinned reference stays unchanged: no wait for each copy
                P.ifa_push_segment(h, ref_pin[a - off:b - off], pc, P.IFA_MEM_HOST_PINNED_ASYNC)
                n, over, _ = P.ifa_poll_hits(h, out[got:])
                got += n
                over_any |= over
            n_polled = got
            while True:   # what the last segments left in the ring
                n, over, more = P.ifa_drain_into(h, out[got:])
                got += n
                over_any |= over
                if not more:
                    break
            return got, n_polled, over_any

        for s in SUBS:  # warm the pinned path
            e2e_pass(s)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = 0
        polled = 0
        overflow = False
        for s in SUBS:
            n, npol, ov = e2e_pass(s)
            d2h += n * 16 + 24
            polled += npol
            overflow |= ov
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = allmax(dt, world)
        pk = pcie_peaks(dev)
        pk_h2d = max(pk["h2d_gbps"], pk["h2d_gbps_back_to_back"])
        h2d = wl.ref.size * len(SUBS) / dt / 1e9
        e2e = {"value": qb_all / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(wl.ref.size) * len(SUBS), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": dt * 1e3, "pcie_h2d_gbps": h2d,
               "pcie_peak": pk, "pcie_h2d_frac": h2d / pk_h2d,
               "hit_ring": {"entries": ring, "bytes": ring * 16, "hits_per_step": (d2h - 24 * len(SUBS)) // 16,
                            "hits_polled_during_stream": polled, "overflow": overflow}}

        # The same sweep as one stream: the queries loaded once per maxSubs,
        # each copy at its own maxSubs (ifa_set_query_max_subs), so the
        # reference crosses PCIe once per step instead of once per maxSubs.
        # Same comparisons and hits (labelled by copy); reported beside the
        # per-pass figure above, which stays the headline.
        P.ifa_destroy(h)
        nq = len(wl.queries)
        h = P.ifa_create(device=dev, hit_capacity=ring, segment_bytes=SEG)
        P.ifa_set_stream(h, stream)
        P.ifa_load_queries(h, list(wl.queries) * len(SUBS))
        P.ifa_set_query_max_subs(h, [s for s in SUBS for _ in range(nq)])
        P.ifa_set_mode(h, P.IFA_MODE_BRUTE)

        def one_stream():
            P.ifa_reset_results(h)
            if halo:
                P.ifa_prime_halo(h, halo[0], halo[1], ref_pin[halo[2] - off:halo[3] - off])
            got, over_any = 0, False
            for a, b, pc in segs:
                P.ifa_push_segment(h, ref_pin[a - off:b - off], pc, P.IFA_MEM_HOST_PINNED_ASYNC)
                n, over, _ = P.ifa_poll_hits(h, out[got:])
                got += n
                over_any |= over
            while True:
                n, over, more = P.ifa_drain_into(h, out[got:])
                got += n
                over_any |= over
                if not more:
                    break
            return got, over_any

        one_stream()   # warm
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n1, ov1 = one_stream()
        torch.cuda.synchronize()
        dt1 = allmax(time.perf_counter() - t0, world)
        _, counts1 = P.ifa_get_digest(h, nq * len(SUBS))
        per_copy = {str(s): int(np.asarray(counts1[i * nq:(i + 1) * nq]).sum()) for i, s in enumerate(SUBS)}
        e2e["one_stream"] = {
            "value": qb_all / dt1, "unit": UNIT, "ms_per_step": dt1 * 1e3,
            "h2d_bytes_per_step": int(wl.ref.size), "d2h_bytes_per_step": int(n1 * 16 + 24),
            "pcie_h2d_gbps": wl.ref.size / dt1 / 1e9, "overflow": ov1,
            "hits_per_max_subs": per_copy,
            "hits_match_per_pass": all(per_copy[str(s)] == int(hits_per_s[s]) for s in SUBS),
            "what": "the four maxSubs of the sweep in one stream: %d query copies, copy i at maxSubs %s"
                    % (nq * len(SUBS), "/".join(str(s) for s in SUBS))}
    P.ifa_destroy(h)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        sel = cpu_sample(wl, 4_000_000)
        v, threads, dt, nb = time_oracle(wl, sel)
        sel1 = cpu_sample(wl, 250_000)
        v1, _, dt1, nb1 = time_oracle(wl, sel1, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "first %d contigs (%d bases) at maxSubs 0/4/8/16, %.1f s" % (
                   len(sel), nb, dt),
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1,
                                 "sample": "first %d contigs (%d bases) at maxSubs 0/4/8/16, %.1f s"
                                           % (len(sel1), nb1, dt1)}}

    if rank != 0:
        return
    lat = sorted(step_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "10q30-40bp_4Gbp_GC40_sweep0-4-8-16",
                   "reference_bases": int(bases_all), "contigs": int(wl.contig_len.size),
                   "sharding": ("one reference of %d bases split by range over %d ranks "
                                "(%d bases each, halo inside split contigs, no exchange)"
                                % (bases_all, world, hi - lo)) if world > 1 else "none",
                   "queries": len(wl.queries), "query_lengths": [len(q) for q in wl.queries],
                   "max_subs": list(SUBS), "segment_bytes": SEG, "mode": "brute-force",
                   "l2": "inputs (4 GB ASCII, 2 GB packed) exceed the 126 MB L2; no flush",
                   "generation_s": round(t_gen, 1)},
        "ref_gbps": gbps,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "what": "one step (4 passes over 4 Gbp)"},
        "sweep": {str(s): {"ms": float(np.mean(per_s[s])), "hits": int(hits_per_s[s]),
                           "qbase_per_s": qb_pass / (float(np.mean(per_s[s])) * 1e-3)}
                  for s in SUBS},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpopc/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_scan_brute_events + k_expand_events (one pair per segment and pass)",
                     "launches": pairs,
                     "avg_launch_ms": avg_launch_s * 1e3,
                     "peak_basis": "%d SMs x %.1f POPC/clk/SM (measured, profiles/int_pipe_rates.md) x "
                                   "%.0f MHz (median SM clock sampled during the timed region)"
                                   % (sms, popc_clk, sm_mhz)},
        "clocks": clk,
        "gpu_launches": int(launches),
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    if world == 1 and not args.no_extras:
        line.update(extras(args))
    print(json.dumps(line), flush=True)


def extras(args):
    """The other workloads, each measured once more in the same run: one
    short query's call latency (1 query, 10 x 1 Mbp), indexed mode (10,000
    queries vs 1 Gbp at maxSubs 4/8/16), 256 query sets in one persistent
    launch vs one launch per set (16 Gbp), and continuous-batching serving
    against a 200 Gbp store in HBM: the trace's first 16 requests at once,
    served to completion (capacity), then Poisson arrivals at 50/s for 30 s
    served for at most 45 s (one B300 falls far behind 50/s at 200 Gbp:
    the line reports the backlog and the throughput while saturated)."""
    import torch
    out = {}
    jobs = (("latency", lambda: latency_result(50, 5)),
            ("indexed", lambda: indexed_result(int(1e9), 5, 1, brute=False)),
            ("batched", lambda: batched_result(args, int(16e9), 1)),
            ("serving", lambda: serving_result(int(2e11), 50.0, 30.0, 64, None, 45.0, burst=16)))
    for name, fn in jobs:
        t = time.perf_counter()
        try:
            r = fn()
        except Exception as e:  # keep the headline line if one workload fails
            r = {"error": "%s: %s" % (type(e).__name__, e)}
        r["run_s"] = round(time.perf_counter() - t, 1)
        out[name] = r
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- many sets

def _store_from_device(P, h, ref_dev, lens):
    for a, b, pc in P.segment_pieces(lens, 256 << 20):
        P.ifa_ref_append(h, ref_dev[a:b], pc)


def run_batched(args):
    print(json.dumps(batched_result(args, int(args.total if args.total != 4e9 else 16e9), args.steps)),
          flush=True)


def batched_result(args, total, steps):
    """Query sets of uneven sizes against a device-resident reference: one
    persistent graph-replayed launch vs one launch per set."""
    import torch
    import paper_2607_27291_b300 as P
    import synth
    t = time.perf_counter()
    ref, lens, sets = synth.workload_sets_16gbp(total=total, n_sets=args.sets)
    t_gen = time.perf_counter() - t
    ref_dev = torch.from_numpy(ref).cuda()
    h = P.ifa_create(count_only=1, segment_bytes=256 << 20, minhits_trials=100_000, minhits_seed=1)
    _store_from_device(P, h, ref_dev, lens)
    del ref_dev
    torch.cuda.empty_cache()
    for qs, s in sets:
        P.ifa_set_add(h, qs, s, P.IFA_MODE_AUTO)
    nq = np.array([len(qs) for qs, _ in sets])
    work = float(nq.sum()) * ref.size          # bp x queries per run
    t = time.perf_counter()
    res = P.ifa_batch_run(h, P.IFA_BATCH_PERSISTENT, len(sets))   # calibrates, plans, captures
    t_plan = time.perf_counter() - t
    runs = []
    for _ in range(max(1, steps)):
        P.ifa_reset_results(h)
        res = P.ifa_batch_run(h, P.IFA_BATCH_PERSISTENT, len(sets))
        runs.append(float(res["done_ms"].max()))
    dig_p, cnt_p = P.ifa_get_digest(h, int(nq.sum()))
    P.ifa_reset_results(h)
    res_s = P.ifa_batch_run(h, P.IFA_BATCH_PER_SET, len(sets))
    dig_s, cnt_s = P.ifa_get_digest(h, int(nq.sum()))
    per_set_ms = float(res_s["done_ms"].max())
    P.ifa_destroy(h)
    pers_ms = float(np.median(runs))
    line = {
        "workload": "batched", "metric": "aggregate Gbp x queries/s", "unit": "Gbp*queries/s",
        "value": work / 1e9 / (pers_ms * 1e-3), "per_set_value": work / 1e9 / (per_set_ms * 1e-3),
        "persistent_ms": pers_ms, "per_set_ms": per_set_ms,
        "latency_ms": {"persistent": {"p50": pers_ms, "p99": pers_ms},
                       "per_set": {"p50": float(np.percentile(res_s["done_ms"], 50)),
                                   "p99": float(np.percentile(res_s["done_ms"], 99))}},
        "same_results": bool(dig_p == dig_s and (cnt_p == cnt_s).all()),
        "modes": {"brute_sets": int((res["mode"] == P.IFA_MODE_BRUTE).sum()),
                  "indexed_sets": int((res["mode"] == P.IFA_MODE_INDEXED).sum())},
        "hits": int(dig_p[0]),
        "config": {"reference_bases": int(ref.size), "contigs": int(lens.size), "sets": len(sets),
                   "queries": int(nq.sum()), "set_sizes": "log-uniform 1-5000",
                   "lengths": "18-50", "max_subs": "0-12 per set", "gc": "0.30-0.65 per contig",
                   "generation_s": round(t_gen, 1), "timed_runs": len(runs),
                   # the first ifa_batch_run: calibration, plan, graph capture and one full run
                   "first_run_s": round(t_plan, 1),
                   "plan_s": round(max(0.0, t_plan - pers_ms * 1e-3), 1)},
        "data": "synthetic",
    }
    del ref
    return line


def serve_trace(P, h, reqs, slices, budget, max_wall):
    """Replay the arrival trace through the serving loop; budget = HBM bytes
    for admission (1 admits one request at a time).  Stops early after
    max_wall seconds, leaving later requests unfinished."""
    P.ifa_serve_start(h, slices, budget, 1 << 20)
    ids = []
    open_ids = []   # submitted, not yet drained
    nxt = 0
    t0 = time.perf_counter()
    steps = 0
    cut = False
    drained_hits = 0
    while True:
        now = time.perf_counter() - t0
        if now > max_wall:
            cut = True
            break
        while nxt < len(reqs) and reqs[nxt][0] <= now:
            rid = P.ifa_serve_submit(h, reqs[nxt][1], reqs[nxt][2], P.IFA_MODE_AUTO)
            ids.append(rid)
            open_ids.append(rid)
            nxt += 1
        active, completed = P.ifa_serve_step(h)
        steps += 1
        if completed:
            # the client collects finished requests' hits (frees their rings)
            still = []
            for rid in open_ids:
                info = P.ifa_serve_poll(h, rid)
                if info["state"] == 2:
                    got, _ = P.ifa_serve_drain(h, rid, min(int(info["hits"]), 1 << 20))
                    drained_hits += got.size
                else:
                    still.append(rid)
            open_ids = still
        if nxt == len(reqs) and active == 0 and not open_ids:
            break
        if nxt < len(reqs) and active == 0:
            time.sleep(max(0.0, min(0.01, reqs[nxt][0] - now)))
    wall = time.perf_counter() - t0
    infos = [P.ifa_serve_poll(h, r) for r in ids]
    sst = P.ifa_serve_stats(h)
    P.ifa_serve_stop(h)
    done = [i for i in infos if i["state"] >= 2]
    # unfinished requests count with their latency so far (a lower bound)
    lat = np.array([i["done_s"] - i["submit_s"] for i in done] +
                   [wall - i["submit_s"] for i in infos if i["state"] < 2] +
                   [wall - r[0] for r in reqs[nxt:]])
    queue = np.array([i["admit_s"] - i["submit_s"] for i in done]) if done else np.zeros(1)
    return {"value": sst["query_bases"] / wall, "hits_drained": drained_hits,
            "cycle_s": wall / max(1.0, steps / slices),
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "p999": float(np.percentile(lat, 99.9))},
            "queue_s": {"p50": float(np.percentile(queue, 50)), "p99": float(np.percentile(queue, 99))},
            "modes": {"brute": sum(1 for i in infos if i["mode"] == P.IFA_MODE_BRUTE),
                      "indexed": sum(1 for i in infos if i["mode"] == P.IFA_MODE_INDEXED),
                      "not_admitted": sum(1 for i in infos if i["mode"] == P.IFA_MODE_AUTO)},
            "completed": len(done), "requests": len(reqs), "wall_s": wall, "steps": steps,
            "stopped_at_wall_limit": cut, "host_plan_s": sst["plan_s"], "device_scan_s": sst["scan_s"]}


def run_serving(args):
    total = int(args.total if args.total != 4e9 else 2e11)
    print(json.dumps(serving_result(total, args.rate, args.duration, args.slices,
                                    None if args.no_solo else args.solo_max_s, args.max_wall, args.burst)),
          flush=True)


def counter_store(P, h, ref, chunk=256 << 20):
    """Append a synth.CounterReference to the handle's store, generating
    each 256 MB chunk straight into device memory (the reference never
    exists on the host).  Returns (seconds, device bytes the store took)."""
    import torch
    from synth.devgen import DeviceFiller
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    t = time.perf_counter()
    fill = DeviceFiller(ref)
    P.ifa_ref_reserve(h, ref.total)
    buf = torch.empty(chunk, dtype=torch.uint8, device="cuda")
    for a, b, pc in P.segment_pieces(ref.contig_len, chunk):
        fill.fill(buf[:b - a], a)
        torch.cuda.synchronize()           # the append runs on the library's own stream
        P.ifa_ref_append(h, buf[:b - a], pc)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t
    del buf, fill
    torch.cuda.empty_cache()
    free1, _ = torch.cuda.mem_get_info()
    return dt, free0 - free1


def serving_result(total, rate, duration, slices, solo_max_s, max_wall, burst=0):
    """Poisson arrivals of query sets served by continuous batching over a
    device-resident reference, and optionally the same trace served one
    request at a time (admission limited to one active request).  References
    of 32 Gbp and more are counter-generated on the device (GC 45 %, 0.05 % N
    in runs, log-uniform contigs 1 kbp - 10 Mbp); smaller ones come from the
    host generator of the same recipe.  max_wall bounds the continuous-
    batching run (requests unfinished then count with their age)."""
    import torch
    import paper_2607_27291_b300 as P
    import synth
    reqs = synth.serving_requests(rate, duration)
    h = P.ifa_create(hit_capacity=1024, segment_bytes=256 << 20, minhits_trials=100_000, minhits_seed=1)
    if total >= 32e9:
        ref = synth.serving_reference(total)
        build_s, store_bytes = counter_store(P, h, ref)
        nbases, ncontigs = ref.total, len(ref.contig_len)
    else:
        ref_h, lens, _ = synth.workload_serving(total, rate, 0.0)
        ref_dev = torch.from_numpy(ref_h).cuda()
        t = time.perf_counter()
        _store_from_device(P, h, ref_dev, lens)
        build_s, store_bytes = time.perf_counter() - t, None
        nbases, ncontigs = int(ref_h.size), int(lens.size)
        del ref_dev, ref_h
        torch.cuda.empty_cache()
    # warm the planner's MinHits bins and the kernels with a one-query request
    P.ifa_serve_start(h, slices, 64 << 30, 1 << 20)
    P.ifa_serve_submit(h, reqs[0][1][:1], reqs[0][2], P.IFA_MODE_AUTO)
    while P.ifa_serve_step(h)[0]:
        pass
    burst_r = None
    if burst:
        # capacity: the trace's first `burst` requests all arrive at once and
        # are served together by continuous batching until every one is done
        burst_r = serve_trace(P, h, [(0.0, qs, s) for _, qs, s in reqs[:burst]], slices, 64 << 30,
                              float("inf"))
        burst_r["requests_per_s"] = burst / burst_r["wall_s"]
    cb = serve_trace(P, h, reqs, slices, 64 << 30, max_wall)
    solo = None
    if solo_max_s:
        solo = serve_trace(P, h, reqs, slices, 1, solo_max_s)
    P.ifa_destroy(h)
    return {
        "workload": "serving", "metric": "query-base comparisons/s (nominal) and request latency",
        "unit": "query-base comparisons/s", "value": cb["value"],
        "latency_s": cb["latency_s"], "queue_s": cb["queue_s"], "requests": len(reqs),
        "completed": cb["completed"], "wall_s": cb["wall_s"], "steps": cb["steps"],
        "stopped_at_wall_limit": cb["stopped_at_wall_limit"],
        "cycle_s": cb["cycle_s"], "sustained_requests_per_s": cb["completed"] / cb["wall_s"],
        "host_plan_s": cb["host_plan_s"], "device_scan_s": cb["device_scan_s"],
        "one_request_at_a_time": solo,
        "burst": burst_r,
        "config": {"reference_bases": nbases, "contigs": ncontigs, "rate_per_s": rate,
                   "duration_s": duration, "slices": slices, "max_wall_s": max_wall,
                   "store_build_s": round(build_s, 1), "store_device_bytes": store_bytes,
                   "set_sizes": "log-uniform 1-2000", "lengths": "18-50", "max_subs": "0-8",
                   "gc": 0.45, "n_frac": 0.0005, "mode": "auto by measured rates",
                   "admission": "HBM budget 64 GiB (continuous batching); baseline: one active request"},
        "data": "synthetic" + (", reference generated on the device" if total >= 32e9 else ""),
    }


def run_indexed(args):
    print(json.dumps(indexed_result(int(args.total if args.total != 4e9 else 1e9), args.steps, args.warmup,
                                    brute=True)), flush=True)


def indexed_result(total, steps, warmup, brute=True):
    """Indexed mode at scale: 10,000 queries of 20-40 bp against 1 Gbp
    (GC 50 %), maxSubs 4 / 8 / 16, MinHits from a 10^5-trial Monte Carlo on
    Philox seed 1; 5 % of the queries are planted once with exactly maxSubs
    substitutions.  Per maxSubs: a device-resident count-only pass timed with
    CUDA events, indexed (and, with `brute`, brute force) on the same handle,
    and the planted windows found (indexed mode's recall, the paper's
    false-negative rate)."""
    import torch
    import paper_2607_27291_b300 as P
    import synth
    out = {}
    for s in (4, 8, 16):
        wl = synth.workload_1gbp_indexed(total=total, plant_subs=s)
        dev = torch.from_numpy(wl.ref).cuda()
        stream = torch.cuda.Stream()
        h = P.ifa_create(count_only=1, segment_bytes=SEG, minhits_trials=100_000, minhits_seed=1, profile=1)
        P.ifa_set_stream(h, stream)
        P.ifa_load_queries(h, wl.queries)
        P.ifa_set_max_subs(h, s)
        segs = list(P.segment_pieces(wl.contig_len, SEG))
        _, qb = nominal_work(wl)
        res = {}
        modes = ((P.IFA_MODE_INDEXED, "indexed"), (P.IFA_MODE_BRUTE, "brute")) if brute else \
            ((P.IFA_MODE_INDEXED, "indexed"),)
        for mode, name in modes:
            P.ifa_set_mode(h, mode)
            times = []
            reps = steps if name == "indexed" else 1   # brute force: seconds per pass
            for rep in range(max(1, warmup) + reps):
                P.ifa_reset_results(h)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for x, y, pc in segs:
                    P.ifa_push_segment(h, dev[x:y], pc)
                b.record(stream)
                P.ifa_flush(h)
                b.synchronize()
                if rep >= max(1, warmup):
                    times.append(a.elapsed_time(b))
            st = P.ifa_get_stats(h)
            dg, _ = P.ifa_get_digest(h)
            ms = float(np.mean(times))
            res[name] = {"ms": ms, "effective_qbase_per_s": qb / (ms * 1e-3), "hits": dg[0],
                         "candidates": st["candidates"],
                         "candidates_per_s": st["candidates"] / (ms * 1e-3)}
            if name == "indexed":
                # roofline: random L2 accesses -- one k-mer lookup per position
                # and seeded table, one candidate window per verification --
                # against the measured random-gather rate
                kq, _, exq = P.ifa_get_query_plan(h, len(wl.queries))
                tables = len({int(k) for k, x in zip(kq, exq) if not x})
                acc = float(wl.ref.size) * tables + float(st["candidates"])
                peak = gather_rate()
                res[name]["roofline"] = {"bound": "l2 random access", "achieved": acc / (ms * 1e-3),
                                         "peak": peak, "unit": "accesses/s", "frac": acc / (ms * 1e-3) / peak,
                                         "tables": tables,
                                         "peak_basis": "random 32-bit gathers from an L2-resident table, "
                                                       "profiles/int_pipe_rates.md"}
        P.ifa_destroy(h)
        del dev
        torch.cuda.empty_cache()
        # recall on the planted windows: whether a window is a candidate
        # depends only on the window, so excerpts around the plants suffice
        pq = sorted({pl.query for pl in wl.plants})
        remap = {q: i for i, q in enumerate(pq)}
        starts = np.concatenate([[0], np.cumsum(wl.contig_len)[:-1]])
        parts, lens, where = [], [], []
        for pl in wl.plants:
            L = len(wl.queries[pl.query])
            a, b = pl.pos, pl.pos + L   # the planted window alone
            parts.append(wl.ref[starts[pl.contig] + a:starts[pl.contig] + b])
            lens.append(b - a)
            where.append((remap[pl.query], len(lens) - 1, pl.pos - a, pl.strand))
        exc = np.concatenate(parts)
        h = P.ifa_create(hit_capacity=1 << 25, segment_bytes=max(1 << 20, exc.size + 64),
                         minhits_trials=100_000, minhits_seed=1)
        P.ifa_load_queries(h, [wl.queries[q] for q in pq])
        P.ifa_set_max_subs(h, s)
        P.ifa_set_mode(h, P.IFA_MODE_INDEXED)
        for x, y, pc in P.segment_pieces(np.array(lens, np.int64), exc.size + 64):
            P.ifa_push_segment(h, exc[x:y], pc)
        hits, over = P.ifa_drain_hits(h)
        P.ifa_destroy(h)
        assert not over
        got = set(zip(hits["query"].tolist(), hits["contig"].tolist(), hits["pos"].tolist(),
                      hits["strand"].tolist()))
        found = sum(1 for w in where if w in got)
        res["planted"] = len(where)
        res["planted_found"] = found
        res["false_negative_rate"] = 1.0 - found / max(1, len(where))
        out[str(s)] = res
    line = {"workload": "indexed", "metric": "query-base comparisons/s (effective) and candidates verified/s",
            "unit": "query-base comparisons/s", "value": out["8"]["indexed"]["effective_qbase_per_s"],
            "per_max_subs": out,
            "config": {"reference_bases": total, "queries": 10000, "lengths": "20-40", "gc": 0.5,
                       "contigs": "log-uniform 10 kbp - 2 Mbp", "minhits_trials": 100000, "philox_seed": 1,
                       "planted": "5 % of queries, exactly maxSubs substitutions", "hits": "count only",
                       "steps": steps, "warmup": max(1, warmup), "brute_steps": 1 if brute else 0},
            "data": "synthetic"}
    return line


def run_latency(args):
    print(json.dumps(latency_result(args.steps, args.warmup)), flush=True)


def latency_result(steps, warmup):
    """One 20 bp query against 10 contigs of 1 Mbp (uniform ACGT), maxSubs 2,
    20 planted hits: latency of one whole call from pinned host ASCII (push,
    scan, drain) and of the device-resident scan alone."""
    import torch
    import paper_2607_27291_b300 as P
    import synth
    wl = synth.workload_1mbp_x10()
    pin = torch.from_numpy(wl.ref).pin_memory()
    dev = torch.from_numpy(wl.ref).cuda()
    h = P.ifa_create(hit_capacity=1 << 16, segment_bytes=16 << 20)
    P.ifa_load_queries(h, wl.queries)
    P.ifa_set_max_subs(h, 2)
    P.ifa_set_mode(h, P.IFA_MODE_BRUTE)
    segs = list(P.segment_pieces(wl.contig_len, 16 << 20))
    e2e, devl, nh = [], [], 0
    for rep in range(warmup + max(steps, 50)):
        for src, acc in ((pin, e2e), (dev, devl)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            P.ifa_reset_results(h)
            for x, y, pc in segs:
                P.ifa_push_segment(h, src[x:y], pc)
            hits, _ = P.ifa_drain_hits(h)
            dt = time.perf_counter() - t0
            if rep >= warmup:
                acc.append(dt * 1e3)
            nh = hits.size
    P.ifa_destroy(h)
    q = lambda a, p: float(np.percentile(a, p))
    line = {"workload": "latency", "metric": "latency of one call (ms) and ref Gbp/s",
            "unit": "ms", "value": q(e2e, 50), "higher_is_better": False,
            "e2e_ms": {"p50": q(e2e, 50), "p99": q(e2e, 99)},
            "device_resident_ms": {"p50": q(devl, 50), "p99": q(devl, 99)},
            "ref_gbps_e2e": wl.ref.size / (q(e2e, 50) * 1e-3) / 1e9, "hits": nh, "planted": len(wl.plants),
            "config": {"queries": 1, "length": 20, "reference": "10 x 1 Mbp uniform ACGT", "max_subs": 2,
                       "input": "ASCII from pinned host memory (e2e) or device memory",
                       "reps": len(e2e)},
            "data": "synthetic"}
    return line


def run_brute_kernels(args):
    """The two brute-force kernels on the same pass: bit-plane popcount and
    the tensor-core one-hot GEMM, over query-set sizes (queries of 20-40 bp,
    maxSubs 4) against a reference of the 4 Gbp recipe cut to --total bases
    (default 256 Mbp), device-resident, hits counted only.  Kernel time from
    the library's CUDA events; the digests of both kernels must agree."""
    import torch
    import paper_2607_27291_b300 as P
    import synth
    total = int(args.total if args.total != 4e9 else 256e6)
    sizes = [int(x) for x in args.sizes.split(",")]
    wl = synth.workload_4gbp(total=total, plants_per_k=1)
    dev = torch.from_numpy(wl.ref).cuda()
    segs = list(P.segment_pieces(wl.contig_len, SEG))
    allq = synth.random_queries(max(sizes), 20, 40, 11)
    import math

    def window_hit_rate(qs, s):
        # mean over queries of P(Binomial(L, 3/4) <= s): a uniform random window hits
        p = [sum(math.comb(len(q), i) * 0.75 ** i * 0.25 ** (len(q) - i) for i in range(min(s, len(q)) + 1))
             for q in qs]
        return sum(p) / len(p)

    rows = []
    for s_max, nq in [(int(x), n) for x in args.subs.split(",") for n in sizes]:
        r = {"queries": nq, "max_subs": s_max, "mean_window_hit_rate": window_hit_rate(allq[:nq], s_max)}
        for kern, name in ((P.IFA_BRUTE_POPC, "popcount"), (P.IFA_BRUTE_TENSOR, "tensor")):
            h = P.ifa_create(count_only=1, segment_bytes=SEG, profile=1, brute_kernel=kern)
            P.ifa_load_queries(h, allq[:nq])
            P.ifa_set_max_subs(h, s_max)
            P.ifa_set_mode(h, P.IFA_MODE_BRUTE)
            best = None
            for rep in range(max(1, args.warmup) + args.steps):
                P.ifa_reset_results(h)
                for a, b, pc in segs:
                    P.ifa_push_segment(h, dev[a:b], pc)
                P.ifa_flush(h)
                st = P.ifa_get_stats(h)
                if rep >= max(1, args.warmup):
                    ms = st["scan_ns"] / 1e6
                    best = ms if best is None else min(best, ms)
            dg, _ = P.ifa_get_digest(h)
            P.ifa_destroy(h)
            r[name] = {"ms": best, "evals_per_s": st["windows"] / (best * 1e-3), "digest": list(dg),
                       "hit_rate": dg[0] / max(1, st["windows"])}
        r["speedup"] = r["popcount"]["ms"] / r["tensor"]["ms"]
        r["same_digest"] = r["popcount"]["digest"] == r["tensor"]["digest"]
        rows.append(r)
    line = {"workload": "brute-kernels", "metric": "(query, strand, window) evaluations/s per brute-force kernel",
            "unit": "evaluations/s", "value": rows[-1]["tensor"]["evals_per_s"], "sizes": rows,
            "config": {"reference_bases": int(wl.ref.size), "query_lengths": "20-40",
                       "max_subs": [int(x) for x in args.subs.split(",")],
                       "hits": "count only", "timing": "best of --steps passes, library CUDA events"},
            "data": "synthetic"}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "indexed":
        return run_indexed(args)
    if args.workload == "latency":
        return run_latency(args)
    if args.workload == "brute-kernels":
        return run_brute_kernels(args)
    if args.workload == "pipe-rates":
        return run_pipe_rates(args)
    rank, world = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
