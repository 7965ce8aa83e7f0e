"""Compile the CUDA library (libifa.so) in-tree for sm_103a with nvcc.

Usage: python -m paper_2607_27291_b300.build [--force]
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(ROOT, "_build")
LIB_PATH = os.path.join(HERE, "libifa.so")
# the same library with every read of the packed reference bounds-checked
# (-DIFA_BOUNDS_CHECK: a device error word, no trap); select it with IFA_LIB
BC_LIB_PATH = os.path.join(HERE, "libifa_bc.so")
# the integer-pipe issue-rate microbenchmark (a measurement tool, not the aligner)
PROBE_SRC = os.path.join(HERE, "probe", "pipe_rates.cu")
PROBE_LIB = os.path.join(HERE, "libifa_probe.so")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-I", CSRC, "-I", INCLUDE,
         "--expt-relaxed-constexpr"]
# extra nvcc flags for tuning builds (for example -DIFA_SCAN_MIN_CTAS=2)
FLAGS += os.environ.get("IFA_NVCC_EXTRA", "").split()


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=(), out: str = None, objs: str = None) -> str:
    lib_path = out or LIB_PATH
    build_dir = objs or (BUILD_DIR if out is None else out + ".objs")
    os.makedirs(build_dir, exist_ok=True)
    srcs = _sources()
    hdrs = _headers()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(build_dir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [NVCC] + ARCH + FLAGS + list(extra) + ["-c", s, "-o", o]
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(min(8, len(jobs))) as ex:
            futs = [ex.submit(subprocess.run, c, capture_output=True, text=True) for c in jobs]
            for c, f in zip(jobs, futs):
                r = f.result()
                if verbose or r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed: " + " ".join(c))
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib_path)
    if out is None and (force or _stale(PROBE_LIB, [PROBE_SRC])):
        tmp = PROBE_LIB + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
                               PROBE_SRC, "-o", tmp, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("probe build failed")
        os.replace(tmp, PROBE_LIB)
    return lib_path


def build_bounds_check(force: bool = False) -> str:
    return build(force=force, extra=["-DIFA_BOUNDS_CHECK"], out=BC_LIB_PATH, objs=os.path.join(BUILD_DIR, "bc"))


if __name__ == "__main__":
    out = None
    if "--out" in sys.argv:
        out = os.path.abspath(sys.argv[sys.argv.index("--out") + 1])
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else (), out=out))
