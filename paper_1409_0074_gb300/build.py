"""Build liblagp_gb300.so (the CUDA kernels and the C ABI of include/lagp.h)
in-tree for sm_103a.

Translation units compile in parallel; the FP64 design kernels take
--fmad=false so that no multiply-add is contracted in the parity path (the
code also spells every operation with an explicitly rounded intrinsic).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblagp_gb300.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
UNITS = {
    "knn.cu": [],
    "knn_tc.cu": [],
    "design_fp64.cu": ["--fmad=false"],
    "design_fp32.cu": [],
    "ray32.cu": [],
    "exh_tc.cu": [],
    "lagp_api.cu": [],
    "profile.cu": [],
    "knn_noalloc.cu": [],
    "schedule.cu": [],
    "serve.cu": [],
    "mle.cu": [],
    "kdtree.cu": [],
    "prescale.cu": [],
}


def _sources():
    return [os.path.join(CSRC, f) for f in UNITS] + [
        os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))
    ] + [os.path.join(os.path.dirname(HERE), "include", "lagp.h")]


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _compile(unit, extra, verbose_ptxas=False):
    src = os.path.join(CSRC, unit)
    obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
    cmd = [NVCC] + ARCH + COMMON + extra + (["-Xptxas", "-v"] if verbose_ptxas else []) + [
        "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, r.stdout, r.stderr))
    return obj, r.stderr


def build(force=False, verbose_ptxas=False):
    """Compile every translation unit and link the shared library; returns its path."""
    if not force and not verbose_ptxas and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        results = list(ex.map(lambda kv: _compile(kv[0], kv[1], verbose_ptxas), UNITS.items()))
    if verbose_ptxas:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
