"""Builds the CUDA library liblbm.so for sm_103a (in-tree, under _lib/).

Every translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a -O3 -lineinfo`` and linked into
one shared library exporting the C ABI of include/lbm.h; alongside, the
stand-alone ``pattern_probe`` program (the bandwidth ceiling of the step's
streaming pattern, run by bench.py).  Nothing here needs a GPU: nvcc
cross-compiles.
"""
from __future__ import annotations

import concurrent.futures
import os
import shlex
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(HERE, "_lib")
OBJDIR = os.path.join(LIBDIR, "obj")
LIBRARY = os.path.join(LIBDIR, "liblbm.so")
PROBE = os.path.join(LIBDIR, "pattern_probe")  # streaming-pattern bandwidth ceiling (pattern_probe.cu)

SOURCES = ["lbm_api.cu", "lbm_step.cu", "lbm_pair.cu", "lbm_pair_fp32.cu", "lbm_pair_fp16.cu", "lbm_pair_bf16.cu",
           "lbm_pair_wide.cu", "lbm_aux.cu", "lbm_noalloc.cu", "lbm_batch.cu", "lbm_unfused.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                     "-I", CSRC, "-I", INCLUDE]


def extra_flags() -> list:
    """Additional nvcc flags from LBM_NVCC_FLAGS (tuning builds, e.g. -DLBM_MIN_BLOCKS=4)."""
    return shlex.split(os.environ.get("LBM_NVCC_FLAGS", ""))


STAMP = os.path.join(LIBDIR, "flags.txt")


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbm.h"), __file__]
    return [f for f in files if os.path.isfile(f)]


def up_to_date() -> bool:
    if not os.path.exists(LIBRARY) or not os.path.exists(STAMP) or not os.path.exists(PROBE):
        return False
    if open(STAMP).read() != " ".join(extra_flags()):
        return False
    t = os.path.getmtime(LIBRARY)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(src: str, ptxas_verbose: bool) -> tuple:
    obj = os.path.join(OBJDIR, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc()] + NVCC_FLAGS + extra_flags() + (["-Xptxas", "-v"] if ptxas_verbose else []) + [
        "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _compile_probe() -> tuple:
    cmd = [nvcc()] + ARCH + ["-O3", "-std=c++17", os.path.join(CSRC, "pattern_probe.cu"), "-o", PROBE + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for pattern_probe.cu:\n{r.stdout}\n{r.stderr}")
    os.replace(PROBE + ".tmp", PROBE)
    return PROBE, r.stderr


def build(force: bool = False, ptxas_verbose: bool = False) -> str:
    """Compiles (if stale) and returns the path of liblbm.so."""
    if not force and not ptxas_verbose and up_to_date():
        return LIBRARY
    os.makedirs(OBJDIR, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        probe = ex.submit(_compile_probe)
        results = list(ex.map(lambda s: _compile(s, ptxas_verbose), SOURCES))
        probe.result()
    if ptxas_verbose:
        for _, log in results:
            print(log)
    tmp = LIBRARY + ".tmp"
    cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart_static", "-lrt",
                                                                                 "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIBRARY)
    with open(STAMP, "w") as f:
        f.write(" ".join(extra_flags()))
    return LIBRARY


if __name__ == "__main__":
    import sys

    print(build(force=True, ptxas_verbose="-v" in sys.argv))
