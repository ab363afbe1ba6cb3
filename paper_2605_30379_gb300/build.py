"""Build libmrc.so (sm_103a) in-tree with nvcc; no cmake, no torch extension."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmrc.so")
SOURCES = ["api.cu", "misc.cu", "prof.cu", "noalloc.cu", "ozaki_tc.cu", "pair_tc.cu", "k_f64.cu", "k_f32.cu", "k_dd.cu",
           "k_f64_fft_lo.cu", "k_f64_fft_hi.cu", "k_f32_fft_lo.cu", "k_f32_fft_hi.cu", "k_dd_fft_lo.cu",
           "k_dd_fft_hi.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps_mtime():
    ts = [os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC)]
    ts.append(os.path.getmtime(os.path.join(HERE, "..", "include", "mrc.h")))
    ts.append(os.path.getmtime(__file__))
    return max(ts)


STAMP = os.path.join(BUILD, "flags.txt")


def _extra_flags():
    return os.environ.get("MRC_NVCC_FLAGS", "").split()


def _stamp_matches():
    try:
        with open(STAMP) as fh:
            return fh.read() == " ".join(_extra_flags())
    except OSError:
        return not _extra_flags()


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link libmrc.so unless it is newer than every source and was
    built with the same MRC_NVCC_FLAGS (extra nvcc options, e.g. -D macros)."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime() and _stamp_matches():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *_extra_flags(), "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(STAMP, "w") as fh:
        fh.write(" ".join(_extra_flags()))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
