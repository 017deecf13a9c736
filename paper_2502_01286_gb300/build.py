"""Build libsncc.so in-tree for sm_103a (GB300).

Every translation unit is compiled by nvcc in parallel with one -gencode
(compute_103a -> sm_103a), then linked into
paper_2502_01286_gb300/_build/libsncc.so against the shared CUDA runtime.
Host code is compiled with -ffp-contract=off so that the segmentation's
floating-point comparisons round the same way on x86-64 and AArch64.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsncc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["sncc_host.cpp", "sncc_sat.cu", "sncc_match.cu", "sncc_refine.cu", "sncc_exact.cu", "sncc_probe.cu",
           "sncc_refine_seg.cu", "sncc_batch.cu",
           "sncc_diff.cu", "sncc_pipeline.cpp"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _flags(extra=()):
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I", INCLUDE, "-I", CSRC,
                   "-Xcompiler", "-fPIC,-ffp-contract=off,-O3", *extra]


def _compile(src: str, verbose_ptxas: bool) -> str:
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(["-Xptxas", "-v"] if verbose_ptxas else [])
    if src.endswith(".cpp"):
        cmd = [_nvcc(), "-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj] + _flags()
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    if verbose_ptxas:
        sys.stderr.write(r.stderr)
    return obj


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return any(os.path.getmtime(d) > t for d in deps) or os.path.getmtime(__file__) > t


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile and link libsncc.so if it is missing or older than its sources."""
    if not force and not verbose_ptxas and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [_nvcc(), "-shared", "-cudart", "shared", *ARCH, "-o", tmp, *objs,
           "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
