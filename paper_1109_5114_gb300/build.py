"""Build libbsf.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_1109_5114_gb300/lib/libbsf.so`` with the static CUDA runtime.  Built
files are git-ignored.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libbsf.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                 "-I", INCLUDE, "-I", CSRC]
# The step solve (and the float64 covariance of log parameters) must give the
# same bits in every unit that runs it: no contraction of multiplies and adds
# into fused multiply-adds there.
_NOFMA = ["-fmad=false"]
EXTRA = {"bsf_steps.cu": _NOFMA, "bsf_continuous.cu": _NOFMA, "bsf_continuous64.cu": _NOFMA,
         "bsf_continuous128.cu": _NOFMA, "bsf_stencil.cu": _NOFMA, "bsf_backward.cu": _NOFMA,
         "bsf_two_pass.cu": _NOFMA, "bsf_stencil_second.cu": _NOFMA,
         "bsf_tiles.cu": _NOFMA, "bsf_sampled.cu": _NOFMA, "bsf_persistent.cu": _NOFMA}

SOURCES = ["bsf_api.cu", "bsf_steps.cu", "bsf_scan.cu", "bsf_stencil.cu", "bsf_backward.cu",
           "bsf_batch.cu", "bsf_noalloc.cu", "bsf_continuous.cu", "bsf_continuous64.cu",
           "bsf_continuous128.cu", "bsf_two_pass.cu", "bsf_stencil_second.cu", "bsf_tiles.cu",
           "bsf_sampled.cu", "bsf_persistent.cu"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbsf.so")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _headers():
    hs = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    hs += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return hs


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile (if stale) and return the path of libbsf.so."""
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    headers = _headers()
    jobs = []
    objs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [cc] + COMMON + EXTRA.get(src, []) + (["-Xptxas", "-v"] if ptxas_info else []) + ["-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or ptxas_info:
                print(" ".join(cmd))
                print(r.stdout, r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if force or jobs or _stale(LIB, objs):
        cmd = [cc] + ARCH + ["-shared", "-cudart", "static", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
