"""Build libmdjump.so (the CUDA path behind include/md.h) in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library next to this file. No cmake, no torch extension machinery.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libmdjump.so")
BUILD_DIR = os.path.join(HERE, "_build")
SOURCES = ["md_api.cu", "k_lists.cu", "k_force.cu", "k_jump.cu", "k_pme.cu", "k_vacf.cu", "noalloc.cu"]
# the velocity-phase kernel comes in several occupancy variants, and the pair
# kernels in thread-per-atom and half-list variants, that must give identical
# results: no mul/add contraction there (the compiler would fuse differently
# in each variant), every FMA is written out
PER_FILE = {"k_jump.cu": ["-fmad=false"], "k_force.cu": ["-fmad=false"]}
HEADERS = ["common.cuh", "engine.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                "-Xcompiler", "-fno-strict-aliasing", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmdjump.so")
    return p


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    """Compile every CUDA translation unit and link libmdjump.so; returns its path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "md.h")]
    flags = FLAGS + list(extra_flags or [])
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([nvcc(), *flags, *PER_FILE.get(src, []), "-c", s, "-o", o])
    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr
    with cf.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for out in ex.map(run, jobs):
            if verbose and out.strip():
                print(out)
    if force or jobs or _stale(OUT, objs):
        tmp = OUT + f".{os.getpid()}.tmp"
        # cuFFT (the PME transforms) is found at run time through the toolkit's library folder
        cudalib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc()))), "lib64")
        run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcufft", "-Xlinker", "-rpath=" + cudalib])
        os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
