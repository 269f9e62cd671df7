"""Compiles the CUDA library ``libph_gb300.so`` in place (sm_103a only).

Every translation unit is compiled in parallel with nvcc, then linked into one shared library
that exports the C ABI of ``include/ph_gb300.h``. No GPU is needed to build. ``debug=True``
builds ``libph_gb300_debug.so`` instead, with the device-side bounds checks (``-DPH_DEBUG``);
the binding loads it when ``PH_GB300_DEBUG=1``.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = PKG / "libph_gb300.so"
BUILD_DEBUG = PKG / "_build_debug"
LIB_DEBUG = PKG / "libph_gb300_debug.so"
SOURCES = ["ph_scan.cu", "ph_build.cu", "ph_reduce.cu", "ph_api.cu", "ph_diff.cu",
           "ph_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    return "nvcc"


def _flags(extra=()):
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
            "--expt-relaxed-constexpr", *extra]


def build(force: bool = False, verbose: bool = False, extra_flags=(), debug: bool = False) -> Path:
    build_dir, lib = (BUILD_DEBUG, LIB_DEBUG) if debug else (BUILD, LIB)
    if debug:
        extra_flags = (*extra_flags, "-DPH_DEBUG")
    build_dir.mkdir(exist_ok=True)
    headers = list(CSRC.glob("*.cuh")) + [PKG.parent / "include" / "ph_gb300.h"]
    newest_header = max(p.stat().st_mtime for p in headers)
    objs = []
    jobs = []
    for src in SOURCES:
        s = CSRC / src
        o = build_dir / (Path(src).stem + ".o")
        objs.append(o)
        if force or not o.exists() or o.stat().st_mtime < max(s.stat().st_mtime, newest_header):
            jobs.append([nvcc(), *_flags(extra_flags), "-c", str(s), "-o", str(o)])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if verbose or r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd))

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if jobs or force or not lib.exists():
        tmp = lib.with_suffix(f".{os.getpid()}.tmp.so")
        run([nvcc(), *ARCH, "-shared", *map(str, objs), "-o", str(tmp), "-lcuda"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
