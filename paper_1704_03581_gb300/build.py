"""Build the pulda CUDA library in-tree: paper_1704_03581_gb300/_build/libpulda.so.

Every translation unit is compiled by nvcc for sm_103a only (GB300), in
parallel, then linked into one shared library exposing the C ABI of
include/pulda.h.  No cmake, no torch extension machinery.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libpulda.so")
GENCODE = "arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the pulda library needs the CUDA toolkit to build")
    return cand


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "pulda.h"))
    return hs


def _flags() -> list[str]:
    return ["-gencode", GENCODE, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
            "-fmad=false", "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
            "-I", os.path.join(ROOT, "include")]


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          out_dir: str | None = None) -> str:
    """Compile every source that changed and link the library; ``extra``
    nvcc flags (e.g. -D tile constants) and ``out_dir`` build a variant."""
    build_dir = out_dir or BUILD
    lib = os.path.join(build_dir, "libpulda.so")
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    srcs = sources()
    hdrs = headers()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(build_dir, os.path.basename(s) + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc, *_flags(), *(extra or []), "-c", s, "-o", o]
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed on {cmd[-3]}")
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [nvcc, "-gencode", GENCODE, "-shared", "-o", tmp, *objs, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("linking libpulda.so failed")
        os.replace(tmp, lib)
    return lib


BUILD_CHECKED = os.path.join(PKG, "_build_checked")


def build_checked(force: bool = False) -> str:
    """The library with PULDA_CHECKED defined: indices read from device data
    (topics) are bounds-checked in the kernels, and a bad one raises an error
    that pulda_sync reports instead of an out-of-bounds access.  For tests and
    debugging; load it through PULDA_LIB."""
    return build(force=force, extra=["-DPULDA_CHECKED"], out_dir=BUILD_CHECKED)


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
