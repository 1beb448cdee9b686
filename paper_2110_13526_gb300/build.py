"""Build the sm_103a CUDA library ``libct_gb300.so`` in-tree with nvcc.

Each ``csrc/*.cu`` compiles in parallel to an object under ``_build/``; they
link into one shared library exporting the C ABI of ``include/ct.h``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libct_gb300.so")
# The bounds-checking variant (-DCT_DEBUG_BOUNDS; see csrc/ct_debug.cuh).
DEBUG_BUILD = os.path.join(BUILD, "debug")
DEBUG_LIB = os.path.join(BUILD, "libct_gb300_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = (sources() + glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))
    return any(os.path.getmtime(d) > t for d in deps)


def _variants(debug: bool):
    out = [(LIB, BUILD, [])]
    if debug:
        out.append((DEBUG_LIB, DEBUG_BUILD, ["-DCT_DEBUG_BOUNDS"]))
    return out


def build(force: bool = False, ptxas_verbose: bool = False, debug: bool = True) -> str:
    """Compile every CUDA source for sm_103a and link the shared library (and,
    with debug, the bounds-checking variant), all translation units of both in
    one parallel pool."""
    todo = [v for v in _variants(debug) if force or _stale(v[0])]
    if not todo:
        return LIB
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []
    jobs = []
    for lib, bdir, defs in todo:
        os.makedirs(bdir, exist_ok=True)
        for src in sources():
            jobs.append((src, os.path.join(bdir, os.path.basename(src)[:-3] + ".o"), defs))

    def one(job):
        src, obj, defs = job
        cmd = [cc] + ARCH + FLAGS + defs + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1))) as ex:
        results = list(ex.map(one, jobs))
    if ptxas_verbose:
        for _, log in results:
            print(log)
    for lib, bdir, _ in todo:
        objs = [o for o, _ in results if os.path.dirname(o) == bdir]
        tmp = lib + ".%d.tmp" % os.getpid()
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv))
