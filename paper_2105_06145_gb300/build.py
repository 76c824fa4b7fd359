"""Build libsssp.so (the CUDA C-ABI library) in-tree with nvcc for sm_103a.

Usage: ``python -m paper_2105_06145_gb300.build`` (or ``__graft_entry__.build()``).
The translation units (and the narrow-shape build of the solve kernel) compile
in parallel; the result lands next to this file as ``libsssp.so``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsssp.so")
SOURCES = ["sssp_kernels.cu", "sssp_api.cu", "sssp_noalloc.cu", "sssp_batch.cu", "sssp_tune.cu",
           "sssp_tourney.cu", "sssp_msbatch.cu"]
HEADERS = ["sssp_internal.h", "sssp_device.cuh", os.path.join("..", "..", "include", "sssp.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NARROW_FLAGS = ["-Dsssp=sssp_narrow", "-DSSSP_BLOCK=512"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-v"] + ARCH


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          out: str | None = None) -> str:
    """Compile libsssp.so; `extra` adds nvcc flags (e.g. -D switches) and `out`
    writes the library elsewhere (objects then go to a separate folder)."""
    lib = out or LIB
    if not force and out is None and not extra and not _stale():
        return LIB
    bdir = BUILD if out is None else os.path.join(os.path.dirname(os.path.abspath(out)), "_build_variant")
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    # (source, object, extra flags): the solve kernel is also built in its narrow
    # shape, into its own namespace
    units = [(s, s.replace(".cu", ".o"), []) for s in SOURCES]
    units.append(("sssp_kernels.cu", "sssp_kernels_narrow.o", NARROW_FLAGS))
    for s, o, fl in units:
        obj = os.path.join(bdir, o)
        log = obj + ".log"
        cmd = [cc, *NVCC_FLAGS, *(extra or []), *fl, "-c", os.path.join(CSRC, s), "-o", obj]
        procs.append((subprocess.Popen(cmd, stdout=open(log, "w"), stderr=subprocess.STDOUT), cmd, log))
        objs.append(obj)
    failed = False
    for pr, cmd, log in procs:
        if pr.wait() != 0:
            failed = True
            sys.stderr.write(open(log).read())
        elif verbose:
            sys.stdout.write(open(log).read())
    if failed:
        raise RuntimeError("nvcc failed building libsssp")
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.check_call([cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
