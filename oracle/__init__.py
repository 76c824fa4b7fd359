"""CPU oracle for stepping SSSP -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: the C source ``oracle.c`` is compiled with plain gcc into
``liboracle.so`` and called through ctypes.  Inputs are plain numpy CSR arrays
(off uint64[n+1], tgt uint32[m], w uint32[m]).

What it computes (see oracle.c for the passages each function follows):
  dijkstra        -- d(s, .), the plain definition of the output (pinned)
  bellman_ford    -- brute force, pins dijkstra on tiny graphs
  stepping        -- Algorithm 1 run sequentially with the ExtDist of Table 2
                     (rho, Delta*, Bellman-Ford, Delta with FinishCheck, Dijkstra)
  rho_extdist     -- the sampled rho-th smallest threshold (Sec. 6, App. B)
  delta_extdist   -- theta = i * Delta (Delta*-Stepping, Table 2)
  splitmix64      -- the counter-based generator the sampler uses
  check           -- the invariants that characterise d
  hops            -- fewest-hop shortest-path depth (Sec. 2), for step bounds
  lbpq_extract    -- LaB-PQ Extract(theta) on the plain set (Sec. 3.1, Table 1)
  lbpq_min        -- LaB-PQ Reduce (min) on the plain set
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

RHO, DELTA_STAR, BELLMAN_FORD, DELTA, DIJKSTRA = 0, 1, 2, 3, 4
INF = np.uint64(0xFFFFFFFFFFFFFFFF)


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class Stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("extracted", ctypes.c_uint64),
                ("edges", ctypes.c_uint64), ("updates", ctypes.c_uint64),
                ("full_steps", ctypes.c_uint64), ("partial_steps", ctypes.c_uint64),
                ("max_ext", ctypes.c_uint32), ("pad", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "pad"}


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P, u32, u64, i32, i64 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                 ctypes.c_int, ctypes.c_int64)
        lib.oracle_splitmix64.argtypes = [u64, u64]
        lib.oracle_splitmix64.restype = u64
        for f in (lib.oracle_dijkstra, lib.oracle_bellman_ford):
            f.argtypes = [u32, P, P, P, u32, P]
            f.restype = i32
        lib.oracle_reach.argtypes = [u32, P, P, u32, P]
        lib.oracle_reach.restype = i32
        lib.oracle_check.argtypes = [u32, P, P, P, u32, P, ctypes.POINTER(u32)]
        lib.oracle_check.restype = i32
        lib.oracle_hops.argtypes = [u32, P, P, P, u32, P]
        lib.oracle_hops.restype = i64
        lib.oracle_rho_extdist.argtypes = [P, u32, P, u32, u64, u64, u64, u32, u32]
        lib.oracle_rho_extdist.restype = u64
        lib.oracle_rho_extdist_capped.argtypes = [P, u32, P, u32, u64, u64, u64, u32, u32, u32]
        lib.oracle_rho_extdist_capped.restype = u64
        lib.oracle_delta_extdist.argtypes = [ctypes.POINTER(u64), u64, u64]
        lib.oracle_delta_extdist.restype = u64
        lib.oracle_delta_theta.argtypes = [ctypes.POINTER(u64), u64, u64]
        lib.oracle_delta_theta.restype = u64
        lib.oracle_delta_finish.argtypes = [ctypes.POINTER(u64), u64, u64]
        lib.oracle_delta_finish.restype = None
        lib.oracle_stepping.argtypes = [u32, P, P, P, u32, i32, u64, u64, u32, u32, u64, P, P,
                                        ctypes.POINTER(Stats)]
        lib.oracle_stepping.restype = i32
        lib.oracle_lbpq_extract.argtypes = [u32, P, P, u64, P]
        lib.oracle_lbpq_extract.restype = u32
        lib.oracle_lbpq_min.argtypes = [u32, P, P]
        lib.oracle_lbpq_min.restype = u64
        _lib = lib
    return _lib


def _arrs(g):
    off = np.ascontiguousarray(g.off, dtype=np.uint64)
    tgt = np.ascontiguousarray(g.tgt, dtype=np.uint32)
    w = np.ascontiguousarray(g.w, dtype=np.uint32)
    if tgt.size == 0:  # ctypes needs a valid pointer even for empty arrays
        tgt = np.zeros(1, np.uint32)
        w = np.zeros(1, np.uint32)
    return off, tgt, w


def splitmix64(seed: int, k: int) -> int:
    return int(_L().oracle_splitmix64(seed, k))


def dijkstra(g, s: int) -> np.ndarray:
    off, tgt, w = _arrs(g)
    dist = np.empty(g.n, dtype=np.uint64)
    rc = _L().oracle_dijkstra(g.n, off.ctypes.data, tgt.ctypes.data, w.ctypes.data, s,
                              dist.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_dijkstra failed")
    return dist


def bellman_ford(g, s: int) -> np.ndarray:
    off, tgt, w = _arrs(g)
    dist = np.empty(g.n, dtype=np.uint64)
    rc = _L().oracle_bellman_ford(g.n, off.ctypes.data, tgt.ctypes.data, w.ctypes.data, s,
                                  dist.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_bellman_ford failed")
    return dist


def reach(g, s: int) -> np.ndarray:
    off, tgt, _ = _arrs(g)
    r = np.empty(g.n, dtype=np.uint8)
    assert _L().oracle_reach(g.n, off.ctypes.data, tgt.ctypes.data, s, r.ctypes.data) == 0
    return r


def check(g, s: int, dist: np.ndarray) -> tuple[int, int]:
    """(code, vertex): code 0 when every invariant holds."""
    off, tgt, w = _arrs(g)
    dist = np.ascontiguousarray(dist, dtype=np.uint64)
    bad = ctypes.c_uint32(0)
    rc = _L().oracle_check(g.n, off.ctypes.data, tgt.ctypes.data, w.ctypes.data, s,
                           dist.ctypes.data, ctypes.byref(bad))
    return int(rc), int(bad.value)


def hops(g, s: int) -> tuple[np.ndarray, int]:
    """(h, depth): fewest-hop shortest-path hop counts and their maximum."""
    off, tgt, w = _arrs(g)
    h = np.empty(g.n, dtype=np.uint32)
    depth = _L().oracle_hops(g.n, off.ctypes.data, tgt.ctypes.data, w.ctypes.data, s,
                             h.ctypes.data)
    if depth < 0:
        raise ValueError("oracle_hops failed")
    return h, int(depth)


def rho_extdist(queue: np.ndarray, dist: np.ndarray, n: int, rho: int, seed: int, step: int,
                dense_before: int, reduced: int = 2, max_samples: int = 0) -> int:
    """reduced: how many dense steps use rho/10 (Sec. 6 uses the first two);
    max_samples: cap on the sample count (0 = 4096, the default rule)."""
    queue = np.ascontiguousarray(queue, dtype=np.uint32)
    dist = np.ascontiguousarray(dist, dtype=np.uint64)
    qp = queue.ctypes.data if queue.size else np.zeros(1, np.uint32).ctypes.data
    if max_samples:
        return int(_L().oracle_rho_extdist_capped(qp, queue.size, dist.ctypes.data, n, rho, seed, step,
                                                  dense_before, reduced, max_samples))
    return int(_L().oracle_rho_extdist(qp, queue.size, dist.ctypes.data, n, rho, seed, step,
                                       dense_before, reduced))


def delta_extdist(i: int, delta: int, qmin: int) -> tuple[int, int]:
    """(theta, next_i)."""
    ii = ctypes.c_uint64(i)
    th = int(_L().oracle_delta_extdist(ctypes.byref(ii), delta, qmin))
    return th, int(ii.value)


def delta_theta(i: int, delta: int, qmin: int) -> tuple[int, int]:
    """Original Delta-Stepping: (theta, i after the empty-bucket jump)."""
    ii = ctypes.c_uint64(i)
    th = int(_L().oracle_delta_theta(ctypes.byref(ii), delta, qmin))
    return th, int(ii.value)


def delta_finish(i: int, theta: int, min_new: int) -> int:
    """Original Delta-Stepping FinishCheck: the next i."""
    ii = ctypes.c_uint64(i)
    _L().oracle_delta_finish(ctypes.byref(ii), theta, min_new)
    return int(ii.value)


def stepping(g, s: int, algo: int, param: int, seed: int = 0,
             want_ext: bool = False, reduced: int = 2, warm_steps: int = 0,
             warm_rho: int = 0) -> tuple[np.ndarray, dict, np.ndarray | None]:
    """Algorithm 1 run sequentially: (dist, stats, per-vertex extraction counts).
    reduced: rho-Stepping's count of dense steps that use rho/10 (the paper's 2).
    warm_steps, warm_rho: rho-Stepping's first warm_steps steps use rho =
    warm_rho, without the dense-step reduction and without counting as dense
    steps (0 = the paper's schedule)."""
    off, tgt, w = _arrs(g)
    dist = np.empty(g.n, dtype=np.uint64)
    ext = np.empty(g.n, dtype=np.uint32) if want_ext else None
    st = Stats()
    rc = _L().oracle_stepping(g.n, off.ctypes.data, tgt.ctypes.data, w.ctypes.data, s, algo,
                              param, seed, reduced, warm_steps, warm_rho, dist.ctypes.data,
                              ext.ctypes.data if want_ext else None, ctypes.byref(st))
    if rc != 0:
        raise ValueError("oracle_stepping failed")
    return dist, st.as_dict(), ext


def lbpq_extract(inq: np.ndarray, key: np.ndarray, theta: int) -> np.ndarray:
    """LaB-PQ Extract(theta) on the plain set (inq: uint8[n], updated in place):
    the ids in Q with key <= theta, increasing."""
    assert inq.dtype == np.uint8 and inq.flags.c_contiguous
    key = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(max(1, inq.size), dtype=np.uint32)
    c = _L().oracle_lbpq_extract(inq.size, inq.ctypes.data, key.ctypes.data, theta, out.ctypes.data)
    return out[:c].copy()


def lbpq_min(inq: np.ndarray, key: np.ndarray) -> int:
    """LaB-PQ Reduce (min): the smallest key in Q, UINT64_MAX when empty."""
    inq = np.ascontiguousarray(inq, dtype=np.uint8)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    return int(_L().oracle_lbpq_min(inq.size, inq.ctypes.data, key.ctypes.data))
