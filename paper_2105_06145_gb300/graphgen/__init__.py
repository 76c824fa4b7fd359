"""Seeded synthetic CSR graphs (input side only; no SSSP arithmetic).

The paper measures on real social, web and road graphs (Sec. 7, "Experimental
setup"); these generators stand in for them with the same structure: RMAT
power-law graphs with weights uniform in [1, 2^18) for the social/web class,
and jittered, bond-percolated grids with geometric weights for the road class.
Every choice is a pure function of (seed, index) (splitmix64), so the same
call gives the same graph on any host.  Both the CUDA path's tests and the CPU
oracle's tests take their inputs from here; this module computes no distance.

The C part (graphgen.c) is compiled by :func:`build` into ``libgraphgen.so``
next to this file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")

WMAX_EXCL = 1 << 18  # weights uniform in [1, 2^18) (Sec. 7)


def build(force: bool = False) -> str:
    """Compile libgraphgen.so with gcc (portable flags, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                _SRC, "-o", tmp, "-lm"]
        try:  # OpenMP when the toolchain has it; results do not depend on the thread count
            subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u32, u64, i32, i64, dbl = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int,
                                   ctypes.c_int64, ctypes.c_double)
        P = ctypes.c_void_p
        PP = ctypes.POINTER(ctypes.c_void_p)
        lib.graphgen_grid_edges.argtypes = [u32, u32]
        lib.graphgen_grid_edges.restype = u64
        lib.graphgen_grid.argtypes = [u32, u32, u64, u32, P, P, P]
        lib.graphgen_grid.restype = i32
        lib.graphgen_rmat.argtypes = [u32, u32, dbl, dbl, dbl, u64, u64, u32,
                                      ctypes.POINTER(u32), ctypes.POINTER(u64), PP, PP, PP]
        lib.graphgen_rmat.restype = i32
        lib.graphgen_road.argtypes = [u32, u64, dbl, dbl, u64,
                                      ctypes.POINTER(u32), ctypes.POINTER(u64), PP, PP, PP]
        lib.graphgen_road.restype = i32
        lib.graphgen_road_w.argtypes = [u32, u64, dbl, dbl, u64, u32, u64,
                                        ctypes.POINTER(u32), ctypes.POINTER(u64), PP, PP, PP]
        lib.graphgen_road_w.restype = i32
        lib.graphgen_rmat_n.argtypes = [u32, u32, dbl, dbl, dbl, u64, u64, u32, u32,
                                        ctypes.POINTER(u32), ctypes.POINTER(u64), PP, PP, PP]
        lib.graphgen_rmat_n.restype = i32
        lib.graphgen_random.argtypes = [u32, u64, u32, u32, u64, i32,
                                        ctypes.POINTER(u64), PP, PP, PP]
        lib.graphgen_random.restype = i32
        lib.graphgen_knn.argtypes = [u32, u32, dbl, u32, dbl, u64, ctypes.POINTER(u64), PP, PP, PP, P]
        lib.graphgen_knn.restype = i32
        lib.graphgen_largest_cc.argtypes = [u32, P, P, P]
        lib.graphgen_largest_cc.restype = i64
        lib.graphgen_kth_labelled.argtypes = [u32, P, u64]
        lib.graphgen_kth_labelled.restype = i64
        lib.graphgen_free.argtypes = [P]
        lib.graphgen_free.restype = None
        _lib = lib
    return _lib


@dataclass
class CSR:
    """Directed CSR graph: out-edges of u are tgt[off[u]:off[u+1]] with weights w."""
    n: int
    off: np.ndarray  # uint64[n+1]
    tgt: np.ndarray  # uint32[m]
    w: np.ndarray    # uint32[m]
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.tgt.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.off).astype(np.int64)

    def validate(self) -> None:
        assert self.off.dtype == np.uint64 and self.tgt.dtype == np.uint32 and self.w.dtype == np.uint32
        assert self.off.shape[0] == self.n + 1 and int(self.off[0]) == 0
        assert int(self.off[-1]) == self.m
        assert np.all(self.off[1:] >= self.off[:-1])
        if self.m:
            assert int(self.tgt.max()) < self.n


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _take(ptr: ctypes.c_void_p, dtype, count: int) -> np.ndarray:
    """Copy a malloc'd C array into numpy and free it."""
    lib = _L()
    if count == 0:
        lib.graphgen_free(ptr)
        return np.zeros(0, dtype=dtype)
    buf = (ctypes.c_char * (count * np.dtype(dtype).itemsize)).from_address(ptr.value)
    out = np.frombuffer(buf, dtype=dtype, count=count).copy()
    lib.graphgen_free(ptr)
    return out


def from_edges(n: int, src, dst, w, name: str = "edges") -> CSR:
    """CSR from an explicit directed edge list (kept in the given order per source)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.uint32)
    w = np.asarray(w, dtype=np.uint32)
    order = np.argsort(src, kind="stable")
    counts = np.bincount(src, minlength=n) if src.size else np.zeros(n, np.int64)
    off = np.zeros(n + 1, dtype=np.uint64)
    off[1:] = np.cumsum(counts).astype(np.uint64)
    return CSR(n, off, dst[order].copy(), w[order].copy(), name)


def grid(R: int, C: int, wseed: int = 1, wmax_excl: int = WMAX_EXCL) -> CSR:
    """4-neighbour R x C grid, id = r*C + c, both directions of every edge.
    wmax_excl = 0 gives unit weights."""
    lib = _L()
    m = int(lib.graphgen_grid_edges(R, C))
    off = np.zeros(R * C + 1, dtype=np.uint64)
    tgt = np.zeros(m, dtype=np.uint32)
    w = np.zeros(m, dtype=np.uint32)
    rc = lib.graphgen_grid(R, C, wseed, wmax_excl, _ptr(off), _ptr(tgt), _ptr(w))
    assert rc == 0
    return CSR(R * C, off, tgt, w, f"grid{R}x{C}", {"R": R, "C": C, "wseed": wseed})


def _cached(key: str, make):
    """When SSSP_GRAPH_CACHE names a directory, keep generated graphs there as
    .npy files so that several processes of one run share one generation."""
    d = os.environ.get("SSSP_GRAPH_CACHE")
    if not d:
        return make()
    base = os.path.join(d, key)
    try:
        off = np.load(base + ".off.npy")
        tgt = np.load(base + ".tgt.npy")
        w = np.load(base + ".w.npy")
        meta = {}
        return CSR(off.shape[0] - 1, off, tgt, w, key, meta)
    except (OSError, ValueError):
        pass
    g = make()
    os.makedirs(d, exist_ok=True)
    for nm, arr in (("off", g.off), ("tgt", g.tgt), ("w", g.w)):
        tmp = f"{base}.{nm}.tmp{os.getpid()}.npy"
        np.save(tmp, arr)
        os.replace(tmp, f"{base}.{nm}.npy")
    return g


def rmat(scale: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         gen_seed: int = 2, wseed: int = 3, wmax_excl: int = WMAX_EXCL) -> CSR:
    """RMAT power-law graph, symmetrised, no self-loops or duplicates, vertices
    randomly relabelled; weights uniform in [1, wmax_excl)."""
    key = f"rmat_s{scale}_ef{edgefactor}_{a}_{b}_{c}_g{gen_seed}_w{wseed}_{wmax_excl}"
    g = _cached(key, lambda: _rmat(scale, edgefactor, a, b, c, gen_seed, wseed, wmax_excl))
    g.name = f"rmat{scale}"
    g.meta = {"scale": scale, "edgefactor": edgefactor, "gen_seed": gen_seed, "wseed": wseed}
    return g


def _rmat(scale, edgefactor, a, b, c, gen_seed, wseed, wmax_excl, n_keep=0) -> CSR:
    lib = _L()
    n = ctypes.c_uint32()
    m = ctypes.c_uint64()
    po, pt, pw = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    rc = lib.graphgen_rmat_n(scale, edgefactor, a, b, c, gen_seed, wseed, wmax_excl, n_keep,
                             ctypes.byref(n), ctypes.byref(m),
                             ctypes.byref(po), ctypes.byref(pt), ctypes.byref(pw))
    if rc != 0:
        raise MemoryError("graphgen_rmat failed")
    nn, mm = n.value, m.value
    return CSR(nn, _take(po, np.uint64, nn + 1), _take(pt, np.uint32, mm), _take(pw, np.uint32, mm),
               f"rmat{scale}", {"scale": scale, "edgefactor": edgefactor, "gen_seed": gen_seed,
                                "wseed": wseed})


def road(side: int, keep: float = 0.75, seed: int = 5, jitter: float = 0.4,
         wscale: float = 1000.0) -> CSR:
    """Road-like graph: jittered side x side point grid, each 4-neighbour edge
    kept with probability `keep`, weight floor(wscale * length) + 1."""
    key = f"road_{side}_{keep}_{seed}_{jitter}_{wscale}"
    g = _cached(key, lambda: _road(side, keep, seed, jitter, wscale))
    g.name = f"road{side}"
    g.meta = {"side": side, "keep": keep, "seed": seed}
    return g


def _road(side, keep, seed, jitter, wscale, wmax_excl=0, wseed=0) -> CSR:
    lib = _L()
    keep_num = min((1 << 64) - 1, int(round(keep * float(1 << 64))))
    n = ctypes.c_uint32()
    m = ctypes.c_uint64()
    po, pt, pw = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    rc = lib.graphgen_road_w(side, keep_num, jitter, wscale, seed, wmax_excl, wseed,
                             ctypes.byref(n), ctypes.byref(m),
                             ctypes.byref(po), ctypes.byref(pt), ctypes.byref(pw))
    if rc != 0:
        raise MemoryError("graphgen_road failed")
    nn, mm = n.value, m.value
    return CSR(nn, _take(po, np.uint64, nn + 1), _take(pt, np.uint32, mm), _take(pw, np.uint32, mm),
               f"road{side}", {"side": side, "keep": keep, "seed": seed})


def random_graph(n: int, m: int, wlo: int = 1, whi: int = (1 << 18) - 1, seed: int = 0,
                 drop_self_loops: bool = False) -> CSR:
    """Uniform random directed multigraph (self-loops and duplicates allowed
    unless dropped); weights uniform in [wlo, whi]."""
    lib = _L()
    mo = ctypes.c_uint64()
    po, pt, pw = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    rc = lib.graphgen_random(n, m, wlo, whi, seed, int(drop_self_loops), ctypes.byref(mo),
                             ctypes.byref(po), ctypes.byref(pt), ctypes.byref(pw))
    if rc != 0:
        raise MemoryError("graphgen_random failed")
    mm = mo.value
    return CSR(n, _take(po, np.uint64, n + 1), _take(pt, np.uint32, mm), _take(pw, np.uint32, mm),
               f"random{n}x{m}", {"seed": seed})


def largest_cc(g: CSR) -> np.ndarray:
    """uint8 mask of the largest connected component of the undirected view."""
    lib = _L()
    lab = np.zeros(g.n, dtype=np.uint8)
    sz = lib.graphgen_largest_cc(g.n, _ptr(g.off), _ptr(g.tgt), _ptr(lab))
    assert sz >= 0
    return lab


def _sm64(seed: int, k: int) -> int:
    M = (1 << 64) - 1
    z = (seed + (k + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def pick_sources(g: CSR, k: int, seed: int, mask: np.ndarray | None = None) -> list[int]:
    """k distinct sources drawn uniformly from the largest connected component
    (or from `mask` when given), deterministic in `seed`."""
    if mask is None:
        mask = largest_cc(g)
    ids = np.flatnonzero(mask)
    k = min(k, ids.size)
    out, seen, j = [], set(), 0
    while len(out) < k:
        r = (_sm64(seed, j) * ids.size) >> 64
        j += 1
        v = int(ids[r])
        if v not in seen:
            seen.add(v)
            out.append(v)
    return out


def chain(n: int, wseed: int = 0, wlo: int = 1, whi: int = 100, both: bool = False) -> CSR:
    """Path 0-1-...-(n-1); weights uniform in [wlo, whi] from wseed."""
    src, dst, w = [], [], []
    for i in range(n - 1):
        ww = wlo + ((_sm64(wseed, i) * (whi - wlo + 1)) >> 64)
        src.append(i); dst.append(i + 1); w.append(ww)
        if both:
            src.append(i + 1); dst.append(i); w.append(ww)
    return from_edges(n, src, dst, w, f"chain{n}")


def star(n: int, wseed: int = 0, wlo: int = 1, whi: int = 1000) -> CSR:
    """Directed star: centre 0 with edges 0 -> i for i = 1..n-1."""
    src = [0] * (n - 1)
    dst = list(range(1, n))
    w = [wlo + ((_sm64(wseed, i) * (whi - wlo + 1)) >> 64) for i in range(n - 1)]
    return from_edges(n, src, dst, w, f"star{n}")


def complete(n: int, wseed: int = 0, wlo: int = 1, whi: int = 1000) -> CSR:
    """Complete directed graph without self-loops."""
    src, dst, w = [], [], []
    k = 0
    for u in range(n):
        for v in range(n):
            if u != v:
                src.append(u); dst.append(v)
                w.append(wlo + ((_sm64(wseed, k) * (whi - wlo + 1)) >> 64))
                k += 1
    return from_edges(n, src, dst, w, f"complete{n}")


# ---------------------------------------------------------------------------
# The named workloads (synthetic stand-ins for the paper's graphs).
# ---------------------------------------------------------------------------

def workload_grid256() -> tuple[CSR, int]:
    """256 x 256 grid, weights uniform in [1, 2^18) from seed 1, source 0."""
    return grid(256, 256, wseed=1), 0


def workload_rmat(scale: int = 22, source_seed: int = 4) -> tuple[CSR, int]:
    """RMAT scale 22 (default), edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
    generator seed 2, weight seed 3; one source uniform in the largest
    connected component (seed 4)."""
    g = rmat(scale, 16, 0.57, 0.19, 0.19, gen_seed=2, wseed=3)
    return g, pick_sources(g, 1, source_seed)[0]


def workload_road(side: int = 4096) -> tuple[CSR, int]:
    """Road-like 4096^2 jittered grid (seed 5), source at the centre, moved to
    the nearest vertex of the largest component (by raster distance) if needed."""
    g = road(side, 0.75, seed=5)
    lab = largest_cc(g)
    c = (side // 2) * side + side // 2
    d = 0
    while True:
        for v in (c + d, c - d):
            if 0 <= v < g.n and lab[v]:
                return g, int(v)
        d += 1


def rmat_n(n: int, edgefactor: int, gen_seed: int, wseed: int, wmax_excl: int = WMAX_EXCL) -> CSR:
    """RMAT at scale ceil(log2 n) with the edges that have an endpoint >= n
    rejected (after the relabelling), so the graph has exactly n vertices."""
    scale = max(1, int(n - 1).bit_length())
    g = _rmat(scale, edgefactor, 0.57, 0.19, 0.19, gen_seed, wseed, wmax_excl, n)
    g.name = f"rmat_n{n}"
    return g


def jittered_grid_uniform(side: int, seed: int, wseed: int, keep: float = 0.75,
                          wmax_excl: int = WMAX_EXCL) -> CSR:
    """The road generator's topology (jittered side x side grid, edges kept with
    probability `keep`) with weights uniform in [1, wmax_excl)."""
    g = _road(side, keep, seed, 0.4, 1000.0, wmax_excl, wseed)
    g.name = f"jgrid{side}"
    return g


def workload_multi(count: int = 512, lo_log2: int = 10, hi_log2: int = 18, seed: int = 7,
                   rmat_edgefactor: int = 6) -> list[tuple[CSR, int]]:
    """Many independent graphs of uneven size: n log-uniform in
    [2^lo_log2, 2^hi_log2]; the first half jittered grids (side ceil(sqrt n),
    edges kept with probability 0.75), the second half RMAT at scale
    ceil(log2 n) with out-of-range endpoints rejected (edge factor 6 keeps the
    total near 2^27 directed edges for the default 512 graphs); weights uniform
    in [1, 2^18); one source per graph uniform in its largest component."""
    out = []
    for i in range(count):
        u = (_sm64(seed, 3 * i) >> 11) * (1.0 / (1 << 53))
        n = int(round(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * u)))
        gseed = _sm64(seed, 3 * i + 1) & 0x7FFFFFFF
        wseed = _sm64(seed, 3 * i + 2) & 0x7FFFFFFF
        if i < count // 2:
            side = int(np.ceil(np.sqrt(n)))
            g = jittered_grid_uniform(side, gseed, wseed)
        else:
            g = rmat_n(n, rmat_edgefactor, gseed, wseed)
        src = pick_sources(g, 1, gseed)[0]
        out.append((g, src))
    return out


def knn(npts: int = 2_000_000, clusters: int = 64, sigma: float = 0.02, k: int = 10,
        wscale: float = float(1 << 20), seed: int = 10, with_points: bool = False):
    """Symmetrised k-NN graph of points from a 3-D cluster mixture (see
    graphgen_knn); weight floor(2^20 * distance) + 1.  Returns the CSR (and the
    points when with_points)."""
    key = f"knn_{npts}_{clusters}_{sigma}_{k}_{wscale}_{seed}"

    def make():
        lib = _L()
        m = ctypes.c_uint64()
        po, pt, pw = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        rc = lib.graphgen_knn(npts, clusters, sigma, k, wscale, seed, ctypes.byref(m),
                              ctypes.byref(po), ctypes.byref(pt), ctypes.byref(pw), None)
        if rc != 0:
            raise MemoryError("graphgen_knn failed")
        mm = m.value
        return CSR(npts, _take(po, np.uint64, npts + 1), _take(pt, np.uint32, mm), _take(pw, np.uint32, mm))

    g = _cached(key, make)
    g.name = f"knn{npts}"
    g.meta = {"npts": npts, "clusters": clusters, "sigma": sigma, "k": k, "seed": seed}
    if with_points:
        lib = _L()
        pts = np.zeros(3 * npts, dtype=np.float64)
        m = ctypes.c_uint64()
        po, pt, pw = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        rc = lib.graphgen_knn(npts, clusters, sigma, k, wscale, seed, ctypes.byref(m),
                              ctypes.byref(po), ctypes.byref(pt), ctypes.byref(pw), pts.ctypes.data)
        assert rc == 0
        for ptr in (po, pt, pw):
            lib.graphgen_free(ptr)
        return g, pts.reshape(npts, 3)
    return g
