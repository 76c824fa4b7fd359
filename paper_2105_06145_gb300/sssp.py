"""Python binding of libsssp.so (argument marshalling only).

Every function here has the name of the C-ABI call it wraps (include/sssp.h)
and does nothing but convert arguments: the solve itself runs in the CUDA
kernels of libsssp.so.  Device buffers and streams come from PyTorch
(``tensor.data_ptr()``, ``torch.cuda.current_stream().cuda_stream``); host
graph arrays are numpy.  Importing this module fails loudly when the library
has not been built: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SSSP_LIB may name another build of the same library (e.g. a variant for A/B timing)
LIB_PATH = os.environ.get("SSSP_LIB") or os.path.join(_HERE, "libsssp.so")

SSSP_RHO, SSSP_DELTA_STAR, SSSP_BELLMAN_FORD, SSSP_DELTA, SSSP_DIJKSTRA = 0, 1, 2, 3, 4
ALGOS = {"rho": SSSP_RHO, "delta_star": SSSP_DELTA_STAR, "bellman_ford": SSSP_BELLMAN_FORD,
         "delta": SSSP_DELTA, "dijkstra": SSSP_DIJKSTRA}
SSSP_SOLVE_BIDIRECTIONAL, SSSP_SOLVE_FUSED = 1, 2
SSSP_SHAPE_WIDE, SSSP_SHAPE_NARROW = 0, 1
SSSP_GRAPH_SYMMETRIC, SSSP_GRAPH_VERIFY, SSSP_GRAPH_REORDER = 1, 2, 4
SSSP_OK = 0
SSSP_ERR_INVALID_ARG, SSSP_ERR_OUT_OF_MEMORY, SSSP_ERR_CUDA = -1, -2, -3
SSSP_ERR_TIMEOUT, SSSP_ERR_INTERNAL = -4, -5
SSSP_MAX_BATCH = 2048  # instances per batched call
SSSP_RHO_REDUCED_NONE = 0xFFFFFFFF  # sssp_options.rho_reduced: plain rho on every step
SSSP_BATCH_AUTO, SSSP_BATCH_SHARED, SSSP_BATCH_SEPARATE = 0, 1, 2  # sssp_solve_sources_ex modes
INF = (1 << 64) - 1

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsssp.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                      "or python -m paper_2105_06145_gb300.build")

_lib = ctypes.CDLL(LIB_PATH)


class sssp_step_trace(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_uint64), ("queued", ctypes.c_uint32),
                ("extracted", ctypes.c_uint32), ("edges", ctypes.c_uint64),
                ("updates", ctypes.c_uint64), ("t_ns", ctypes.c_uint64),
                ("t_relax_ns", ctypes.c_uint64), ("t_extract_end_max", ctypes.c_uint64),
                ("t_relax_end_min", ctypes.c_uint64), ("t_relax_end_max", ctypes.c_uint64)]


TRACE_DTYPE = [("theta", "<u8"), ("queued", "<u4"), ("extracted", "<u4"), ("edges", "<u8"),
               ("updates", "<u8"), ("t_ns", "<u8"), ("t_relax_ns", "<u8"),
               ("t_extract_end_max", "<u8"), ("t_relax_end_min", "<u8"), ("t_relax_end_max", "<u8")]


class sssp_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_uint64), ("queued", ctypes.c_uint64),
                ("extracted", ctypes.c_uint64), ("edges", ctypes.c_uint64),
                ("updates", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("grid", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class sssp_options(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("timeout_ns", ctypes.c_uint64),
                ("max_steps", ctypes.c_uint64), ("ext_count", ctypes.c_void_p),
                ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_uint32),
                ("grid_limit", ctypes.c_uint32), ("test_exit_block", ctypes.c_uint32),
                ("stats_out", ctypes.c_void_p), ("solve_timeout_ns", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("local_budget", ctypes.c_uint32),
                ("shape", ctypes.c_uint32), ("rho_reduced", ctypes.c_uint32),
                ("small_deg", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("rho_warmup_steps", ctypes.c_uint32), ("rho_warmup", ctypes.c_uint32)]


TRACE_RECORD_BYTES = ctypes.sizeof(sssp_step_trace)
STATS_BYTES = ctypes.sizeof(sssp_stats)

_P, _u32, _u64, _i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
_lib.sssp_graph_create.argtypes = [_u32, _u64, _P, _P, _P, ctypes.POINTER(_P)]
_lib.sssp_graph_create.restype = _i32
_lib.sssp_graph_create_ex.argtypes = [_u32, _u64, _P, _P, _P, _u32, ctypes.POINTER(_P)]
_lib.sssp_graph_create_ex.restype = _i32
_lib.sssp_graph_destroy.argtypes = [_P]
_lib.sssp_graph_destroy.restype = _i32
_lib.sssp_graph_info.argtypes = [_P, ctypes.POINTER(_u32), ctypes.POINTER(_u64)]
_lib.sssp_graph_info.restype = _i32
_lib.sssp_solve.argtypes = [_P, _u32, _i32, _u64, _P, _P]
_lib.sssp_solve.restype = _i32
_lib.sssp_solve_ex.argtypes = [_P, _u32, _i32, _u64, _P, ctypes.POINTER(sssp_options), _P]
_lib.sssp_solve_ex.restype = _i32
_lib.sssp_solve_host.argtypes = [_P, _u32, _i32, _u64, _P, _P]
_lib.sssp_solve_host.restype = _i32
_lib.sssp_solve_host_ex.argtypes = [_P, _u32, _i32, _u64, _P, ctypes.POINTER(sssp_options), _P]
_lib.sssp_solve_host_ex.restype = _i32
_lib.sssp_last_status.argtypes = [_P, _P]
_lib.sssp_last_status.restype = _i32
_lib.sssp_last_stats.argtypes = [_P, ctypes.POINTER(sssp_stats), _P]
_lib.sssp_last_stats.restype = _i32
_lib.sssp_rho_threshold.argtypes = [_P, _u32, _P, _u32, _u64, _u64, _u64, _u32, _u32, _u32, _P, _P]
_lib.sssp_rho_threshold.restype = _i32
_lib.sssp_solve_noalloc.argtypes = [_u32, _u64, _P, _P, _u32, _i32, _u64, _P, _P, _P]
_lib.sssp_solve_noalloc.restype = _i32
_lib.sssp_solve_sources.argtypes = [_P, _P, _u32, _i32, _P, _P, _P]
_lib.sssp_solve_sources.restype = _i32
_lib.sssp_solve_sources_ex.argtypes = [_P, _P, _u32, _i32, _P, _u32, _P, _P]
_lib.sssp_solve_sources_ex.restype = _i32
_lib.sssp_solve_multi.argtypes = [_P, _P, _u32, _i32, _P, _P, _P]
_lib.sssp_solve_multi.restype = _i32
_lib.sssp_batch_last_stats.argtypes = [_P, _u32, _P]
_lib.sssp_batch_last_stats.restype = _i32
class sssp_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("algo", ctypes.c_int), ("param", ctypes.c_uint64),
                ("idle_ns", ctypes.c_uint64), ("hbm_fraction", ctypes.c_double), ("batch_mode", ctypes.c_uint32),
                ("gang", ctypes.c_uint32), ("gang_wait_ns", ctypes.c_uint64)]


class sssp_query_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps", ctypes.c_uint32), ("latency_ns", ctypes.c_uint64),
                ("device_ns", ctypes.c_uint64), ("device_admit_ns", ctypes.c_uint64),
                ("device_done_ns", ctypes.c_uint64), ("edges", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib.sssp_server_create.argtypes = [_P, ctypes.POINTER(sssp_server_config), ctypes.POINTER(_P)]
_lib.sssp_server_create.restype = _i32
_lib.sssp_server_slots.argtypes = [_P, ctypes.POINTER(_u32)]
_lib.sssp_server_slots.restype = _i32
_lib.sssp_server_mode.argtypes = [_P, ctypes.POINTER(_u32)]
_lib.sssp_server_mode.restype = _i32
_lib.sssp_server_submit.argtypes = [_P, _u32, _P, ctypes.POINTER(_u64)]
_lib.sssp_server_submit.restype = _i32
_lib.sssp_server_poll.argtypes = [_P, _u64, ctypes.POINTER(sssp_query_info)]
_lib.sssp_server_poll.restype = _i32
_lib.sssp_server_wait.argtypes = [_P, _u64, _u64, ctypes.POINTER(sssp_query_info)]
_lib.sssp_server_wait.restype = _i32
_lib.sssp_server_drain.argtypes = [_P, _P, _P, _u32]
_lib.sssp_server_drain.restype = _i32
_lib.sssp_server_stats.argtypes = [_P, ctypes.POINTER(_u64), ctypes.POINTER(_u32), ctypes.POINTER(_u64)]
_lib.sssp_server_stats.restype = _i32
_lib.sssp_server_destroy.argtypes = [_P]
_lib.sssp_server_destroy.restype = _i32
_lib.sssp_status_string.argtypes = [_i32]
_lib.sssp_status_string.restype = ctypes.c_char_p

EXPORTED = ["sssp_graph_create", "sssp_graph_destroy", "sssp_graph_info", "sssp_solve",
            "sssp_solve_ex", "sssp_solve_host", "sssp_last_status", "sssp_last_stats",
            "sssp_rho_threshold", "sssp_status_string", "sssp_solve_noalloc", "sssp_solve_sources",
            "sssp_solve_multi", "sssp_batch_last_stats", "sssp_server_create", "sssp_server_slots",
            "sssp_server_submit", "sssp_server_poll", "sssp_server_wait", "sssp_server_stats",
            "sssp_server_destroy", "sssp_server_drain", "sssp_graph_create_ex", "sssp_solve_host_ex",
            "sssp_autotune", "sssp_graph_get_tuning", "sssp_graph_set_tuning", "sssp_graph_class",
            "sssp_solve_tuned", "sssp_autotune_ex", "sssp_tourney_create", "sssp_tourney_destroy",
            "sssp_tourney_update", "sssp_tourney_extract", "sssp_tourney_min", "sssp_tourney_inq",
            "sssp_array_extract", "sssp_autotune_batch", "sssp_solve_sources_ex", "sssp_server_mode"]

_lib.sssp_tourney_create.argtypes = [_u32, ctypes.POINTER(_P)]
_lib.sssp_tourney_create.restype = _i32
_lib.sssp_tourney_destroy.argtypes = [_P]
_lib.sssp_tourney_destroy.restype = _i32
_lib.sssp_tourney_update.argtypes = [_P, _P, _u32, _P]
_lib.sssp_tourney_update.restype = _i32
_lib.sssp_tourney_extract.argtypes = [_P, _P, _u64, _P, _P, _P]
_lib.sssp_tourney_extract.restype = _i32
_lib.sssp_tourney_min.argtypes = [_P, _P, _P, _P]
_lib.sssp_tourney_min.restype = _i32
_lib.sssp_tourney_inq.argtypes = [_P, _P, _P]
_lib.sssp_tourney_inq.restype = _i32
_lib.sssp_array_extract.argtypes = [_P, _u32, _P, _u64, _P, _P, _P, _P, _P]
_lib.sssp_array_extract.restype = _i32


class sssp_tuning(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("shape", ctypes.c_uint32), ("param", ctypes.c_uint64),
                ("flags", ctypes.c_uint32), ("local_budget", ctypes.c_uint32), ("ms", ctypes.c_double),
                ("candidates", ctypes.c_uint32), ("slots", ctypes.c_uint32),
                ("rho_reduced", ctypes.c_uint32), ("small_deg", ctypes.c_uint32), ("chunk", ctypes.c_uint32),
                ("batch_mode", ctypes.c_uint32), ("rho_warmup_steps", ctypes.c_uint32),
                ("rho_warmup", ctypes.c_uint32)]

    def as_dict(self) -> dict:
        return {k: (float(getattr(self, k)) if k == "ms" else int(getattr(self, k))) for k, _ in self._fields_}


_lib.sssp_autotune.argtypes = [_P, _P, _u32, ctypes.POINTER(sssp_tuning), _P]
_lib.sssp_autotune.restype = _i32
_lib.sssp_autotune_batch.argtypes = [_P, _P, _u32, _u32, ctypes.POINTER(sssp_tuning), _P]
_lib.sssp_autotune_batch.restype = _i32
_lib.sssp_autotune_ex.argtypes = [_P, _P, _u32, _u32, ctypes.POINTER(sssp_tuning), _P]
_lib.sssp_autotune_ex.restype = _i32
_lib.sssp_graph_get_tuning.argtypes = [_P, ctypes.POINTER(sssp_tuning)]
_lib.sssp_graph_get_tuning.restype = _i32
_lib.sssp_graph_set_tuning.argtypes = [_P, ctypes.POINTER(sssp_tuning)]
_lib.sssp_graph_set_tuning.restype = _i32
_lib.sssp_graph_class.argtypes = [_P, ctypes.POINTER(_u64)]
_lib.sssp_graph_class.restype = _i32
_lib.sssp_solve_tuned.argtypes = [_P, _u32, _P, _P]
_lib.sssp_solve_tuned.restype = _i32

MAX_BATCH = 2048

NOALLOC_MAX_VERTICES = 1 << 18
NOALLOC_MAX_EDGES = 1 << 22


class SSSPError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {sssp_status_string(code)} ({code})")
        self.code = code


def _check(code: int, what: str) -> int:
    if code != SSSP_OK:
        raise SSSPError(code, what)
    return code


def sssp_status_string(code: int) -> str:
    return _lib.sssp_status_string(code).decode()


def sssp_graph_create(n: int, m: int, offsets: np.ndarray, targets: np.ndarray,
                      weights: np.ndarray) -> int:
    return sssp_graph_create_ex(n, m, offsets, targets, weights, 0)


def sssp_graph_create_ex(n: int, m: int, offsets: np.ndarray, targets: np.ndarray,
                         weights: np.ndarray, flags: int) -> int:
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    targets = np.ascontiguousarray(targets, dtype=np.uint32)
    weights = np.ascontiguousarray(weights, dtype=np.uint32)
    h = _P()
    _check(_lib.sssp_graph_create_ex(n, m, offsets.ctypes.data, targets.ctypes.data if m else None,
                                     weights.ctypes.data if m else None, flags, ctypes.byref(h)),
           "sssp_graph_create_ex")
    return h.value


def sssp_graph_destroy(g: int) -> None:
    _check(_lib.sssp_graph_destroy(g), "sssp_graph_destroy")


def sssp_graph_info(g: int) -> tuple[int, int]:
    n, m = _u32(), _u64()
    _check(_lib.sssp_graph_info(g, ctypes.byref(n), ctypes.byref(m)), "sssp_graph_info")
    return n.value, m.value


def sssp_solve(g: int, source: int, algo: int, param: int, dist_out_ptr: int, stream: int = 0) -> int:
    """Enqueue a solve; dist_out_ptr is a device pointer to uint64[n]."""
    return _check(_lib.sssp_solve(g, source, algo, param, dist_out_ptr, stream or None), "sssp_solve")


def make_options(seed: int = 0, timeout_ns: int = 0, max_steps: int = 0, ext_count_ptr: int = 0,
                 trace_ptr: int = 0, trace_cap: int = 0, grid_limit: int = 0,
                 test_exit_block: int = 0, stats_out_ptr: int = 0,
                 solve_timeout_ns: int = 0, flags: int = 0, local_budget: int = 0,
                 shape: int = 0, rho_reduced: int = 0, small_deg: int = 0, chunk: int = 0,
                 rho_warmup_steps: int = 0, rho_warmup: int = 0) -> sssp_options:
    o = sssp_options()
    o.seed, o.timeout_ns, o.max_steps = seed, timeout_ns, max_steps
    o.ext_count = ext_count_ptr or None
    o.trace = trace_ptr or None
    o.trace_cap, o.grid_limit, o.test_exit_block = trace_cap, grid_limit, test_exit_block
    o.stats_out = stats_out_ptr or None
    o.solve_timeout_ns = solve_timeout_ns
    o.flags = flags
    o.local_budget = local_budget
    o.shape = shape
    o.rho_reduced, o.small_deg, o.chunk = rho_reduced, small_deg, chunk
    o.rho_warmup_steps, o.rho_warmup = rho_warmup_steps, rho_warmup
    return o


def sssp_solve_ex(g: int, source: int, algo: int, param: int, dist_out_ptr: int,
                  opts: sssp_options | None = None, stream: int = 0, check: bool = True) -> int:
    rc = _lib.sssp_solve_ex(g, source, algo, param, dist_out_ptr,
                            ctypes.byref(opts) if opts is not None else None, stream or None)
    return _check(rc, "sssp_solve_ex") if check else rc


def sssp_solve_host(g: int, source: int, algo: int, param: int, host_out: np.ndarray,
                    stream: int = 0, check: bool = True) -> int:
    assert host_out.dtype == np.uint64 and host_out.flags.c_contiguous
    rc = _lib.sssp_solve_host(g, source, algo, param, host_out.ctypes.data, stream or None)
    return _check(rc, "sssp_solve_host") if check else rc


def sssp_solve_host_ptr(g: int, source: int, algo: int, param: int, host_ptr: int,
                        stream: int = 0, opts: sssp_options | None = None) -> int:
    """sssp_solve_host_ex with a raw host pointer (e.g. a pinned torch tensor)."""
    return _lib.sssp_solve_host_ex(g, source, algo, param, host_ptr,
                                   ctypes.byref(opts) if opts is not None else None, stream or None)


def sssp_last_status(g: int, stream: int = 0) -> int:
    return int(_lib.sssp_last_status(g, stream or None))


def sssp_last_stats(g: int, stream: int = 0) -> dict:
    s = sssp_stats()
    _check(_lib.sssp_last_stats(g, ctypes.byref(s), stream or None), "sssp_last_stats")
    return s.as_dict()


def sssp_rho_threshold(queue_ptr: int, q: int, dist_ptr: int, n: int, rho: int, seed: int,
                       step: int, dense_before: int, reduced: int, theta_out_ptr: int, stream: int = 0,
                       max_samples: int = 0) -> int:
    return _check(_lib.sssp_rho_threshold(queue_ptr or None, q, dist_ptr, n, rho, seed, step,
                                          dense_before, reduced, max_samples, theta_out_ptr, stream or None),
                  "sssp_rho_threshold")


def sssp_solve_noalloc(n: int, m: int, offsets_ptr: int, edges_ptr: int, source: int, algo: int,
                       param: int, dist_out_ptr: int, stats_out_ptr: int = 0, stream: int = 0,
                       check: bool = True) -> int:
    """All pointers are device pointers; see include/sssp.h (no allocation)."""
    rc = _lib.sssp_solve_noalloc(n, m, offsets_ptr or None, edges_ptr or None, source, algo, param,
                                 dist_out_ptr or None, stats_out_ptr or None, stream or None)
    return _check(rc, "sssp_solve_noalloc") if check else rc


def sssp_solve_sources(g: int, sources, algo: int, params, dist_out_ptr: int, stream: int = 0,
                       check: bool = True) -> int:
    """k sources on one graph; dist_out_ptr: device uint64[k*n] (instance-major)."""
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    prm = None if params is None else np.ascontiguousarray(params, dtype=np.uint64)
    rc = _lib.sssp_solve_sources(g, src.ctypes.data, src.size, algo,
                                 prm.ctypes.data if prm is not None else None, dist_out_ptr, stream or None)
    return _check(rc, "sssp_solve_sources") if check else rc


def sssp_solve_sources_ex(g: int, sources, algo: int, params, mode: int, dist_out_ptr: int, stream: int = 0,
                          check: bool = True) -> int:
    """sssp_solve_sources with an SSSP_BATCH_* mode (shared edge scan or separate instances)."""
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    prm = None if params is None else np.ascontiguousarray(params, dtype=np.uint64)
    rc = _lib.sssp_solve_sources_ex(g, src.ctypes.data, src.size, algo,
                                    prm.ctypes.data if prm is not None else None, mode, dist_out_ptr,
                                    stream or None)
    return _check(rc, "sssp_solve_sources_ex") if check else rc


def sssp_solve_multi(graphs, sources, algo: int, params, dist_out_ptrs, stream: int = 0,
                     check: bool = True) -> int:
    """One source per graph; graphs: sequence of handles; dist_out_ptrs: device pointers."""
    k = len(graphs)
    gs = (ctypes.c_void_p * k)(*graphs)
    outs = (ctypes.c_void_p * k)(*dist_out_ptrs)
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    prm = None if params is None else np.ascontiguousarray(params, dtype=np.uint64)
    rc = _lib.sssp_solve_multi(gs, src.ctypes.data, k, algo, prm.ctypes.data if prm is not None else None,
                               outs, stream or None)
    return _check(rc, "sssp_solve_multi") if check else rc


def sssp_batch_last_stats(k: int, stream: int = 0) -> tuple[int, list]:
    """(device status, per-instance stats dicts) of the last batched call."""
    arr = (sssp_stats * max(k, 1))()
    rc = _lib.sssp_batch_last_stats(arr, k, stream or None)
    if rc < 0 and rc not in (SSSP_ERR_TIMEOUT, SSSP_ERR_INTERNAL):
        raise SSSPError(rc, "sssp_batch_last_stats")
    return rc, [arr[i].as_dict() for i in range(k)]


def sssp_server_create(g: int, slots: int = 0, algo: int = SSSP_RHO, param: int = 0, idle_ns: int = 0,
                       hbm_fraction: float = 0.0, batch_mode: int = SSSP_BATCH_AUTO, gang: int = 0,
                       gang_wait_ns: int = 0) -> int:
    cfg = sssp_server_config(slots, algo, param, idle_ns, hbm_fraction, batch_mode, gang, gang_wait_ns)
    h = _P()
    _check(_lib.sssp_server_create(g, ctypes.byref(cfg), ctypes.byref(h)), "sssp_server_create")
    return h.value


def sssp_server_slots(s: int) -> int:
    v = _u32()
    _check(_lib.sssp_server_slots(s, ctypes.byref(v)), "sssp_server_slots")
    return v.value


def sssp_server_mode(s: int) -> int:
    """SSSP_BATCH_SHARED or SSSP_BATCH_SEPARATE: how the server runs its slots."""
    v = _u32()
    _check(_lib.sssp_server_mode(s, ctypes.byref(v)), "sssp_server_mode")
    return v.value


def sssp_server_submit(s: int, source: int, dist_out_ptr: int) -> int:
    t = _u64()
    _check(_lib.sssp_server_submit(s, source, dist_out_ptr, ctypes.byref(t)), "sssp_server_submit")
    return t.value


def sssp_server_poll(s: int, ticket: int):
    """None while pending, else the query info dict."""
    info = sssp_query_info()
    rc = _lib.sssp_server_poll(s, ticket, ctypes.byref(info))
    if rc < 0:
        raise SSSPError(rc, "sssp_server_poll")
    return info.as_dict() if rc == 1 else None


def sssp_server_wait(s: int, ticket: int, timeout_ns: int = 0) -> dict:
    info = sssp_query_info()
    rc = _lib.sssp_server_wait(s, ticket, timeout_ns, ctypes.byref(info))
    if rc != 1:
        raise SSSPError(rc, "sssp_server_wait")
    return info.as_dict()


def sssp_server_drain(s: int, max_items: int = 1024) -> list:
    """[(ticket, info dict)] of queries completed since the last drain."""
    tk = (ctypes.c_uint64 * max_items)()
    inf = (sssp_query_info * max_items)()
    rc = _lib.sssp_server_drain(s, tk, inf, max_items)
    if rc < 0:
        raise SSSPError(rc, "sssp_server_drain")
    return [(int(tk[i]), inf[i].as_dict()) for i in range(rc)]


def sssp_server_stats(s: int) -> dict:
    a, b, c = _u64(), _u32(), _u64()
    _check(_lib.sssp_server_stats(s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "sssp_server_stats")
    return {"launches": a.value, "busy_slots": b.value, "pending": c.value}


def sssp_server_destroy(s: int) -> None:
    _check(_lib.sssp_server_destroy(s), "sssp_server_destroy")


def sssp_autotune(g: int, sources, stream: int = 0) -> dict:
    """Time candidate configurations on the sample sources; returns the choice."""
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    t = sssp_tuning()
    _check(_lib.sssp_autotune(g, src.ctypes.data, src.size, ctypes.byref(t), stream or None), "sssp_autotune")
    return t.as_dict()


def sssp_autotune_ex(g: int, sources, rules: int, stream: int = 0) -> dict:
    """sssp_autotune restricted to the rules in the bit mask (1 << SSSP_RHO, 1 << SSSP_DELTA_STAR)."""
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    t = sssp_tuning()
    _check(_lib.sssp_autotune_ex(g, src.ctypes.data, src.size, rules, ctypes.byref(t), stream or None),
           "sssp_autotune_ex")
    return t.as_dict()


def sssp_autotune_batch(g: int, sources, rules: int, stream: int = 0) -> dict:
    """Best configuration of batched launches of these sources (stored as the graph's batch tuning)."""
    src = np.ascontiguousarray(sources, dtype=np.uint32)
    t = sssp_tuning()
    _check(_lib.sssp_autotune_batch(g, src.ctypes.data, src.size, rules, ctypes.byref(t), stream or None),
           "sssp_autotune_batch")
    return t.as_dict()


def sssp_graph_get_tuning(g: int):
    t = sssp_tuning()
    rc = _lib.sssp_graph_get_tuning(g, ctypes.byref(t))
    return t.as_dict() if rc == SSSP_OK else None


def sssp_graph_set_tuning(g: int, tuning: dict) -> None:
    t = sssp_tuning()
    for k, v in tuning.items():
        setattr(t, k, v)
    _check(_lib.sssp_graph_set_tuning(g, ctypes.byref(t)), "sssp_graph_set_tuning")


def sssp_graph_class(g: int) -> int:
    key = ctypes.c_uint64()
    _check(_lib.sssp_graph_class(g, ctypes.byref(key)), "sssp_graph_class")
    return int(key.value)


def sssp_solve_tuned(g: int, source: int, dist_out_ptr: int, stream: int = 0) -> int:
    return _check(_lib.sssp_solve_tuned(g, source, dist_out_ptr, stream or None), "sssp_solve_tuned")


def sssp_tourney_create(n: int) -> int:
    h = _P()
    _check(_lib.sssp_tourney_create(n, ctypes.byref(h)), "sssp_tourney_create")
    return h.value


def sssp_tourney_destroy(t: int) -> None:
    _check(_lib.sssp_tourney_destroy(t), "sssp_tourney_destroy")


def sssp_tourney_update(t: int, ids_ptr: int, b: int, stream: int = 0) -> None:
    _check(_lib.sssp_tourney_update(t, ids_ptr or None, b, stream or None), "sssp_tourney_update")


def sssp_tourney_extract(t: int, keys_ptr: int, theta: int, out_ptr: int, count_ptr: int, stream: int = 0) -> None:
    _check(_lib.sssp_tourney_extract(t, keys_ptr, theta, out_ptr, count_ptr, stream or None), "sssp_tourney_extract")


def sssp_tourney_min(t: int, keys_ptr: int, min_ptr: int, stream: int = 0) -> None:
    _check(_lib.sssp_tourney_min(t, keys_ptr, min_ptr, stream or None), "sssp_tourney_min")


def sssp_tourney_inq(t: int, inq_ptr: int, stream: int = 0) -> None:
    _check(_lib.sssp_tourney_inq(t, inq_ptr, stream or None), "sssp_tourney_inq")


def sssp_array_extract(list_ptr: int, q: int, keys_ptr: int, theta: int, ext_ptr: int, ext_count_ptr: int,
                       keep_ptr: int, keep_count_ptr: int, stream: int = 0) -> None:
    _check(_lib.sssp_array_extract(list_ptr or None, q, keys_ptr, theta, ext_ptr, ext_count_ptr, keep_ptr,
                                   keep_count_ptr, stream or None), "sssp_array_extract")


class Graph:
    """Owning wrapper of an sssp_graph handle built from a CSR (graphgen.CSR or
    any object with n, off, tgt, w)."""

    def __init__(self, csr, flags: int = 0):
        self.n = int(csr.n)
        self.m = int(csr.tgt.shape[0])
        self.handle = sssp_graph_create_ex(self.n, self.m, csr.off, csr.tgt, csr.w, flags)

    def close(self) -> None:
        if self.handle:
            sssp_graph_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, source: int, algo: int, param: int, dist_out, stream: int = 0,
              opts: sssp_options | None = None) -> None:
        """dist_out: a CUDA tensor with n 8-byte elements (int64 or uint64)."""
        assert dist_out.is_cuda and dist_out.numel() == self.n and dist_out.element_size() == 8
        sssp_solve_ex(self.handle, source, algo, param, dist_out.data_ptr(), opts, stream)

    def status(self, stream: int = 0) -> int:
        return sssp_last_status(self.handle, stream)

    def stats(self, stream: int = 0) -> dict:
        return sssp_last_stats(self.handle, stream)
