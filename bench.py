#!/usr/bin/env python
"""Benchmark: exact SSSP throughput (GTEPS) of the stepping solver on one GB300.

Workload (default): RMAT scale 22, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
symmetrised, no self-loops or duplicates, weights uniform in [1, 2^18) -- the
power-law stand-in for the paper's social graphs -- solved by rho-Stepping.
One "step" is one complete solve (init + every ExtDist / Extract / relax step
until the queue is empty) from one source; sources cycle over 10 vertices drawn
uniformly from the largest connected component.  GTEPS = m / solve time
(m = directed edges of the graph), aggregated as K*m / total time.

Each rank solves its own sources on its own graph replica (the single solve
does not shard; multi-GPU runs are independent replicas).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (binary-heap Dijkstra, one host core)
on the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SSSP GTEPS and % HBM roofline on 1 GB300; batched queries/s and p50/p99 latency vs plain"
ALGO_NAMES = {0: "rho", 1: "delta_star", 2: "bellman_ford", 3: "delta", 4: "dijkstra"}

# Algorithmic bytes per unit of work of one solve, from its device counters
# (what the method itself must move per queued id, extracted vertex, scanned
# edge and successful update):
BYTES_PER_QUEUED = 16     # Extract filter: 4 B id + 8 B delta + 4 B re-append / F write
BYTES_PER_EXTRACTED = 32  # 16 B offsets + 8 B delta[u] + 4 B F write + 4 B F read
BYTES_PER_EDGE = 16       # 8 B packed (target, weight) + 8 B delta[v]
BYTES_PER_UPDATE = 8      # 4 B queue-bit test-and-set + 4 B queue append


def algorithmic_bytes(st: dict) -> int:
    return (BYTES_PER_QUEUED * st["queued"] + BYTES_PER_EXTRACTED * st["extracted"] +
            BYTES_PER_EDGE * st["edges"] + BYTES_PER_UPDATE * st["updates"])


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("paper_2105_06145_gb300/csrc/sssp_kernels.cu", "paper_2105_06145_gb300/csrc/sssp_internal.h",
              "paper_2105_06145_gb300/csrc/sssp_device.cuh"):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic():
    """(bytes, edges) of the committed ncu DRAM capture of solve_kernel, if it
    was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "solve_kernel_rmat22_rho2e18_dram.md")
    try:
        for line in open(path):
            if line.startswith("traffic:"):
                kv = dict(x.split("=") for x in line.split()[1:])
                if kv.get("kernel_sha256_16") == kernel_hash():
                    return int(kv["bytes"]), int(kv["edges"])
    except OSError:
        pass
    return None


def load_peaks() -> tuple[float, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks / throttle reasons while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def build_workload(name: str, scale: int):
    from paper_2105_06145_gb300 import graphgen as gg
    if name == "rmat":
        g = gg.rmat(scale, 16, 0.57, 0.19, 0.19, gen_seed=2, wseed=3)
        srcs = gg.pick_sources(g, 10, 4)
        label = f"rmat{scale}_ef16"
    elif name == "road":
        g, s0 = gg.workload_road(4096 if scale == 22 else (1 << (scale // 2)))
        srcs = [s0] + gg.pick_sources(g, 9, 6)
        label = f"road{int(round(g.n ** 0.5))}"
    elif name == "grid":
        g, s0 = gg.workload_grid256()
        srcs = [s0] + gg.pick_sources(g, 9, 6)
        label = "grid256"
    else:
        raise SystemExit(f"unknown workload {name}")
    return g, srcs, label


def rank_sources(srcs: list, rank: int) -> list:
    """Each rank cycles through the workload's sources starting at its own offset
    (replicas solve different sources; no data-path collective)."""
    nsrc = len(srcs)
    return [srcs[(i + rank) % nsrc] for i in range(nsrc)]


def aggregate(total_ms: float, K: int, m: int, world: int, pg=None, device="cuda") -> tuple[float, float]:
    """Whole-job GTEPS over all ranks: every rank solved K sources of an m-edge
    graph; the time is the maximum over ranks.  Returns (gteps, max_ms)."""
    if pg is not None and world > 1:
        import torch
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * K * m / (total_ms * 1e-3) / 1e9, total_ms


def gg_sources(g, k=256, seed=9):
    from paper_2105_06145_gb300 import graphgen as gg
    return gg.pick_sources(g, k, seed)


def run_reference(args, g, srcs, label, rank, world):
    """CPU oracle (binary-heap Dijkstra, one core) timed on the same metric."""
    import oracle
    if rank != 0:
        return
    for i in range(args.warmup):
        oracle.dijkstra(g, srcs[i % len(srcs)])
    times = []
    for i in range(args.steps):
        t0 = time.perf_counter()
        oracle.dijkstra(g, srcs[i % len(srcs)])
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    gteps = args.steps * g.m / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gteps, "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": label, "n": g.n, "m": g.m, "algo": "dijkstra (CPU oracle)"},
        "cpu_baseline": {"value": gteps, "unit": "GTEPS", "cores": 1, "cpu_model": cpu_model(), "kind": "oracle",
                         "sample": f"{args.steps} full single-source solves of {label}"},
        "e2e": {"value": gteps, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _timed(torch, stream_obj, fn) -> float:
    """ms of one call of fn (after one untimed call), CUDA events on the stream."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream_obj):
        fn()
        torch.cuda.synchronize()
        e0.record(stream_obj)
        fn()
        e1.record(stream_obj)
        torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def rows_equal_to_single(torch, stream_obj, rows, sources, solve_one) -> int:
    """How many rows[i] (a batched or served result) equal the single solve of
    sources[i] (solve_one(source, out_tensor) enqueues it); run after the
    timed region."""
    one = torch.empty_like(rows[0])
    eq = 0
    with torch.cuda.stream(stream_obj):
        for i, s_ in enumerate(sources):
            solve_one(int(s_), one)
            torch.cuda.synchronize()
            eq += int(bool(torch.equal(rows[i], one)))
    return eq


class _View:
    """A CSR over arrays in shared memory (what the oracle reads: n, off, tgt, w)."""

    def __init__(self, n, off, tgt, w):
        self.n, self.off, self.tgt, self.w = n, off, tgt, w


def _oracle_worker(job):
    """Parallel oracle baseline, one worker: binary-heap Dijkstra for each of its
    (graph, source) tasks, graphs read from shared memory.  job = (names,
    tasks); tasks = [(n, m, off_base, edge_base, source), ...].  Returns the
    XOR of each solve's distance array, one per task (a job with no tasks
    only attaches: pool warm-up)."""
    from multiprocessing import shared_memory
    import oracle
    names, tasks = job
    shm = [shared_memory.SharedMemory(name=x) for x in names]
    OFF = np.ndarray((shm[0].size // 8,), np.uint64, buffer=shm[0].buf)
    TGT = np.ndarray((shm[1].size // 4,), np.uint32, buffer=shm[1].buf)
    WW = np.ndarray((shm[2].size // 4,), np.uint32, buffer=shm[2].buf)
    digests = []
    for n, m, ob, eb, src in tasks:
        d = oracle.dijkstra(_View(n, OFF[ob:ob + n + 1], TGT[eb:eb + m], WW[eb:eb + m]), src)
        digests.append(int(np.bitwise_xor.reduce(d)))
    del OFF, TGT, WW
    for x in shm:
        x.close()
    return digests


def oracle_parallel(graphs_sources, with_digests: bool = False) -> dict:
    """Throughput of P independent oracle solves on all P host cores (spawned
    workers, graphs shared read-only): queries/s over the wall time of the
    solves alone (pool start and attach are outside the timed region).
    with_digests: also return each task's distance XOR, in task order."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    from multiprocessing import shared_memory
    P = os.cpu_count() or 1
    graphs = {}
    for h, _ in graphs_sources:
        graphs.setdefault(id(h), h)
    offs, tgts, ws, base = [], [], [], {}
    ob = eb = 0
    for key, h in graphs.items():
        base[key] = (ob, eb)
        offs.append(np.asarray(h.off, np.uint64)); tgts.append(np.asarray(h.tgt, np.uint32))
        ws.append(np.asarray(h.w, np.uint32))
        ob += h.n + 1
        eb += h.m
    arrays = [np.concatenate(offs), np.concatenate(tgts) if eb else np.zeros(1, np.uint32),
              np.concatenate(ws) if eb else np.zeros(1, np.uint32)]
    shm = []
    try:
        for a in arrays:
            x = shared_memory.SharedMemory(create=True, size=max(8, a.nbytes))
            np.ndarray(a.shape, a.dtype, buffer=x.buf)[:] = a
            shm.append(x)
        names = [x.name for x in shm]
        tasks = [(h.n, h.m, base[id(h)][0], base[id(h)][1], int(s_)) for h, s_ in graphs_sources]
        jobs = [(names, tasks[i::P]) for i in range(P)]
        # an executor (not a Pool): a worker that dies fails the call instead
        # of being replaced forever
        with ProcessPoolExecutor(max_workers=P, mp_context=mp.get_context("spawn")) as ex:
            for f in [ex.submit(_oracle_worker, (names, [])) for _ in range(P)]:
                f.result(timeout=300)
            t0 = time.perf_counter()
            parts = [f.result(timeout=600) for f in [ex.submit(_oracle_worker, j) for j in jobs]]
            dt = time.perf_counter() - t0
        done = sum(len(x) for x in parts)
        digests = [0] * len(tasks)
        for i, part in enumerate(parts):  # job i ran tasks i, i+P, i+2P, ...
            for j, dg in enumerate(part):
                digests[i + j * P] = dg
    finally:
        for x in shm:
            x.close()
            x.unlink()
    out = {"value": done / dt, "unit": "queries/s", "cores": P, "cpu_model": cpu_model(), "kind": "oracle",
           "sample": f"{done} binary-heap Dijkstra solves over {len(graphs)} graph(s), "
                     f"{P} spawned workers ({dt:.1f} s)"}
    if with_digests:
        out["digests"] = digests
    return out


def measure_batched(sssp, G, g, torch, stream, stream_obj, cpu: bool = False) -> dict:
    """Batched solves: (a) 64 sources on this graph in one launch, (b) 512 graphs of
    uneven size in one launch with per-instance rho from the autotuner (one tuning
    per graph class); each against the plain loop of single solves, each plain
    solve in its own tuned configuration (sssp_solve_tuned)."""
    from paper_2105_06145_gb300 import graphgen as gg
    res = {}
    srcs = gg.pick_sources(g, 64, 6)
    tune = sssp.sssp_autotune_ex(G.handle, srcs[:3], 1 << sssp.SSSP_RHO, stream)
    out = torch.empty(64 * g.n, dtype=torch.int64, device="cuda")
    one = torch.empty(g.n, dtype=torch.int64, device="cuda")
    tb = _timed(torch, stream_obj, lambda: sssp.sssp_solve_sources(G.handle, srcs, sssp.SSSP_RHO, None,
                                                                   out.data_ptr(), stream))
    st, _ = sssp.sssp_batch_last_stats(64, stream)
    tp = _timed(torch, stream_obj, lambda: [sssp.sssp_solve_tuned(G.handle, s_, one.data_ptr(), stream)
                                            for s_ in srcs])
    eq = rows_equal_to_single(torch, stream_obj, out.view(64, g.n), srcs,
                              lambda s_, o: sssp.sssp_solve_tuned(G.handle, s_, o.data_ptr(), stream))
    res["sources64_rmat22"] = {"queries_per_s": 64e3 / tb, "plain_queries_per_s": 64e3 / tp,
                               "speedup": tp / tb, "status": st, "all_equal": eq == 64,
                               "instances_equal_to_single": eq, "tuning": tune}
    del out, one
    W = gg.workload_multi()
    Gs = [sssp.Graph(h, sssp.SSSP_GRAPH_SYMMETRIC) for h, _ in W]
    outs = [torch.empty(h.n, dtype=torch.int64, device="cuda") for h, _ in W]
    classes = {}
    for (h, s_), Gx in zip(W, Gs):
        key = sssp.sssp_graph_class(Gx.handle)
        if key not in classes:
            more = gg.pick_sources(h, 1, 11)
            classes[key] = sssp.sssp_autotune_ex(Gx.handle, [s_] + more, 1 << sssp.SSSP_RHO, stream)
    hs, ss, ptrs = [x.handle for x in Gs], [s_ for _, s_ in W], [o.data_ptr() for o in outs]
    tb = _timed(torch, stream_obj, lambda: sssp.sssp_solve_multi(hs, ss, sssp.SSSP_RHO, None, ptrs, stream))
    st, _ = sssp.sssp_batch_last_stats(len(W), stream)
    keep = [o.clone() for o in outs]
    tp = _timed(torch, stream_obj, lambda: [sssp.sssp_solve_tuned(Gx.handle, s_, o.data_ptr(), stream)
                                            for (h, s_), Gx, o in zip(W, Gs, outs)])
    torch.cuda.synchronize()
    eq = sum(int(bool(torch.equal(a, b))) for a, b in zip(keep, outs))
    del keep
    res["graphs512"] = {"queries_per_s": len(W) * 1e3 / tb, "plain_queries_per_s": len(W) * 1e3 / tp,
                        "speedup": tp / tb, "status": st, "edges_total": int(sum(h.m for h, _ in W)),
                        "graph_classes_tuned": len(classes), "all_equal": eq == len(W),
                        "instances_equal_to_single": eq}
    for Gx in Gs:
        Gx.close()
    if cpu:
        # the oracle on every host core: 2 sources per core on the RMAT-22 graph,
        # and all 512 graphs
        P = os.cpu_count() or 1
        res["sources64_rmat22"]["cpu_baseline"] = oracle_parallel([(g, s_) for s_ in (srcs * 64)[:2 * P]])
        res["graphs512"]["cpu_baseline"] = oracle_parallel(W)
    return res


def measure_workload(name, sssp, torch, stream, stream_obj, rates_x=(2, 20), cpu: bool = False) -> dict:
    """Road-like (4096^2 jittered grid) or k-NN (2M points) workload: the
    autotuner's single-solve choice as a plain loop of single solves; 64
    sources in one batched launch and the continuous-batching server, both in
    the batch autotuner's choice, at offered rates of rates_x times the plain
    loop's rate."""
    from paper_2105_06145_gb300 import graphgen as gg
    if name == "road4096":
        h, _ = gg.workload_road(4096)
        srcs = gg.pick_sources(h, 256, 9, mask=gg.largest_cc(h))
    else:
        h = gg.knn(2_000_000, 64, 0.02, 10, float(1 << 20), seed=10)
        srcs = gg.pick_sources(h, 256, 9, mask=np.ones(h.n, np.uint8))
    Gx = sssp.Graph(h, sssp.SSSP_GRAPH_SYMMETRIC)
    one = torch.empty(h.n, dtype=torch.int64, device="cuda")
    # the best configuration of each rule alone (rho-Stepping, Delta*-Stepping)
    per_rule = {}
    for rname, rule in (("rho", sssp.SSSP_RHO), ("delta_star", sssp.SSSP_DELTA_STAR)):
        tr = sssp.sssp_autotune_ex(Gx.handle, srcs[:3], 1 << rule, stream)
        tq = _timed(torch, stream_obj, lambda: [sssp.sssp_solve_tuned(Gx.handle, s_, one.data_ptr(), stream)
                                                for s_ in srcs[:10]])
        per_rule[rname] = {"tuning": tr, "ms_per_solve": tq / 10, "gteps": 10 * h.m / (tq * 1e-3) / 1e9}
    t0 = time.perf_counter()
    tune = sssp.sssp_autotune(Gx.handle, srcs[:3], stream)
    tune_s = time.perf_counter() - t0
    tp = _timed(torch, stream_obj, lambda: [sssp.sssp_solve_tuned(Gx.handle, s_, one.data_ptr(), stream)
                                            for s_ in srcs[:10]])
    plain_qps = 10e3 / tp
    t0 = time.perf_counter()
    btune = sssp.sssp_autotune_batch(Gx.handle, srcs[:64], (1 << sssp.SSSP_RHO) | (1 << sssp.SSSP_DELTA_STAR),
                                     stream)
    btune_s = time.perf_counter() - t0
    torch.cuda.empty_cache()
    out = torch.empty(64 * h.n, dtype=torch.int64, device="cuda")
    tb = _timed(torch, stream_obj, lambda: sssp.sssp_solve_sources(Gx.handle, srcs[:64], btune["algo"], None,
                                                                   out.data_ptr(), stream))
    st, _ = sssp.sssp_batch_last_stats(64, stream)
    eq = rows_equal_to_single(torch, stream_obj, out.view(64, h.n), srcs[:64],
                              lambda s_, o: sssp.sssp_solve_tuned(Gx.handle, s_, o.data_ptr(), stream))
    del out
    torch.cuda.empty_cache()
    res = {"n": h.n, "m": h.m, "tuning": tune, "tune_s": tune_s, "batch_tuning": btune, "batch_tune_s": btune_s,
           "plain": {"queries_per_s": plain_qps, "gteps": plain_qps * h.m / 1e9}, "per_rule": per_rule,
           "batched64": {"queries_per_s": 64e3 / tb, "speedup": tp / 10 * 64 / tb, "status": st,
                         "all_equal": eq == 64, "instances_equal_to_single": eq}}
    rates = [int(max(1, round(x * plain_qps))) for x in rates_x]
    sv = measure_serving(sssp, Gx, h, torch, srcs, rates, window_s=1.0, hard_s=8.0, slots=0,
                         algo=btune["algo"], param=btune["param"], tuned=True)
    res["served"] = sv
    Gx.close()
    del Gx
    torch.cuda.empty_cache()
    if cpu:  # the oracle on every host core, 2 sources per core
        res["cpu_baseline"] = oracle_parallel([(h, s_) for s_ in srcs[:2 * (os.cpu_count() or 1)]])
    return res


def measure_serving(sssp, G, g, torch, sources, rates, window_s=1.0, hard_s=10.0, slots=0,
                    algo=None, param=0, seed=8, tuned=False, gang=0, gang_wait_ns=0) -> dict:
    """Serving: a Poisson query stream at each offered rate
    for `window_s` seconds against the resident graph; queries go to the
    continuous-batching server as client-side result buffers allow.  Latency
    is from the scheduled arrival to the completion seen by the client; the
    plain loop (one sssp_solve at a time) is measured on the same sources.
    Every rate keeps a sample of its served results (the first completions and
    every 8th after them, their buffers held back from reuse) and compares each
    with the single solve of its source after the window (`checked`,
    `all_equal`)."""
    algo = sssp.SSSP_RHO if algo is None else algo
    srv = sssp.sssp_server_create(G.handle, slots=slots, algo=algo, param=param, gang=gang, gang_wait_ns=gang_wait_ns)
    S = sssp.sssp_server_slots(srv)
    # enough client buffers that a full cohort of S queries can wait while S
    # run (a shared-scan server admits queries in cohorts of S)
    nbuf = 2 * S + 32
    free_b, _ = torch.cuda.mem_get_info()
    nbuf = int(max(1, min(nbuf, (free_b * 0.8) // (8 * g.n))))
    bufs = [torch.empty(g.n, dtype=torch.int64, device="cuda") for _ in range(nbuf)]
    torch.cuda.synchronize()
    # plain loop: one query at a time, result synchronised
    stream = torch.cuda.current_stream().cuda_stream
    prm = param or (max(64, g.n // 16) if algo == sssp.SSSP_RHO else 0)

    def plain_one(s_):
        if tuned:  # the graph's tuned configuration (shape, flags, local relaxation)
            sssp.sssp_solve_tuned(G.handle, s_, bufs[0].data_ptr(), stream)
        else:
            G.solve(s_, algo, prm, bufs[0], stream)
        torch.cuda.synchronize()

    plain_one(sources[0])
    t0 = time.perf_counter()
    nplain = min(10, len(sources))
    for s_ in sources[:nplain]:
        plain_one(s_)
    plain_qps = nplain / (time.perf_counter() - t0)
    rng = np.random.default_rng(seed)
    out = {"slots": S, "mode": "shared" if sssp.sssp_server_mode(srv) == sssp.SSSP_BATCH_SHARED else "separate",
           "result_buffers": nbuf, "plain_queries_per_s": plain_qps, "rates": []}
    for rate in rates:
        arr = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * window_s * 1.2) + 16))
        arr = arr[arr < window_s]
        srcs = rng.choice(np.asarray(sources), size=arr.size)
        free = list(range(nbuf))
        outstanding = {}
        lat = []
        held = []            # (source, buffer) of served results kept for the check
        hold_max = max(1, min(8, nbuf // 4))
        ndone = 0
        i = 0
        t0 = time.perf_counter()
        last_done = t0
        while (i < arr.size or outstanding) and time.perf_counter() - t0 < hard_s:
            now = time.perf_counter() - t0
            progressed = False
            while i < arr.size and arr[i] <= now and free:
                b = free.pop()
                tk = sssp.sssp_server_submit(srv, int(srcs[i]), bufs[b].data_ptr())
                outstanding[tk] = (arr[i], b, int(srcs[i]))
                i += 1
                progressed = True
            done = sssp.sssp_server_drain(srv)
            if done:
                tnow = time.perf_counter()
                for tk, info in done:
                    a_, b, src_ = outstanding.pop(tk)
                    lat.append(tnow - t0 - a_)
                    if len(held) < hold_max and (ndone < 2 or ndone % 8 == 0):
                        held.append((src_, b))
                    else:
                        free.append(b)
                    ndone += 1
                last_done = tnow
                progressed = True
            if not progressed:
                time.sleep(0.00005)
        elapsed = last_done - t0
        backlog = int(arr.size - i)
        lat_ms = np.asarray(lat) * 1e3
        out["rates"].append({
            "offered_per_s": rate, "arrived": int(arr.size), "completed": len(lat),
            "not_admitted_in_window": backlog,
            "queries_per_s": len(lat) / elapsed if elapsed > 0 else 0.0,
            "p50_ms": float(np.percentile(lat_ms, 50)) if lat else None,
            "p99_ms": float(np.percentile(lat_ms, 99)) if lat else None})
        # let anything still outstanding finish before the next rate
        for tk in list(outstanding):
            sssp.sssp_server_wait(srv, tk, 120_000_000_000)
        sssp.sssp_server_drain(srv)
        torch.cuda.synchronize()
        if held:  # the sampled served results against single solves of their sources
            one = torch.empty(g.n, dtype=torch.int64, device="cuda")
            eq = 0
            for src_, b in held:
                if tuned:
                    sssp.sssp_solve_tuned(G.handle, src_, one.data_ptr(), stream)
                else:
                    G.solve(src_, algo, prm, one, stream)
                torch.cuda.synchronize()
                eq += int(bool(torch.equal(bufs[b], one)))
            del one
            out["rates"][-1]["checked"] = len(held)
            out["rates"][-1]["equal_to_single"] = eq
    best = max(r["queries_per_s"] for r in out["rates"])
    out["checked"] = sum(r.get("checked", 0) for r in out["rates"])
    out["all_equal"] = all(r.get("equal_to_single", 0) == r.get("checked", 0) for r in out["rates"])
    out["saturation_queries_per_s"] = best
    out["speedup_vs_plain"] = best / plain_qps
    out["launches"] = sssp.sssp_server_stats(srv)["launches"]
    sssp.sssp_server_destroy(srv)
    del bufs
    torch.cuda.empty_cache()
    return out


def run_serve_sweep(args):
    """--serve: the serving sweep over resident graphs (RMAT scale 25, the
    4096^2 road-like grid, the 2M-point k-NN graph): each graph is tuned for
    single solves (the plain loop) and for batched launches (the server), then
    a Poisson stream at every offered rate for --serve-window seconds."""
    import torch
    from paper_2105_06145_gb300 import graphgen as gg, sssp
    rates = [int(x) for x in args.serve_rates.split(",")]
    stream = torch.cuda.current_stream().cuda_stream
    for name in args.serve_workloads.split(","):
        t0 = time.perf_counter()
        if name == "rmat25":
            g = gg.rmat(25, 16, 0.57, 0.19, 0.19, gen_seed=8, wseed=8)
        elif name == "road":
            g, _ = gg.workload_road(4096)
        elif name == "knn":
            g = gg.knn(2_000_000, 64, 0.02, 10, float(1 << 20), seed=10)
        elif name == "rmat22":
            g, _ = gg.workload_rmat(22)
        else:
            raise SystemExit(f"unknown serving workload {name}")
        gen_s = time.perf_counter() - t0
        lab = np.ones(g.n, np.uint8) if name == "knn" else gg.largest_cc(g)
        sources = gg.pick_sources(g, 256, 9, mask=lab)
        G = sssp.Graph(g, sssp.SSSP_GRAPH_SYMMETRIC)
        tune = sssp.sssp_autotune(G.handle, sources[:3], stream)
        btune = sssp.sssp_autotune_batch(G.handle, sources[:args.serve_slots or 64],
                                         (1 << sssp.SSSP_RHO) | (1 << sssp.SSSP_DELTA_STAR), stream)
        torch.cuda.empty_cache()
        res = measure_serving(sssp, G, g, torch, sources, rates, window_s=args.serve_window,
                              slots=args.serve_slots, algo=btune["algo"], param=btune["param"], tuned=True)
        print(json.dumps({"serve_workload": name, "n": g.n, "m": g.m, "generate_s": gen_s, "tuning": tune,
                          "batch_tuning": btune, **res}), flush=True)
        G.close()
        del G
        torch.cuda.empty_cache()


def run_lbpq(args):
    """--lbpq: the LaB-PQ comparison of App. F on the device: n records all in
    Q with random 40-bit keys; Extract of the rho smallest (theta = the rho-th
    smallest key) from the tournament tree (Sec. 4.2) and from the array
    (Sec. 4.3, a scan of the whole list), 10 runs each, the extracted records
    re-inserted between tree runs (untimed, as the paper leaves out update
    cost)."""
    import torch
    from paper_2105_06145_gb300 import sssp
    n = args.lbpq_n
    rng = np.random.default_rng(12)
    key = rng.integers(0, 1 << 40, n, dtype=np.uint64)
    kd = torch.from_numpy(key.view(np.int64)).cuda()
    del key
    ids = torch.arange(n, dtype=torch.int32, device="cuda")
    srt = torch.sort(kd).values
    stream_obj = torch.cuda.current_stream()
    st = stream_obj.cuda_stream
    t = sssp.sssp_tourney_create(n)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(4, dtype=torch.int32, device="cuda")
    mn = torch.zeros(1, dtype=torch.int64, device="cuda")
    t0 = time.perf_counter()
    sssp.sssp_tourney_update(t, ids.data_ptr(), n, st)
    sssp.sssp_tourney_min(t, kd.data_ptr(), mn.data_ptr(), st)  # builds every interior key
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    ext = torch.empty(n, dtype=torch.int32, device="cuda")
    keep = torch.empty(n, dtype=torch.int32, device="cuda")
    rows = []
    for lg in args.lbpq_rho.split(","):
        rho = 1 << int(lg)
        theta = int(srt[rho - 1].item())
        tree_ms, arr_ms, got = 0.0, 0.0, 0
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream_obj)
            sssp.sssp_tourney_extract(t, kd.data_ptr(), theta, out.data_ptr(), cnt.data_ptr(), st)
            e1.record(stream_obj)
            torch.cuda.synchronize()
            tree_ms += e0.elapsed_time(e1)
            got = int(cnt[0].item())
            sssp.sssp_tourney_update(t, out.data_ptr(), got, st)  # back into Q, untimed
        sssp.sssp_tourney_min(t, kd.data_ptr(), mn.data_ptr(), st)
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream_obj)
            sssp.sssp_array_extract(ids.data_ptr(), n, kd.data_ptr(), theta, ext.data_ptr(), cnt.data_ptr() + 4,
                                    keep.data_ptr(), cnt.data_ptr() + 8, st)
            e1.record(stream_obj)
            torch.cuda.synchronize()
            arr_ms += e0.elapsed_time(e1)
        arr_got = int(cnt[1].item())
        rows.append({"rho": rho, "extracted": got, "tree_ms_10_runs": tree_ms, "array_ms_10_runs": arr_ms,
                     "array_extracted": arr_got})
    sssp.sssp_tourney_destroy(t)
    print(json.dumps({"lbpq_extract": {"n": n, "tree_build_s": build_s, "rows": rows}}), flush=True)


def run_trace(args):
    """--trace: one solve of the workload from its first source with the
    per-step trace on (sssp_options.trace), printed as a per-step phase table
    (device times of Extract, the first grid barrier, the relaxation and the
    end-of-step barrier) and a JSON summary.  The configuration is the bench's
    (rho-Stepping, --param, --rho-reduced, --rho-warmup) unless --trace-config gives
    algo,param,shape,local_budget[,flags] (flags: extra SSSP_SOLVE_* bits, e.g.
    2 = fused super-sparse steps, whose steps have no barrier after Extract:
    there the relaxation column starts when block 0 has extracted)."""
    import torch
    from paper_2105_06145_gb300 import sssp
    g, srcs, label = build_workload(args.workload, args.scale)
    flags = sssp.SSSP_GRAPH_SYMMETRIC | (sssp.SSSP_GRAPH_REORDER if args.workload == "rmat" else 0)
    G = sssp.Graph(g, flags)
    xflags = 0
    if args.trace_config:
        cfg = [int(x) for x in args.trace_config.split(",")]
        a, prm, shape, local = cfg[:4]
        xflags = cfg[4] if len(cfg) > 4 else 0
    else:
        a, prm, shape, local = sssp.ALGOS[args.algo], args.param or (1 << 18), 0, 0
    red = args.rho_reduced if args.rho_reduced > 0 else sssp.SSSP_RHO_REDUCED_NONE
    stream = torch.cuda.current_stream().cuda_stream
    d = torch.empty(g.n, dtype=torch.int64, device="cuda")
    cap = 100000
    trb = torch.zeros(cap * sssp.TRACE_RECORD_BYTES // 8, dtype=torch.int64, device="cuda")
    base = dict(flags=sssp.SSSP_SOLVE_BIDIRECTIONAL | xflags, shape=shape, local_budget=local, rho_reduced=red)
    if a == sssp.SSSP_RHO:
        ws, wr = (int(x) for x in args.rho_warmup.split(","))
        base.update(rho_warmup_steps=ws, rho_warmup=wr)
    s0 = srcs[0]
    for _ in range(2):
        G.solve(s0, a, prm, d, stream, sssp.make_options(**base))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    G.solve(s0, a, prm, d, stream, sssp.make_options(**base))
    e1.record()
    torch.cuda.synchronize()
    G.solve(s0, a, prm, d, stream, sssp.make_options(trace_ptr=trb.data_ptr(), trace_cap=cap, **base))
    st = G.stats(stream)
    tr = np.frombuffer(trb.cpu().numpy().tobytes(), dtype=sssp.TRACE_DTYPE)[:min(st["steps"], cap)]
    t_ns, t_rel = tr["t_ns"].astype(np.int64), tr["t_relax_ns"].astype(np.int64)
    has_q = tr["queued"] > 0  # a fused solve's last step only re-checks (no Extract)
    ext = np.where(has_q, tr["t_extract_end_max"].astype(np.int64) - t_ns, 0)
    bar1 = np.where(has_q, np.maximum(t_rel - tr["t_extract_end_max"].astype(np.int64), 0), 0)
    rel = tr["t_relax_end_max"].astype(np.int64) - t_rel
    bar2 = np.append(t_ns[1:], t_ns[-1]) - tr["t_relax_end_max"].astype(np.int64)
    bar2[-1] = 0
    if args.trace_steps:
        for i, t in enumerate(tr):
            print(f"step {i + 1:5d} q={int(t['queued']):9d} f={int(t['extracted']):9d} edges={int(t['edges']):10d} "
                  f"extract_us={ext[i] / 1e3:7.1f} barrier_us={bar1[i] / 1e3:5.1f} relax_us={rel[i] / 1e3:7.1f} "
                  f"end_us={bar2[i] / 1e3:5.1f}")
    summary = {"workload": label, "source": int(s0), "algo": ALGO_NAMES[a], "param": prm, "shape": shape,
               "local_budget": local, "flags": int(base["flags"]), "rho_reduced": args.rho_reduced,
               "rho_warmup": args.rho_warmup if a == sssp.SSSP_RHO else None, "ms_untraced": e0.elapsed_time(e1),
               "steps": int(st["steps"]), "edges_per_m": st["edges"] / g.m,
               "phase_us_sum": {"extract": float(ext.sum() / 1e3), "barrier_after_extract": float(bar1.sum() / 1e3),
                                "relax": float(rel.sum() / 1e3), "end_of_step": float(bar2.sum() / 1e3)},
               "phase_us_median": {"extract": float(np.median(ext) / 1e3), "barrier_after_extract": float(np.median(bar1) / 1e3),
                                   "relax": float(np.median(rel) / 1e3), "end_of_step": float(np.median(bar2[:-1]) / 1e3) if len(bar2) > 1 else 0.0}}
    print(json.dumps({"trace": summary}), flush=True)
    G.close()


def run_batched_case(args):
    """--batched-case: 64 sources on RMAT at --scale (degree-ordered symmetric
    copy, rho-Stepping rho = n/16 with 6 reduced dense steps, bidirectional),
    two launches with one shared edge scan (SSSP_BATCH_SHARED) and two with
    separate instances (SSSP_BATCH_SEPARATE), every instance checked against
    its single solve; the case the batch kernels' profiles capture."""
    import torch
    from paper_2105_06145_gb300 import graphgen as gg, sssp
    g = gg.rmat(args.scale, 16, 0.57, 0.19, 0.19, gen_seed=2, wseed=3)
    G = sssp.Graph(g, sssp.SSSP_GRAPH_SYMMETRIC | sssp.SSSP_GRAPH_REORDER)
    srcs = gg.pick_sources(g, 64, 6)
    stream = torch.cuda.current_stream().cuda_stream
    rho = max(64, g.n // 16)
    sssp.sssp_graph_set_tuning(G.handle, {"algo": 0, "param": rho, "flags": 1, "rho_reduced": 6})
    out = torch.empty(64 * g.n, dtype=torch.int64, device="cuda")
    one = torch.empty(g.n, dtype=torch.int64, device="cuda")
    res = {}
    for mode, name in ((sssp.SSSP_BATCH_SHARED, "shared"), (sssp.SSSP_BATCH_SEPARATE, "separate")):
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            sssp.sssp_solve_sources_ex(G.handle, srcs, 0, [rho] * 64, mode, out.data_ptr(), stream)
            e1.record()
            torch.cuda.synchronize()
            st, stats = sssp.sssp_batch_last_stats(64, stream)
            assert st == 0, st
        eq = rows_equal_to_single(torch, torch.cuda.current_stream(), out.view(64, g.n), srcs,
                                  lambda s_, o: sssp.sssp_solve_tuned(G.handle, s_, o.data_ptr(), stream))
        res[name] = {"ms": e0.elapsed_time(e1), "edges_per_m": sum(x["edges"] for x in stats) / 64 / g.m,
                     "all_equal": eq == 64}
    print(json.dumps({"batched_case": {"scale": args.scale, "k": 64, **res}}), flush=True)
    G.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat", choices=["rmat", "road", "grid"])
    ap.add_argument("--scale", type=int, default=22)
    ap.add_argument("--algo", default="rho", choices=["rho", "delta_star", "bellman_ford"])
    ap.add_argument("--param", type=int, default=0, help="rho or Delta (0 = workload default)")
    ap.add_argument("--cpu-baseline-sources", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-bidir", action="store_true", help="plain push relaxation only")
    ap.add_argument("--rho-reduced", type=int, default=4,
                    help="rho-Stepping: dense steps that use rho/10 (the paper uses 2; 0 = none)")
    ap.add_argument("--rho-warmup", default="8,256",
                    help="rho-Stepping: STEPS,RHO -- the first STEPS steps use rho = RHO (0,0 = none)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solve measurements")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-other", action="store_true", help="skip the road-like and k-NN workloads")
    ap.add_argument("--no-sweep", action="store_true", help="skip the rho / Delta* / Bellman-Ford sweep")
    ap.add_argument("--serve", action="store_true", help="run the serving sweep (RMAT-25, road, k-NN) only")
    ap.add_argument("--serve-workloads", default="rmat25,road,knn")
    ap.add_argument("--serve-rates", default="1000,2000,5000,10000,20000,50000")
    ap.add_argument("--serve-window", type=float, default=1.0)
    ap.add_argument("--serve-slots", type=int, default=0, help="0 = the batch autotuner's slot count")
    ap.add_argument("--lbpq", action="store_true", help="the tournament-tree vs array LaB-PQ Extract comparison only")
    ap.add_argument("--trace", action="store_true", help="per-step phase summary of one traced solve only")
    ap.add_argument("--trace-config", default="", help="algo,param,shape,local_budget[,flags] for --trace")
    ap.add_argument("--trace-steps", action="store_true", help="--trace: also print every step")
    ap.add_argument("--batched-case", action="store_true",
                    help="64 sources on RMAT --scale with the shared-scan and separate batch kernels only")
    ap.add_argument("--lbpq-n", type=int, default=100_000_000)
    ap.add_argument("--lbpq-rho", default="10,13,16,19,22,25", help="log2 of the rho values")
    args = ap.parse_args()

    rank, world, local = dist_env()
    if args.serve:
        run_serve_sweep(args)
        return
    if args.lbpq:
        run_lbpq(args)
        return
    if args.trace:
        run_trace(args)
        return
    if args.batched_case:
        run_batched_case(args)
        return
    g, srcs, label = build_workload(args.workload, args.scale)

    if args.impl == "reference":
        run_reference(args, g, srcs, label, rank, world)
        return

    import torch
    from paper_2105_06145_gb300 import sssp

    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        pg = dist
    algo = sssp.ALGOS[args.algo]
    param = args.param or {"rho": 1 << 18, "delta_star": 1 << 15, "bellman_ford": 0}[args.algo]
    if args.workload == "road" and not args.param and args.algo == "delta_star":
        param = 1 << 13

    # every workload graph is symmetric: verify once at creation, then use the
    # paper's bidirectional relaxation for undirected graphs (Sec. 6); single
    # solves run on the degree-ordered device copy (distances still come back
    # in the generator's ids, inside the timed solve)
    G = sssp.Graph(g, sssp.SSSP_GRAPH_SYMMETRIC | sssp.SSSP_GRAPH_VERIFY | sssp.SSSP_GRAPH_REORDER)
    bidir = not args.no_bidir
    solve_flags = sssp.SSSP_SOLVE_BIDIRECTIONAL if bidir else 0
    # rho-Stepping runs its first dense steps with rho/10 (Sec. 6 "Threshold
    # estimation"); the count is a tuning knob (the paper's 2 was tuned on its
    # 96-core machine; after the warm-up steps below, 4 measured best for this
    # workload on the GB300)
    red_opt = args.rho_reduced if args.rho_reduced > 0 else sssp.SSSP_RHO_REDUCED_NONE
    # ... and may start with warm-up steps at a small rho (the first, sparse
    # waves, which hold the high-degree vertices, in small groups)
    warm_steps, warm_rho = (int(x) for x in args.rho_warmup.split(","))
    warm = dict(rho_warmup_steps=warm_steps, rho_warmup=warm_rho) if algo == sssp.SSSP_RHO else {}
    stream_obj = torch.cuda.Stream()
    stream = stream_obj.cuda_stream
    dist_out = torch.empty(g.n, dtype=torch.int64, device="cuda")
    nsrc = len(srcs)
    rank_srcs = rank_sources(srcs, rank)

    K, W = args.steps, args.warmup
    stats_buf = torch.zeros((K, sssp.STATS_BYTES // 8), dtype=torch.int64, device="cuda")
    with torch.cuda.stream(stream_obj):
        wopts = sssp.make_options(flags=solve_flags, rho_reduced=red_opt, **warm)
        for i in range(W):
            G.solve(rank_srcs[i % nsrc], algo, param, dist_out, stream, wopts)
        assert G.status(stream) == sssp.SSSP_OK
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        opts = [sssp.make_options(stats_out_ptr=stats_buf[i].data_ptr(), flags=solve_flags, rho_reduced=red_opt,
                                  **warm) for i in range(K)]
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        torch.cuda.synchronize()
        ev[0].record(stream_obj)
        for i in range(K):
            G.solve(rank_srcs[i % nsrc], algo, param, dist_out, stream, opts[i])
            ev[i + 1].record(stream_obj)
        torch.cuda.synchronize()
        if pg:
            pg.barrier()
        clk = clocks.stop()
    per_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(K)]
    total_ms = ev[0].elapsed_time(ev[K])
    raw = stats_buf.cpu().numpy().view(np.uint64)
    stats = []
    for i in range(K):
        r = raw[i]
        stats.append({"steps": int(r[0]), "queued": int(r[1]), "extracted": int(r[2]),
                      "edges": int(r[3]), "updates": int(r[4]),
                      "status": int(np.int32(r[5] & np.uint64(0xFFFFFFFF)))})
    assert all(s["status"] == 0 for s in stats), stats
    gteps, total_ms = aggregate(total_ms, K, g.m, world, pg)
    peak, peak_kind = load_peaks()
    abytes = [algorithmic_bytes(s) for s in stats]
    ach_gbs = float(np.mean([b / (t * 1e-3) / 1e9 for b, t in zip(abytes, per_ms)]))
    floor_bytes = 8 * g.m + 28 * g.n
    cap = captured_traffic() if args.workload == "rmat" and args.scale == 22 else None
    traffic = None
    if cap is not None:  # scale the captured launch's DRAM bytes by edges scanned
        traffic = cap[0] / cap[1] * float(np.mean([s_["edges"] for s_ in stats]))
    floor_gbs = floor_bytes / (np.mean(per_ms) * 1e-3) / 1e9

    # Calibration: a stream + random-gather ceiling on this GPU, measured with a
    # library routine (torch.index_select of the graph's m edge targets into the
    # n-entry distance array: 8 B streamed index + one random 8-byte gather per
    # edge, the relaxation's memory pattern without its atomics).
    gather = None
    if rank == 0:
        idx = torch.from_numpy(g.tgt.astype(np.int64))
        idx = idx.to("cuda", non_blocking=False)
        outg = torch.empty(g.m, dtype=torch.int64, device="cuda")
        for _ in range(2):
            torch.index_select(dist_out, 0, idx, out=outg)
        ge0, ge1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ge0.record()
        for _ in range(3):
            torch.index_select(dist_out, 0, idx, out=outg)
        ge1.record()
        torch.cuda.synchronize()
        gms = ge0.elapsed_time(ge1) / 3
        gather = {"gathers_per_s": g.m / (gms * 1e-3), "kernel": "torch.index_select (int64 index)"}
        del idx, outg

    # the parameter sweep of the workload (RMAT scale 22: rho in {2^18, 2^20,
    # 2^22}, Delta* in {2^13, 2^15, 2^17}, Bellman-Ford), same graph copy,
    # relaxation and sources as the headline; one solve per source
    sweep = None
    if rank == 0 and not args.no_sweep and args.workload == "rmat" and args.scale == 22:
        sweep = []
        for sa, sp in ((sssp.SSSP_RHO, 1 << 18), (sssp.SSSP_RHO, 1 << 20), (sssp.SSSP_RHO, 1 << 22),
                       (sssp.SSSP_DELTA_STAR, 1 << 13), (sssp.SSSP_DELTA_STAR, 1 << 15),
                       (sssp.SSSP_DELTA_STAR, 1 << 17), (sssp.SSSP_BELLMAN_FORD, 0)):
            sbuf = torch.zeros((nsrc, sssp.STATS_BYTES // 8), dtype=torch.int64, device="cuda")
            sw = dict(rho_warmup_steps=warm_steps, rho_warmup=warm_rho) if sa == sssp.SSSP_RHO else {}
            sopt = [sssp.make_options(stats_out_ptr=sbuf[i].data_ptr(), flags=solve_flags, rho_reduced=red_opt, **sw)
                    for i in range(nsrc)]
            ts = _timed(torch, stream_obj, lambda: [G.solve(srcs[i], sa, sp, dist_out, stream, sopt[i])
                                                    for i in range(nsrc)])
            sr = sbuf.cpu().numpy().view(np.uint64)
            assert all(int(np.int32(r[5] & np.uint64(0xFFFFFFFF))) == 0 for r in sr)
            sweep.append({"algo": ALGO_NAMES[sa], "param": sp, "ms_per_solve": ts / nsrc,
                          "gteps": nsrc * g.m / (ts * 1e-3) / 1e9,
                          "steps": float(np.mean(sr[:, 0].astype(np.float64))),
                          "edges_per_m": float(np.mean(sr[:, 3].astype(np.float64))) / g.m})

    # end-to-end through the C ABI with a host output buffer (pinned)
    e2e = None
    if not args.no_e2e:
        host = torch.empty(g.n, dtype=torch.int64, pin_memory=True)
        for i in range(2):
            sssp.sssp_solve_host_ptr(G.handle, rank_srcs[i % nsrc], algo, param, host.data_ptr(), stream, wopts)
        t0 = time.perf_counter()
        for i in range(K):
            rc = sssp.sssp_solve_host_ptr(G.handle, rank_srcs[i % nsrc], algo, param, host.data_ptr(),
                                          stream, wopts)
            assert rc == 0, rc
        te = time.perf_counter() - t0
        e2e = {"value": world * K * g.m / te / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": 12, "d2h_bytes_per_step": 8 * g.n,
               "note": "graph resident; per step the source id and parameter go in as launch "
                       "arguments and the uint64 distance array comes back to pinned host memory"}

    # batched solves: queries/s of one batched launch vs the
    # plain loop of single solves on the same GPU, identical distances
    batched = None
    if rank == 0 and not args.no_batch and args.workload == "rmat" and args.scale == 22:
        batched = measure_batched(sssp, G, g, torch, stream, stream_obj, cpu=not args.no_cpu_baseline)

    served = None
    if rank == 0 and not args.no_serve and args.workload == "rmat" and args.scale == 22:
        # the server's configuration and slot count from the batch autotuner
        btune = sssp.sssp_autotune_batch(G.handle, gg_sources(g)[:64], 1 << sssp.SSSP_RHO, stream)
        torch.cuda.empty_cache()
        served = {"rmat22": measure_serving(sssp, G, g, torch, gg_sources(g), [100, 1000], window_s=2.0,
                                            hard_s=10.0, slots=0, algo=btune["algo"], param=btune["param"],
                                            tuned=True)}
        served["rmat22"]["batch_tuning"] = btune

    # the road-like and k-NN workloads: tuned plain loop, batched and served
    workloads = None
    if rank == 0 and not args.no_other and args.workload == "rmat" and args.scale == 22:
        workloads = {}
        for wname in ("road4096", "knn2m"):
            workloads[wname] = measure_workload(wname, sssp, torch, stream, stream_obj,
                                                cpu=not args.no_cpu_baseline)
            if batched is not None:
                batched[f"sources64_{wname}"] = workloads[wname]["batched64"]
            if served is not None:
                served[wname] = workloads[wname]["served"]

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        ns = args.cpu_baseline_sources
        t0 = time.perf_counter()
        for i in range(ns):
            oracle.dijkstra(g, srcs[i % nsrc])
        tc = time.perf_counter() - t0
        cpu = {"value": ns * g.m / tc / 1e9, "unit": "GTEPS", "cores": 1, "cpu_model": cpu_model(), "kind": "oracle",
               "sample": f"{ns} full single-source binary-heap Dijkstra solves of {label} "
                         f"({tc:.1f} s)"}

    if rank == 0:
        mean_stats = {k: float(np.mean([s[k] for s in stats])) for k in
                      ("steps", "queued", "extracted", "edges", "updates")}
        line = {
            "metric": METRIC, "value": gteps, "unit": "GTEPS", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": label, "n": g.n, "m": g.m, "algo": args.algo, "param": param,
                       "rho_reduced_dense_steps": args.rho_reduced if args.algo == "rho" else None,
                       "rho_warmup": {"steps": warm_steps, "rho": warm_rho} if args.algo == "rho" else None,
                       "bidirectional": bidir, "graph_layout": "relabelled by decreasing degree (SSSP_GRAPH_REORDER)",
                       "sources": nsrc, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (packed edges %.2f GB > 129 MB L2)" % (8 * g.m / 1e9),
                       "per_solve_mean": mean_stats},
            "roofline": {"bound": "hbm", "achieved": ach_gbs, "peak": peak, "unit": "GB/s",
                         "frac": ach_gbs / peak, "traffic": traffic,
                         "frac_dram": (traffic / (np.mean(per_ms) * 1e-3) / 1e9 / peak) if traffic else None,
                         "peak_kind": peak_kind + " (burst copy)",
                         "kernel": "sssp::solve_kernel (persistent, one launch per solve)",
                         "algorithmic_bytes_per_launch": float(np.mean(abytes)),
                         "floor_frac": floor_gbs / peak,
                         "edge_scan_rate": float(np.mean([s_["edges"] for s_ in stats]) / (np.mean(per_ms) * 1e-3)),
                         "gather_ceiling": gather},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "batched": batched,
            "served": served,
            "workloads": workloads,
            "sweep": sweep,
            "gpu_launches": K,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    G.close()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
