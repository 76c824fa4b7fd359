"""Parity of the CUDA solve (through the C ABI) with the CPU oracle.

Distances are unique, so every comparison is element-by-element equality of
uint64 arrays.  Inputs come from the seeded generators; expected values come
from the oracle only.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2105_06145_gb300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INF = (1 << 64) - 1


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_06145_gb300 import sssp
    return sssp


def solve(lib, g, s, algo, param, opts=None, G=None):
    own = G is None
    if own:
        G = lib.Graph(g)
    dist = torch.full((g.n,), 7, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    G.solve(s, algo, param, dist, stream, opts)
    st = G.stats(stream)
    out = dist.cpu().numpy().view(np.uint64).copy()
    if own:
        G.close()
    return out, st


ALGO_PARAMS = [(0, 1), (0, 2), (0, 31), (0, 1 << 10), (0, 65536), (0, (1 << 32) - 1),
               (1, 1), (1, 1 << 13), (1, 1 << 17), (1, INF), (2, 0),
               (3, 1), (3, 1 << 13), (3, INF), (4, 0)]


def test_grid256_all_rules(lib):
    g, s = gg.workload_grid256()
    want = oracle.dijkstra(g, s)
    G = lib.Graph(g)
    for algo, param in ALGO_PARAMS:
        got, st = solve(lib, g, s, algo, param, G=G)
        assert st["status"] == 0, (algo, param, st)
        assert np.array_equal(got, want), (algo, param)
    G.close()


@pytest.mark.parametrize("algo,param", [(0, 1 << 12), (1, 1 << 15), (2, 0), (0, 3), (3, 1 << 15), (4, 0)])
def test_rmat16_and_road(lib, algo, param):
    for g in (gg.rmat(16, 16, gen_seed=11, wseed=12), gg.road(300, 0.75, seed=3)):
        s = gg.pick_sources(g, 1, 5)[0]
        want = oracle.dijkstra(g, s)
        got, st = solve(lib, g, s, algo, param)
        assert st["status"] == 0
        assert np.array_equal(got, want), (g.name, algo, param)


def test_edge_case_graphs(lib):
    cases = [
        (gg.from_edges(1, [], [], []), 0),                              # one vertex, no edges
        (gg.from_edges(2, [0], [1], [0]), 0),                           # zero weight
        (gg.from_edges(3, [0, 0, 1], [0, 1, 1], [5, 7, 3]), 0),         # self-loops
        (gg.from_edges(3, [0, 0, 0], [1, 1, 2], [9, 4, 0xFFFFFFFF]), 0),  # multi-edge, max weight
        (gg.chain(2000, wseed=1, wlo=0, whi=(1 << 32) - 1), 0),          # long chain, huge weights
        (gg.chain(2000, wseed=1, both=True), 1000),
        (gg.star(5000, wseed=2), 0),
        (gg.star(5000, wseed=2), 17),                                    # isolated source
        (gg.complete(90, wseed=4), 3),
        (gg.random_graph(3000, 9000, 0, 3, seed=5), 1),                  # disconnected, w in [0,3]
        (gg.random_graph(50, 2000, 0, 0xFFFFFFFF, seed=6), 0),
        (gg.grid(1, 4099, wseed=3), 2049),                               # ragged 1-D grid
    ]
    for g, s in cases:
        want = oracle.dijkstra(g, s)
        for algo, param in ((0, 1), (0, 64), (0, INF), (1, 1), (1, 1000), (2, 0), (3, 1000), (4, 0)):
            got, st = solve(lib, g, s, algo, param)
            assert st["status"] == 0, (g.name, algo, param)
            assert np.array_equal(got, want), (g.name, s, algo, param)


def test_tiny_random_graphs(lib):
    rng = np.random.default_rng(3)
    for k in range(150):
        n = int(rng.integers(1, 200))
        m = int(rng.integers(0, 6 * n + 1))
        lo, hi = [(0, 0), (0, 5), (1, 1 << 18), (0, 0xFFFFFFFF)][k % 4]
        g = gg.random_graph(n, m, lo, hi, seed=1000 + k)
        s = int(rng.integers(0, n))
        want = oracle.dijkstra(g, s)
        algo, param = ALGO_PARAMS[k % len(ALGO_PARAMS)]
        got, st = solve(lib, g, s, algo, param)
        assert st["status"] == 0 and np.array_equal(got, want), (k, algo, param)


def test_hub_vertices_use_chunked_relaxation(lib):
    """Hubs with 2e5 out-edges (split into many chunk items) plus a sparse rest."""
    n = 300000
    rng = np.random.default_rng(9)
    hubs = [0, 1, 2]
    src, dst, w = [], [], []
    for h in hubs:
        t = rng.integers(0, n, 200000)
        src.append(np.full(t.size, h)); dst.append(t); w.append(rng.integers(1, 1 << 18, t.size))
    t = rng.integers(0, n, 3 * n)
    src.append(rng.integers(0, n, t.size)); dst.append(t); w.append(rng.integers(1, 1 << 18, t.size))
    src.append(np.array([5, 5, 5])); dst.append(np.array(hubs)); w.append(np.array([1, 2, 3]))
    g = gg.from_edges(n, np.concatenate(src), np.concatenate(dst), np.concatenate(w))
    want = oracle.dijkstra(g, 5)
    for algo, param in ((0, 1 << 14), (1, 1 << 16), (2, 0)):
        got, st = solve(lib, g, 5, algo, param)
        assert st["status"] == 0 and np.array_equal(got, want), (algo, param)


def test_repeated_solves_reuse_scratch(lib):
    g = gg.rmat(14, 16, gen_seed=3, wseed=4)
    G = lib.Graph(g)
    srcs = gg.pick_sources(g, 6, 8)
    for i, s in enumerate(srcs * 2):
        algo, param = ALGO_PARAMS[i % len(ALGO_PARAMS)]
        got, st = solve(lib, g, s, algo, param, G=G)
        assert st["status"] == 0 and np.array_equal(got, oracle.dijkstra(g, s))
    G.close()


def test_solve_host_end_to_end(lib):
    g = gg.rmat(15, 16, gen_seed=5, wseed=6)
    s = gg.pick_sources(g, 1, 2)[0]
    G = lib.Graph(g)
    out = np.zeros(g.n, dtype=np.uint64)
    assert lib.sssp_solve_host(G.handle, s, 0, 1 << 12, out) == 0
    assert np.array_equal(out, oracle.dijkstra(g, s))
    G.close()


def test_step_bounds_and_counters(lib):
    """Lemma 5.1 (each vertex extracted <= h(v) times, any interleaving, weights
    >= 1), Bellman-Ford <= k_n + 1 steps, Theorem 5.5 for Delta*, and the
    trace totals agree with the solve totals."""
    for g in (gg.grid(80, 80, wseed=5), gg.rmat(13, 8, gen_seed=7, wseed=8), gg.road(120, 0.75, seed=9)):
        s = gg.pick_sources(g, 1, 3)[0]
        want = oracle.dijkstra(g, s)
        h, kn = oracle.hops(g, s)
        L = int(g.w.max())
        G = lib.Graph(g)
        for algo, param in ((0, 64), (0, 1 << 12), (1, 1 << 12), (1, 1 << 16), (2, 0), (3, 1 << 12), (4, 0)):
            ext = torch.zeros(g.n, dtype=torch.int32, device="cuda")
            cap = 100000
            trace = torch.zeros(cap * lib.TRACE_RECORD_BYTES // 8, dtype=torch.int64, device="cuda")
            opts = lib.make_options(ext_count_ptr=ext.data_ptr(), trace_ptr=trace.data_ptr(),
                                    trace_cap=cap)
            got, st = solve(lib, g, s, algo, param, opts=opts, G=G)
            assert st["status"] == 0 and np.array_equal(got, want)
            e = ext.cpu().numpy().astype(np.int64)
            reach = want != np.uint64(INF)
            assert np.all(e[~reach] == 0)
            hv = h.astype(np.int64)
            hv[s] = 1
            assert np.all(e[reach] <= hv[reach]), (g.name, algo, param)
            assert int(e.sum()) == st["extracted"]
            if algo == 2:
                assert st["steps"] <= kn + 1
            elif algo == 1:
                assert st["steps"] <= math.ceil(kn * L / param) + kn + 1
            elif algo == 4:
                # theta = min_Q delta with positive weights: one distance settled per
                # step, every reachable vertex extracted exactly once
                assert st["steps"] == np.unique(want[reach]).size
                assert np.all(e[reach] == 1)
            rec = np.frombuffer(trace.cpu().numpy().tobytes(),
                                dtype=np.dtype(lib.TRACE_DTYPE))[: st["steps"]]
            assert np.all(np.diff(rec["t_ns"].astype(np.int64)) >= 0)
            assert int(rec["extracted"].sum()) == st["extracted"]
            assert int(rec["queued"].sum()) == st["queued"]
            assert int(rec["edges"].sum()) == st["edges"]
            assert int(rec["updates"].sum()) == st["updates"]
            assert rec["queued"][0] == 1 and np.all(rec["extracted"] >= 1)
            if algo == 2:
                assert np.all(rec["theta"] == np.uint64(INF))
            # edges scanned = sum of out-degrees of the extracted vertices
            deg = g.degrees()
            assert int((e * deg).sum()) == st["edges"]
        G.close()


def test_rho_threshold_matches_oracle(lib):
    """ExtDist of rho-Stepping alone: the device rule equals the oracle's on the
    same queue list, keys, seed and step (sampling, sort, rank, dense rule)."""
    rng = np.random.default_rng(21)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for trial in range(200):
        n = int(rng.integers(1, 300000))
        q = int(rng.integers(0, n + 1))
        dist = rng.integers(0, 1 << 40, n, dtype=np.uint64)
        if trial % 7 == 0:
            dist[:] = 5
        queue = rng.permutation(n)[:q].astype(np.uint32)
        rho = max(1, int([1, 2, 10, 1000, q // 3 + 1, q, 1 << 40][trial % 7]))
        seed = int(rng.integers(0, 1 << 62))
        step = int(rng.integers(1, 1000))
        dense_before = int(trial % 4)
        reduced = [2, 0, 6, 3, 1][trial % 5]  # dense steps that use rho/10 (the paper's 2)
        cap = [0, 1024, 0, 100, 4096, 1][trial % 6]  # sample cap (0: 4096; warm-up steps: 1024)
        want = oracle.rho_extdist(queue, dist, n, rho, seed, step, dense_before, reduced, max_samples=cap)
        dq = torch.from_numpy(queue.view(np.int32).copy()).cuda() if q else torch.zeros(1, dtype=torch.int32, device="cuda")
        dd = torch.from_numpy(dist.view(np.int64).copy()).cuda()
        lib.sssp_rho_threshold(dq.data_ptr(), q, dd.data_ptr(), n, rho, seed, step, dense_before, reduced,
                               out.data_ptr(), stream, max_samples=cap)
        got = int(out.cpu().numpy().view(np.uint64)[0])
        assert got == want, (trial, n, q, rho, reduced, cap)


def test_timeout_is_reported_not_hung(lib):
    """A block that leaves before the first device-wide wait makes the others'
    bounded waits run out: the solve returns SSSP_ERR_TIMEOUT and the context
    stays usable for the next solve."""
    g = gg.grid(64, 64, wseed=2)
    G = lib.Graph(g)
    dist = torch.empty(g.n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    opts = lib.make_options(timeout_ns=50_000_000, test_exit_block=2)
    G.solve(0, 0, 64, dist, stream, opts)
    assert G.status(stream) == lib.SSSP_ERR_TIMEOUT
    got, st = solve(lib, g, 0, 0, 64, G=G)
    assert st["status"] == 0 and np.array_equal(got, oracle.dijkstra(g, 0))
    G.close()


def test_invalid_arguments(lib):
    g = gg.grid(8, 8)
    G = lib.Graph(g)
    dist = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for src, algo, param in ((64, 0, 1), (0, 0, 0), (0, 1, 0), (0, 7, 1), (0, 3, 0)):
        rc = lib.sssp_solve_ex(G.handle, src, algo, param, dist.data_ptr(), None, 0, check=False)
        assert rc == lib.SSSP_ERR_INVALID_ARG
    G.close()


def test_bidirectional_relaxation(lib):
    """Sec. 6 bidirectional relaxation on symmetric graphs (verified at create):
    distances unchanged for every rule; refused on a graph not declared symmetric."""
    flags = lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY
    for g in (gg.rmat(15, 16, gen_seed=7, wseed=8), gg.road(150, 0.75, seed=4), gg.grid(90, 90, wseed=6)):
        s = gg.pick_sources(g, 1, 2)[0]
        want = oracle.dijkstra(g, s)
        G = lib.Graph(g, flags)
        for algo, param in ((0, 64), (0, 1 << 12), (1, 1 << 14), (2, 0), (3, 1 << 14), (4, 0)):
            opts = lib.make_options(flags=lib.SSSP_SOLVE_BIDIRECTIONAL)
            got, st = solve(lib, g, s, algo, param, opts=opts, G=G)
            assert st["status"] == 0 and np.array_equal(got, want), (g.name, algo, param)
        G.close()
    g = gg.rmat(12, 8)
    G = lib.Graph(g)   # not declared symmetric
    dist = torch.empty(g.n, dtype=torch.int64, device="cuda")
    rc = lib.sssp_solve_ex(G.handle, 0, 0, 64, dist.data_ptr(), lib.make_options(flags=1), 0, check=False)
    assert rc == lib.SSSP_ERR_INVALID_ARG
    G.close()


def test_local_relaxation_of_super_sparse_steps(lib):
    """Sec. 6 local BFS in super-sparse steps: distances equal the oracle's for
    rho- and Delta*-Stepping over budgets from tiny to large (including the
    room-making path of the warp's local frontier), with and without
    bidirectional relaxation; edges count the local relaxations too; refused
    for the other rules."""
    flags = lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY
    graphs = [gg.road(150, 0.75, seed=4), gg.grid(90, 90, wseed=6), gg.rmat(14, 8, gen_seed=3, wseed=4),
              gg.chain(3000, wseed=5, both=True), gg.knn(20000, clusters=8, k=6, seed=3)]
    for g in graphs:
        s = gg.pick_sources(g, 1, 9)[0]
        want = oracle.dijkstra(g, s)
        G = lib.Graph(g, flags)
        for algo, param in ((0, 64), (0, 1 << 10), (0, max(64, g.n // 16)), (1, 1 << 12), (1, 1 << 16)):
            for budget in (1, 32, 4096, 1 << 20):
                for fl in (0, lib.SSSP_SOLVE_BIDIRECTIONAL):
                    opts = lib.make_options(local_budget=budget, flags=fl)
                    got, st = solve(lib, g, s, algo, param, opts=opts, G=G)
                    assert st["status"] == 0 and np.array_equal(got, want), (g.name, algo, param, budget, fl)
                    assert st["extracted"] >= 1 and st["updates"] >= 1 or g.n == 1
        G.close()
    # the local relaxation takes several hops per step: far fewer steps on a
    # road-like graph with a small rho
    g = gg.road(200, 0.75, seed=8)
    s = gg.pick_sources(g, 1, 1)[0]
    want = oracle.dijkstra(g, s)
    _, base = solve(lib, g, s, 0, 256)
    got, loc = solve(lib, g, s, 0, 256, opts=lib.make_options(local_budget=1 << 12))
    assert np.array_equal(got, want)
    assert loc["steps"] < base["steps"], (loc, base)
    # only rho- and Delta*-Stepping have it
    G = lib.Graph(g)
    dist = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for algo, param in ((2, 0), (3, 1 << 10), (4, 0)):
        rc = lib.sssp_solve_ex(G.handle, s, algo, param, dist.data_ptr(), lib.make_options(local_budget=8), 0,
                               check=False)
        assert rc == lib.SSSP_ERR_INVALID_ARG
    G.close()


def test_reduced_rho_count_and_degree_cutoffs(lib):
    """The count of dense steps that use rho/10 (Sec. 6; the paper's 2) and
    the degree-bin cut-offs (small-degree bound, chunk length) change how the
    work is split, never the distances: every combination equals the oracle,
    on a grid, an RMAT graph (dense steps, hubs) and a hub graph whose hubs
    span many chunk records, with and without bidirectional relaxation."""
    flags = lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY
    n = 60000
    rng = np.random.default_rng(19)
    hs, hd, hw = [], [], []
    for h in (0, 1):
        t = rng.integers(0, n, 5000)
        hs += [np.full(t.size, h), t]; hd += [t, np.full(t.size, h)]
        ww = rng.integers(1, 1 << 18, t.size); hw += [ww, ww]
    t1, t2 = rng.integers(0, n, 4 * n), rng.integers(0, n, 4 * n)
    ww = rng.integers(1, 1 << 18, t1.size)
    hs += [t1, t2]; hd += [t2, t1]; hw += [ww, ww]
    hub = gg.from_edges(n, np.concatenate(hs), np.concatenate(hd), np.concatenate(hw), name="hubs_sym")
    for g in (gg.grid(120, 130, wseed=5), gg.rmat(15, 16, gen_seed=9, wseed=10), hub):
        s = gg.pick_sources(g, 1, 4)[0]
        want = oracle.dijkstra(g, s)
        G = lib.Graph(g, flags)
        for red in (0, lib.SSSP_RHO_REDUCED_NONE, 1, 6, 40):
            for algo, param in ((0, 64), (0, max(64, g.n // 16))):
                got, st = solve(lib, g, s, algo, param, opts=lib.make_options(rho_reduced=red), G=G)
                assert st["status"] == 0 and np.array_equal(got, want), (g.name, red, algo, param)
        for sd in (8, 16, 33, 64, 128):
            for ch in (128, 256, 512, 1024):
                for fl in (0, lib.SSSP_SOLVE_BIDIRECTIONAL):
                    for algo, param, shape in ((0, 1 << 10, 0), (1, 1 << 15, 1), (2, 0, 0)):
                        o = lib.make_options(small_deg=sd, chunk=ch, flags=fl, shape=shape)
                        got, st = solve(lib, g, s, algo, param, opts=o, G=G)
                        assert st["status"] == 0 and np.array_equal(got, want), (g.name, sd, ch, fl, algo)
        G.close()
    # out-of-range cut-offs are refused
    g = gg.grid(8, 8)
    G = lib.Graph(g)
    dist = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for kw in ({"small_deg": 7}, {"small_deg": 129}, {"chunk": 64}, {"chunk": 300}, {"chunk": 2048}):
        rc = lib.sssp_solve_ex(G.handle, 0, 0, 64, dist.data_ptr(), lib.make_options(**kw), 0, check=False)
        assert rc == lib.SSSP_ERR_INVALID_ARG, kw
    G.close()


def test_reduced_rho_count_full_relabelled_graph(lib):
    """The reduced-rho count on the degree-ordered copy (the benchmark's
    layout) with the local relaxation: RMAT-17, every vertex compared."""
    g = gg.rmat(17, 16, gen_seed=2, wseed=3)
    flags = lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY | lib.SSSP_GRAPH_REORDER
    G = lib.Graph(g, flags)
    for s in gg.pick_sources(g, 3, 4):
        want = oracle.dijkstra(g, s)
        for red in (2, 6, 10):
            o = lib.make_options(rho_reduced=red, flags=lib.SSSP_SOLVE_BIDIRECTIONAL)
            got, st = solve(lib, g, s, 0, g.n // 16, opts=o, G=G)
            assert st["status"] == 0 and np.array_equal(got, want), (s, red)
    G.close()


def test_fused_super_sparse_steps(lib):
    """SSSP_SOLVE_FUSED (narrow shape: a super-sparse step's Extract and
    relaxation run block by block, without the device-wide wait between them,
    and each block re-checks its extractions in the next step): every rule on a
    road-like graph, a unit-weight grid (many equal distances) and RMAT graphs
    with hub vertices (relaxed by the extracting warp in a fused step), with
    local and bidirectional relaxation, in the caller's and the degree-ordered
    layout -- the distances equal the oracle's.  A solve whose last step was
    fused ends with a re-check step (|Q| = 0); the trace totals still equal the
    solve totals; the wide shape ignores the flag."""
    F, B = lib.SSSP_SOLVE_FUSED, lib.SSSP_SOLVE_BIDIRECTIONAL
    sym = lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY
    graphs = [(gg.road(150, 0.75, seed=11), sym), (gg.grid(70, 90, wmax_excl=0), sym),
              (gg.rmat(14, 16, gen_seed=21, wseed=22), 0),
              (gg.rmat(14, 16, gen_seed=23, wseed=24), sym | lib.SSSP_GRAPH_REORDER)]
    cases = [(0, 64), (0, 1 << 12), (1, 1 << 10), (1, 1 << 14), (2, 0), (3, 1 << 12), (4, 0)]
    cap = 200000
    trace = torch.zeros(cap * lib.TRACE_RECORD_BYTES // 8, dtype=torch.int64, device="cuda")
    ended_with_recheck = 0
    for g, gflags in graphs:
        G = lib.Graph(g, gflags)
        for s in gg.pick_sources(g, 2, 5):
            want = oracle.dijkstra(g, s)
            for algo, param in cases:
                variants = [dict(flags=F)]
                if gflags & lib.SSSP_GRAPH_SYMMETRIC:
                    variants.append(dict(flags=F | B))
                if algo in (0, 1):
                    variants.append(dict(flags=F | (B if gflags else 0), local_budget=256))
                for kw in variants:
                    o = lib.make_options(shape=lib.SSSP_SHAPE_NARROW, trace_ptr=trace.data_ptr(), trace_cap=cap, **kw)
                    got, st = solve(lib, g, s, algo, param, opts=o, G=G)
                    assert st["status"] == 0 and np.array_equal(got, want), (g.name, s, algo, param, kw)
                    rec = np.frombuffer(trace.cpu().numpy().tobytes(),
                                        dtype=np.dtype(lib.TRACE_DTYPE))[: st["steps"]]
                    assert int(rec["extracted"].sum()) == st["extracted"]
                    assert int(rec["queued"].sum()) == st["queued"]
                    assert int(rec["edges"].sum()) == st["edges"]
                    # only a re-check step runs with an empty queue, and only last
                    assert np.all(rec["queued"][:-1] >= 1)
                    ended_with_recheck += int(rec["queued"][-1] == 0)
                # the wide shape runs every step unfused
                o = lib.make_options(flags=F, shape=lib.SSSP_SHAPE_WIDE, trace_ptr=trace.data_ptr(), trace_cap=cap)
                got, st = solve(lib, g, s, algo, param, opts=o, G=G)
                assert st["status"] == 0 and np.array_equal(got, want), (g.name, s, algo, param, "wide")
                rec = np.frombuffer(trace.cpu().numpy().tobytes(), dtype=np.dtype(lib.TRACE_DTYPE))[: st["steps"]]
                assert np.all(rec["queued"] >= 1)
        G.close()
    assert ended_with_recheck > 0


def test_rho_warmup_steps(lib):
    """rho-Stepping warm-up steps (the first steps at a small rho, without the
    dense-step reduction): distances equal the oracle's on power-law, grid and
    road-like graphs, in both layouts and shapes, with bidirectional, local
    relaxation and fused steps; a count without a rho (or the reverse) is
    refused."""
    sym = lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY
    graphs = [(gg.rmat(15, 16, gen_seed=51, wseed=52), sym | lib.SSSP_GRAPH_REORDER),
              (gg.rmat(14, 16, gen_seed=53, wseed=54), 0), (gg.grid(60, 70, wseed=55), sym),
              (gg.road(120, 0.75, seed=56), sym)]
    for g, gflags in graphs:
        G = lib.Graph(g, gflags)
        for s in gg.pick_sources(g, 2, 57):
            want = oracle.dijkstra(g, s)
            for ws, wr, red in ((1, 1, 0), (3, 16, 6), (6, 256, 6), (8, 256, 2), (50, 64, 0)):
                for kw in (dict(), dict(shape=lib.SSSP_SHAPE_NARROW), dict(local_budget=64),
                           dict(shape=lib.SSSP_SHAPE_NARROW, flags=lib.SSSP_SOLVE_FUSED, local_budget=256)):
                    kw = dict(kw)
                    if gflags & lib.SSSP_GRAPH_SYMMETRIC:
                        kw["flags"] = kw.get("flags", 0) | lib.SSSP_SOLVE_BIDIRECTIONAL
                    o = lib.make_options(rho_reduced=red, rho_warmup_steps=ws, rho_warmup=wr, **kw)
                    for rho in (64, max(64, g.n // 16)):
                        got, st = solve(lib, g, s, 0, rho, opts=o, G=G)
                        assert st["status"] == 0 and np.array_equal(got, want), (g.name, s, ws, wr, red, kw, rho)
        G.close()
    g = gg.grid(8, 8)
    G = lib.Graph(g)
    dist = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for kw in ({"rho_warmup_steps": 3}, {"rho_warmup": 64}):
        rc = lib.sssp_solve_ex(G.handle, 0, 0, 64, dist.data_ptr(), lib.make_options(**kw), 0, check=False)
        assert rc == lib.SSSP_ERR_INVALID_ARG, kw
    G.close()
