"""Batched solves of many sources on one graph with one shared edge scan per
step (SSSP_BATCH_SHARED): vertex-major distances, one union queue with an
instance mask per vertex, records that carry the mask of the instances that
extracted the vertex.  Every instance must equal the CPU oracle element by
element, for every rule it supports, instance counts from 1 to 64 (row
padding), repeated sources, per-instance parameters, graphs with hubs and
isolated vertices, and the degree-ordered graph copy."""
import numpy as np
import pytest

import oracle
from paper_2105_06145_gb300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2105_06145_gb300 import sssp
    return sssp


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _hub_graph(n=40000, seed=23):
    rng = np.random.default_rng(seed)
    s, d, w = [], [], []
    for h in (0, 1, 2):
        t = rng.integers(0, n, 3000)
        ww = rng.integers(1, 1 << 18, t.size)
        s += [np.full(t.size, h), t]; d += [t, np.full(t.size, h)]; w += [ww, ww]
    a, b = rng.integers(0, n, 3 * n), rng.integers(0, n, 3 * n)
    ww = rng.integers(1, 1 << 18, a.size)
    s += [a, b]; d += [b, a]; w += [ww, ww]
    return gg.from_edges(n, np.concatenate(s), np.concatenate(d), np.concatenate(w), name="hubs")


def _run(lib, G, g, srcs, algo, params, mode):
    k = len(srcs)
    out = torch.full((k * g.n,), 5, dtype=torch.int64, device="cuda")
    lib.sssp_solve_sources_ex(G.handle, srcs, algo, params, mode, out.data_ptr(), _stream())
    st, stats = lib.sssp_batch_last_stats(k, _stream())
    assert st == 0, st
    return out.cpu().numpy().view(np.uint64).reshape(k, g.n), stats


@pytest.mark.parametrize("flags", [0, 4])  # caller's order, degree-ordered copy (SSSP_GRAPH_REORDER)
def test_shared_scan_equals_oracle(lib, flags):
    graphs = [gg.grid(60, 70, wseed=3), gg.rmat(14, 16, gen_seed=5, wseed=6), _hub_graph(),
              gg.road(90, 0.75, seed=2), gg.random_graph(5000, 9000, 0, 7, seed=8)]
    for g in graphs:
        G = lib.Graph(g, flags)
        oracle_cache = {}

        def want(s):
            if s not in oracle_cache:
                oracle_cache[s] = oracle.dijkstra(g, s)
            return oracle_cache[s]
        base = gg.pick_sources(g, 64, 13)
        for k in (1, 2, 3, 5, 17, 33, 64):
            srcs = list(base[:k])
            if k >= 3:
                srcs[2] = srcs[0]  # a repeated source
            for algo, params in ((0, [64] * k), (0, [max(64, g.n // (4 + i)) for i in range(k)]),
                                 (1, [1 << (10 + i % 8) for i in range(k)]), (2, None), (0, None), (1, None)):
                if k not in (3, 33, 64) and params is None:
                    continue
                got, stats = _run(lib, G, g, srcs, algo, params, lib.SSSP_BATCH_SHARED)
                for i, s in enumerate(srcs):
                    assert np.array_equal(got[i], want(s)), (g.name, flags, k, algo, i, s)
                    assert stats[i]["steps"] >= 1 and stats[i]["extracted"] >= 1
        G.close()


def test_shared_scan_matches_separate_and_single(lib):
    """The shared scan, the separate-instance kernel and single solves give the
    same distances; the automatic mode picks one of them."""
    g = gg.rmat(16, 16, gen_seed=9, wseed=10)
    G = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_REORDER)
    srcs = gg.pick_sources(g, 40, 3)
    a, _ = _run(lib, G, g, srcs, 0, None, lib.SSSP_BATCH_SHARED)
    b, _ = _run(lib, G, g, srcs, 0, None, lib.SSSP_BATCH_SEPARATE)
    c, _ = _run(lib, G, g, srcs, 0, None, lib.SSSP_BATCH_AUTO)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    d = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for i in (0, 19, 39):
        G.solve(srcs[i], 0, max(64, g.n // 16), d, _stream())
        assert np.array_equal(d.cpu().numpy().view(np.uint64), a[i])
    G.close()


def test_shared_scan_refuses_what_it_does_not_cover(lib):
    g = gg.grid(16, 16)
    G = lib.Graph(g)
    out = torch.empty(65 * g.n, dtype=torch.int64, device="cuda")
    srcs = list(range(65))
    assert lib.sssp_solve_sources_ex(G.handle, srcs, 0, None, lib.SSSP_BATCH_SHARED, out.data_ptr(), 0,
                                     check=False) == lib.SSSP_ERR_INVALID_ARG      # k > 64
    for algo in (3, 4):  # Delta-Stepping with FinishCheck, Dijkstra: separate instances only
        assert lib.sssp_solve_sources_ex(G.handle, srcs[:4], algo, [64] * 4 if algo == 3 else None,
                                         lib.SSSP_BATCH_SHARED, out.data_ptr(), 0,
                                         check=False) == lib.SSSP_ERR_INVALID_ARG
    assert lib.sssp_solve_sources_ex(G.handle, srcs[:4], 0, None, 7, out.data_ptr(), 0,
                                     check=False) == lib.SSSP_ERR_INVALID_ARG       # unknown mode
    # the automatic mode falls back to separate instances for k > 64
    lib.sssp_solve_sources_ex(G.handle, srcs, 0, None, lib.SSSP_BATCH_AUTO, out.data_ptr(), _stream())
    got = out.cpu().numpy().view(np.uint64).reshape(65, g.n)
    for i in (0, 64):
        assert np.array_equal(got[i], oracle.dijkstra(g, i))
    G.close()


def test_shared_scan_64_sources_rmat22(lib):
    """The batching workload at full size: 64 sources on RMAT scale 22 in one
    shared-scan launch on the degree-ordered copy; every instance equals its
    single solve, and three equal the oracle."""
    g, _ = gg.workload_rmat(22)
    srcs = gg.pick_sources(g, 64, 6)
    G = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_REORDER)
    out = torch.empty(64 * g.n, dtype=torch.int64, device="cuda")
    lib.sssp_solve_sources_ex(G.handle, srcs, 0, [1 << 18] * 64, lib.SSSP_BATCH_SHARED, out.data_ptr(), _stream())
    st, _ = lib.sssp_batch_last_stats(64, _stream())
    assert st == 0
    rows = out.view(64, g.n)
    one = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for i, s in enumerate(srcs):
        G.solve(s, 0, 1 << 18, one, _stream())
        assert torch.equal(rows[i], one), (i, s)
    for i in (0, 31, 63):
        assert np.array_equal(rows[i].cpu().numpy().view(np.uint64), oracle.dijkstra(g, srcs[i]))
    G.close()


def test_shared_scan_bidirectional(lib):
    """With a batch tuning that asks for bidirectional relaxation on a graph
    declared (and verified) symmetric, the shared scan also pulls into the
    extracted vertex before it pushes; distances unchanged."""
    flags = lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY
    for g in (gg.grid(70, 80, wseed=4), gg.rmat(15, 16, gen_seed=7, wseed=8), _hub_graph(30000, 5)):
        for extra in (0, lib.SSSP_GRAPH_REORDER):
            G = lib.Graph(g, flags | extra)
            srcs = gg.pick_sources(g, 37, 21)
            for algo, param in ((0, 256), (0, max(64, g.n // 16)), (1, 1 << 14), (2, 0)):
                lib.sssp_graph_set_tuning(G.handle, {"algo": algo, "param": param, "flags": 1, "batch_mode": 1,
                                                     "rho_reduced": 6})
                got, stats = _run(lib, G, g, srcs, algo, None, lib.SSSP_BATCH_AUTO)
                for i, s in enumerate(srcs):
                    assert np.array_equal(got[i], oracle.dijkstra(g, s)), (g.name, extra, algo, i)
            G.close()


def test_shared_scan_warmup_steps(lib):
    """rho-Stepping warm-up steps in the shared scan (each instance's first
    steps at a small rho, counted per instance, so that queries admitted to
    the server at different steps each get their own): every instance of a
    batch and every served query equals the oracle."""
    flags = lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY
    for g, extra in ((gg.rmat(15, 16, gen_seed=61, wseed=62), lib.SSSP_GRAPH_REORDER), (_hub_graph(30000, 9), 0),
                     (gg.grid(50, 60, wseed=63), 0)):
        G = lib.Graph(g, flags | extra)
        srcs = gg.pick_sources(g, 37, 64)
        for ws, wr, red in ((8, 256, 4), (3, 16, 0), (40, 1, 6)):
            lib.sssp_graph_set_tuning(G.handle, {"algo": 0, "param": max(64, g.n // 16), "flags": 1,
                                                 "batch_mode": lib.SSSP_BATCH_SHARED, "rho_reduced": red,
                                                 "rho_warmup_steps": ws, "rho_warmup": wr})
            got, _ = _run(lib, G, g, srcs, 0, None, lib.SSSP_BATCH_AUTO)
            for i, s in enumerate(srcs):
                assert np.array_equal(got[i], oracle.dijkstra(g, s)), (g.name, ws, wr, red, i)
        # the server: queries admitted one by one (continuous admission)
        srv = lib.sssp_server_create(G.handle, slots=8, algo=0, param=max(64, g.n // 16),
                                     batch_mode=lib.SSSP_BATCH_SHARED, gang=1)
        outs = [torch.full((g.n,), 3, dtype=torch.int64, device="cuda") for _ in srcs[:16]]
        torch.cuda.synchronize()
        tickets = [lib.sssp_server_submit(srv, s, o.data_ptr()) for s, o in zip(srcs[:16], outs)]
        for t in tickets:
            assert lib.sssp_server_wait(srv, t, 60_000_000_000)["status"] == 0
        for s, o in zip(srcs[:16], outs):
            assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s)), (g.name, s)
        lib.sssp_server_destroy(srv)
        G.close()
