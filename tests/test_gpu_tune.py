"""The narrow kernel shape and the autotuner, through the C ABI.

Every configuration the autotuner can pick must give the oracle's distances
(they are unique), so the tests check the shape on the parity workloads and
then check that a tuned solve, a class-table lookup and a batched solve with
tuned parameters all still equal the oracle.
"""
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


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _solve(lib, G, n, s, algo, param, **kw):
    dist = torch.full((n,), 7, dtype=torch.int64, device="cuda")
    G.solve(s, algo, param, dist, _stream(), lib.make_options(**kw))
    st = G.stats(_stream())
    return dist.cpu().numpy().view(np.uint64).copy(), st


@pytest.mark.parametrize("algo,param", [(0, 1), (0, 1 << 10), (0, (1 << 32) - 1), (1, 1 << 13), (1, INF),
                                        (2, 0), (3, 1 << 13), (4, 0)])
def test_narrow_shape_matches_oracle_on_grid(lib, algo, param):
    g, s = gg.workload_grid256()
    want = oracle.dijkstra(g, s)
    G = lib.Graph(g)
    got, st = _solve(lib, G, g.n, s, algo, param, shape=lib.SSSP_SHAPE_NARROW)
    assert st["status"] == 0 and st["grid"] > 0
    assert np.array_equal(got, want)
    G.close()


def test_narrow_shape_rmat_road_hubs_bidir_local(lib):
    graphs = [gg.rmat(16, 16, gen_seed=11, wseed=12), gg.road(300, 0.75, seed=3)]
    # three vertices of degree 2e5 force multi-record chunk relaxation
    rng = np.random.default_rng(5)
    n = 200_003
    src = np.concatenate([np.full(n - 3, i) for i in range(3)] + [rng.integers(0, n, 4000)])
    dst = np.concatenate([np.arange(3, n) for _ in range(3)] + [rng.integers(0, n, 4000)])
    graphs.append(gg.from_edges(n, src, dst, rng.integers(1, 1000, src.size), "hubs"))
    for g in graphs:
        s = gg.pick_sources(g, 1, 5)[0] if g.name != "hubs" else 0
        want = oracle.dijkstra(g, s)
        G = lib.Graph(g)
        for algo, param in ((0, 1 << 12), (1, 1 << 15), (2, 0)):
            got, st = _solve(lib, G, g.n, s, algo, param, shape=lib.SSSP_SHAPE_NARROW)
            assert st["status"] == 0 and np.array_equal(got, want), (g.name, algo, param)
        G.close()
        if g.name != "hubs":
            Gs = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY)
            for kw in ({"flags": lib.SSSP_SOLVE_BIDIRECTIONAL}, {"local_budget": 256}):
                got, st = _solve(lib, Gs, g.n, s, 0, 1 << 12, shape=lib.SSSP_SHAPE_NARROW, **kw)
                assert st["status"] == 0 and np.array_equal(got, want), (g.name, kw)
            Gs.close()


def test_invalid_shape_is_rejected(lib):
    g, s = gg.workload_grid256()
    G = lib.Graph(g)
    dist = torch.empty(g.n, dtype=torch.int64, device="cuda")
    o = lib.make_options(shape=7)
    rc = lib._lib.sssp_solve_ex(G.handle, s, 0, 64, dist.data_ptr(), o, None)
    assert rc == lib.SSSP_ERR_INVALID_ARG
    G.close()


def test_autotune_then_solve_tuned(lib):
    cases = [gg.workload_grid256()[0], gg.rmat(14, 16, gen_seed=21, wseed=22), gg.road(120, 0.75, seed=9)]
    for g in cases:
        G = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY)
        srcs = gg.pick_sources(g, 3, 17)
        t = lib.sssp_autotune(G.handle, srcs, _stream())
        assert t["algo"] in (lib.SSSP_RHO, lib.SSSP_DELTA_STAR)
        assert t["param"] >= 1 and t["shape"] in (0, 1) and t["candidates"] >= 9 and t["ms"] > 0
        assert t["flags"] & lib.SSSP_SOLVE_BIDIRECTIONAL
        assert t["flags"] & ~(lib.SSSP_SOLVE_BIDIRECTIONAL | lib.SSSP_SOLVE_FUSED) == 0
        if t["flags"] & lib.SSSP_SOLVE_FUSED:  # fused steps are tried in the narrow shape only
            assert t["shape"] == lib.SSSP_SHAPE_NARROW and g.m / g.n < 20
        if g.m / g.n >= 20:
            assert t["local_budget"] == 0
        # the count of dense steps at rho/10 and the degree-bin cut-offs it chose
        assert t["rho_reduced"] in (0, 4, 6, 8, lib.SSSP_RHO_REDUCED_NONE)
        assert t["rho_reduced"] == 0 or t["algo"] == lib.SSSP_RHO
        assert t["small_deg"] in (0, 16, 64) and t["chunk"] in (0, 128, 512)
        assert lib.sssp_graph_get_tuning(G.handle) == t
        for s in srcs[:2]:
            dist = torch.full((g.n,), 7, dtype=torch.int64, device="cuda")
            lib.sssp_solve_tuned(G.handle, s, dist.data_ptr(), _stream())
            assert lib.sssp_last_status(G.handle, _stream()) == 0
            assert np.array_equal(dist.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s)), g.name
        G.close()


def test_class_table_serves_untuned_graphs_of_the_class(lib):
    a = gg.rmat(13, 16, gen_seed=31, wseed=32)
    b = gg.rmat(13, 16, gen_seed=33, wseed=34)
    Ga = lib.Graph(a, lib.SSSP_GRAPH_SYMMETRIC)
    Gb = lib.Graph(b, lib.SSSP_GRAPH_SYMMETRIC)
    if lib.sssp_graph_class(Ga.handle) != lib.sssp_graph_class(Gb.handle):
        pytest.skip("the two seeds gave graphs of different classes")
    t = lib.sssp_autotune(Ga.handle, gg.pick_sources(a, 2, 3), _stream())
    tb = lib.sssp_graph_get_tuning(Gb.handle)
    assert tb == t
    # batched solve with the tuned per-instance parameter (params = NULL)
    srcs = gg.pick_sources(b, 3, 4)
    outs = [torch.empty(b.n, dtype=torch.int64, device="cuda") for _ in srcs]
    lib.sssp_solve_multi([Gb.handle] * len(srcs), srcs, t["algo"], None, [o.data_ptr() for o in outs], _stream())
    st, _ = lib.sssp_batch_last_stats(len(srcs), _stream())
    assert st == 0
    for s, o in zip(srcs, outs):
        assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.dijkstra(b, s))
    # solve_tuned on the untuned graph uses the class entry
    dist = torch.empty(b.n, dtype=torch.int64, device="cuda")
    lib.sssp_solve_tuned(Gb.handle, srcs[0], dist.data_ptr(), _stream())
    assert np.array_equal(dist.cpu().numpy().view(np.uint64), oracle.dijkstra(b, srcs[0]))
    Ga.close()
    Gb.close()


def test_set_tuning_validation(lib):
    g, s = gg.workload_grid256()
    G = lib.Graph(g)  # not created symmetric
    good = {"algo": lib.SSSP_RHO, "param": 1024, "shape": lib.SSSP_SHAPE_NARROW, "flags": 0, "local_budget": 64}
    lib.sssp_graph_set_tuning(G.handle, good)
    assert lib.sssp_graph_get_tuning(G.handle)["param"] == 1024
    for bad in ({"param": 0}, {"shape": 2}, {"flags": lib.SSSP_SOLVE_BIDIRECTIONAL}, {"algo": 9},
                {"algo": lib.SSSP_BELLMAN_FORD, "local_budget": 64}, {"small_deg": 7}, {"small_deg": 200},
                {"chunk": 300}, {"chunk": 2048}, {"batch_mode": 3}):
        with pytest.raises(lib.SSSPError):
            lib.sssp_graph_set_tuning(G.handle, {**good, **bad})
    dist = torch.empty(g.n, dtype=torch.int64, device="cuda")
    lib.sssp_solve_tuned(G.handle, s, dist.data_ptr(), _stream())
    assert np.array_equal(dist.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s))
    G.close()


def test_autotune_restricted_to_one_rule(lib):
    g = gg.rmat(12, 16, gen_seed=41, wseed=42)
    G = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC)
    srcs = gg.pick_sources(g, 2, 5)
    t = lib.sssp_autotune_ex(G.handle, srcs, 1 << lib.SSSP_RHO, _stream())
    assert t["algo"] == lib.SSSP_RHO and t["candidates"] >= 5
    t = lib.sssp_autotune_ex(G.handle, srcs, 1 << lib.SSSP_DELTA_STAR, _stream())
    assert t["algo"] == lib.SSSP_DELTA_STAR
    for bad in (0, 1 << lib.SSSP_BELLMAN_FORD, 1 << 7):
        with pytest.raises(lib.SSSPError):
            lib.sssp_autotune_ex(G.handle, srcs, bad, _stream())
    G.close()


@pytest.mark.parametrize("algo,param", [(0, 2048), (1, 1 << 12)])
def test_batched_and_served_with_tuned_local_and_bidirectional_relaxation(lib, algo, param):
    """The batched and serving kernels take the graph's tuned bidirectional and
    local relaxation (local relaxation on graphs of >= 2^20 vertices: the
    1024^2 road-like grid); every instance still equals the oracle."""
    g = gg.road(1024, 0.75, seed=13)
    h = gg.rmat(13, 16, gen_seed=51, wseed=52)
    for x in (g, h):
        G = lib.Graph(x, lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY)
        lib.sssp_graph_set_tuning(G.handle, {"algo": algo, "param": param, "shape": 0,
                                             "flags": lib.SSSP_SOLVE_BIDIRECTIONAL, "local_budget": 256})
        srcs = gg.pick_sources(x, 4, 14)
        out = torch.empty(len(srcs) * x.n, dtype=torch.int64, device="cuda")
        lib.sssp_solve_sources(G.handle, srcs, algo, None, out.data_ptr(), _stream())
        st, stats = lib.sssp_batch_last_stats(len(srcs), _stream())
        assert st == 0
        got = out.view(len(srcs), x.n).cpu().numpy().view(np.uint64)
        for i, s in enumerate(srcs):
            assert np.array_equal(got[i], oracle.dijkstra(x, s)), (x.name, i)
        srv = lib.sssp_server_create(G.handle, slots=4, algo=algo, param=0)
        bufs = [torch.full((x.n,), 7, dtype=torch.int64, device="cuda") for _ in srcs]
        tickets = [lib.sssp_server_submit(srv, s, b.data_ptr()) for s, b in zip(srcs, bufs)]
        for tk, s, b in zip(tickets, srcs, bufs):
            info = lib.sssp_server_wait(srv, tk, 60_000_000_000)
            assert info["status"] == 0
            assert np.array_equal(b.cpu().numpy().view(np.uint64), oracle.dijkstra(x, s)), (x.name, s)
        lib.sssp_server_destroy(srv)
        G.close()


def test_autotune_batch_is_used_by_batched_calls(lib):
    g = gg.rmat(14, 16, gen_seed=61, wseed=62)
    G = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC)
    srcs = gg.pick_sources(g, 8, 15)
    single = lib.sssp_autotune(G.handle, srcs[:2], _stream())
    tb = lib.sssp_autotune_batch(G.handle, srcs, (1 << lib.SSSP_RHO) | (1 << lib.SSSP_DELTA_STAR), _stream())
    assert tb["algo"] in (lib.SSSP_RHO, lib.SSSP_DELTA_STAR) and tb["param"] >= 1 and tb["candidates"] >= 5
    assert tb["batch_mode"] in (lib.SSSP_BATCH_SHARED, lib.SSSP_BATCH_SEPARATE)
    assert lib.sssp_graph_get_tuning(G.handle) == single  # single-solve tuning unchanged
    out = torch.empty(len(srcs) * g.n, dtype=torch.int64, device="cuda")
    lib.sssp_solve_sources(G.handle, srcs, tb["algo"], None, out.data_ptr(), _stream())
    st, _ = lib.sssp_batch_last_stats(len(srcs), _stream())
    assert st == 0
    got = out.view(len(srcs), g.n).cpu().numpy().view(np.uint64)
    for i, s in enumerate(srcs):
        assert np.array_equal(got[i], oracle.dijkstra(g, s))
    with pytest.raises(lib.SSSPError):
        lib.sssp_autotune_batch(G.handle, srcs, 0, _stream())
    G.close()


def test_server_takes_the_tuned_slot_count(lib):
    g = gg.rmat(13, 16, gen_seed=71, wseed=72)
    G = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC)
    srcs = gg.pick_sources(g, 16, 16)
    tb = lib.sssp_autotune_batch(G.handle, srcs, 1 << lib.SSSP_RHO, _stream())
    assert tb["slots"] in (1, 4, 16)
    srv = lib.sssp_server_create(G.handle, slots=0, algo=tb["algo"], param=0)
    assert lib.sssp_server_slots(srv) == tb["slots"]
    bufs = [torch.empty(g.n, dtype=torch.int64, device="cuda") for _ in srcs[:6]]
    tickets = [lib.sssp_server_submit(srv, s, b.data_ptr()) for s, b in zip(srcs, bufs)]
    for tk, s, b in zip(tickets, srcs, bufs):
        assert lib.sssp_server_wait(srv, tk, 60_000_000_000)["status"] == 0
        assert np.array_equal(b.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s))
    lib.sssp_server_destroy(srv)
    G.close()


def test_tuned_solve_applies_every_recorded_choice(lib):
    """A tuning that sets the count of reduced dense steps, both degree-bin
    cut-offs or fused super-sparse steps is applied by sssp_solve_tuned (and by
    the class table) with the oracle's distances."""
    g = gg.rmat(15, 16, gen_seed=81, wseed=82)
    G = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_REORDER)
    for t in ({"algo": 0, "param": 1 << 11, "flags": 1, "rho_reduced": 8, "small_deg": 16, "chunk": 128},
              {"algo": 0, "param": 1 << 11, "flags": 1, "rho_reduced": lib.SSSP_RHO_REDUCED_NONE, "small_deg": 128,
               "chunk": 1024, "shape": 1},
              {"algo": 1, "param": 1 << 15, "flags": 0, "small_deg": 64, "chunk": 512, "local_budget": 64},
              {"algo": 1, "param": 1 << 13, "flags": 3, "shape": 1, "local_budget": 256}):  # + fused steps
        lib.sssp_graph_set_tuning(G.handle, t)
        for s in gg.pick_sources(g, 2, 19):
            dist = torch.full((g.n,), 7, dtype=torch.int64, device="cuda")
            lib.sssp_solve_tuned(G.handle, s, dist.data_ptr(), _stream())
            assert lib.sssp_last_status(G.handle, _stream()) == 0
            assert np.array_equal(dist.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s)), t
    G.close()
