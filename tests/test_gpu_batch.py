"""Batched solves (many sources on one graph; many graphs) through the C ABI:
every instance equals the CPU oracle, and a query's result is the same alone
(a single solve) and in the mix (a batched solve)."""
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


def _single(lib, G, n, s, algo, param):
    d = torch.empty(n, dtype=torch.int64, device="cuda")
    G.solve(s, algo, param, d, _stream())
    assert G.status(_stream()) == 0
    return d.cpu().numpy().view(np.uint64).copy()


@pytest.mark.parametrize("algo,param", [(0, 256), (0, 1 << 14), (1, 1 << 15), (2, 0), (0, None), (3, 1 << 15),
                                        (4, None)])
def test_sources_on_one_graph(lib, algo, param):
    g = gg.rmat(15, 16, gen_seed=31, wseed=32)
    srcs = gg.pick_sources(g, 24, 5) + [int(np.flatnonzero(gg.largest_cc(g) == 0)[0])]  # + an isolated vertex
    k = len(srcs)
    G = lib.Graph(g)
    out = torch.full((k * g.n,), 3, dtype=torch.int64, device="cuda")
    params = None if param is None else [param] * k
    lib.sssp_solve_sources(G.handle, srcs, algo, params, out.data_ptr(), _stream())
    st, stats = lib.sssp_batch_last_stats(k, _stream())
    assert st == 0
    got = out.cpu().numpy().view(np.uint64).reshape(k, g.n)
    for i, s in enumerate(srcs):
        assert np.array_equal(got[i], oracle.dijkstra(g, s)), (i, s)
        assert stats[i]["steps"] >= 1 and stats[i]["extracted"] >= 1
    # alone and in the mix: the batched result equals the single solve
    for i in (0, 7, k - 1):
        p_i = param if param is not None else max(64, g.n // 16) if algo == 0 else param
        if algo in (1, 3) and param is None:
            continue
        assert np.array_equal(got[i], _single(lib, G, g.n, srcs[i], algo, p_i if p_i else 0))
    G.close()


def test_many_graphs_of_uneven_size(lib):
    W = gg.workload_multi(count=48, lo_log2=6, hi_log2=14, seed=11)
    W.append((gg.from_edges(1, [], [], []), 0))                  # one vertex
    W.append((gg.chain(300, wseed=2, wlo=0, whi=(1 << 32) - 1), 0))
    W.append((gg.star(1000, wseed=3), 5))                        # isolated source
    W.append((gg.random_graph(500, 3000, 0, 3, seed=9), 1))
    Gs = [lib.Graph(g) for g, _ in W]
    outs = [torch.full((g.n,), 1, dtype=torch.int64, device="cuda") for g, _ in W]
    srcs = [s for _, s in W]
    for algo, params in ((0, [max(1, g.n // 8) for g, _ in W]), (1, [1 << 16] * len(W)), (2, None), (0, None),
                         (3, [1 << 15] * len(W)), (4, None)):
        lib.sssp_solve_multi([G.handle for G in Gs], srcs, algo, params, [o.data_ptr() for o in outs], _stream())
        st, stats = lib.sssp_batch_last_stats(len(W), _stream())
        assert st == 0
        for (g, s), o in zip(W, outs):
            assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s)), (g.name, algo)
    for G in Gs:
        G.close()


def test_repeated_batches_share_the_workspace(lib):
    g1 = gg.grid(60, 70, wseed=4)
    g2 = gg.rmat(13, 8, gen_seed=4, wseed=5)
    G1, G2 = lib.Graph(g1), lib.Graph(g2)
    for rep in range(3):
        k = [3, 40, 9][rep]
        srcs = gg.pick_sources(g2, k, rep)
        out = torch.empty(k * g2.n, dtype=torch.int64, device="cuda")
        lib.sssp_solve_sources(G2.handle, srcs, 0, [1 << 10] * k, out.data_ptr(), _stream())
        got = out.cpu().numpy().view(np.uint64).reshape(k, g2.n)
        for i in (0, k - 1):
            assert np.array_equal(got[i], oracle.dijkstra(g2, srcs[i]))
        o1 = torch.empty(g1.n, dtype=torch.int64, device="cuda")
        o2 = torch.empty(g2.n, dtype=torch.int64, device="cuda")
        lib.sssp_solve_multi([G1.handle, G2.handle], [0, srcs[0]], 2, None, [o1.data_ptr(), o2.data_ptr()],
                             _stream())
        assert np.array_equal(o1.cpu().numpy().view(np.uint64), oracle.dijkstra(g1, 0))
        assert np.array_equal(o2.cpu().numpy().view(np.uint64), oracle.dijkstra(g2, srcs[0]))
    G1.close()
    G2.close()


def test_batch_argument_errors(lib):
    g = gg.grid(8, 8)
    G = lib.Graph(g)
    out = torch.empty(4 * g.n, dtype=torch.int64, device="cuda")
    assert lib.sssp_solve_sources(G.handle, [], 0, None, out.data_ptr(), check=False) == lib.SSSP_ERR_INVALID_ARG
    assert lib.sssp_solve_sources(G.handle, [0, 64], 0, None, out.data_ptr(), check=False) == \
        lib.SSSP_ERR_INVALID_ARG
    assert lib.sssp_solve_sources(G.handle, [0, 1], 0, [5, 0], out.data_ptr(), check=False) == \
        lib.SSSP_ERR_INVALID_ARG
    assert lib.sssp_solve_sources(G.handle, list(range(64)) * 33, 0, None, out.data_ptr(), check=False) == \
        lib.SSSP_ERR_INVALID_ARG  # k > SSSP_MAX_BATCH
    G.close()


@pytest.mark.slow
def test_full_size_64_sources_rmat22(lib):
    """Batching, many sources: 64 sources on the RMAT scale-22 graph in one launch; every
    instance equals the single solve, four of them also the oracle."""
    g, _ = gg.workload_rmat(22)
    srcs = gg.pick_sources(g, 64, 6)
    G = lib.Graph(g)
    out = torch.empty(64 * g.n, dtype=torch.int64, device="cuda")
    lib.sssp_solve_sources(G.handle, srcs, 0, [1 << 18] * 64, out.data_ptr(), _stream())
    st, _ = lib.sssp_batch_last_stats(64, _stream())
    assert st == 0
    got = out.view(64, g.n)
    one = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for i, s in enumerate(srcs):
        G.solve(s, 0, 1 << 18, one, _stream())
        assert torch.equal(got[i], one), i
    host = got.cpu().numpy().view(np.uint64)
    for i in (0, 21, 42, 63):
        assert np.array_equal(host[i], oracle.dijkstra(g, srcs[i]))
    G.close()


@pytest.mark.slow
def test_full_size_512_graphs(lib):
    """Batching, many graphs: 512 graphs, n log-uniform in [2^10, 2^18], ~2^27 edges."""
    W = gg.workload_multi()
    Gs = [lib.Graph(g) for g, _ in W]
    outs = [torch.empty(g.n, dtype=torch.int64, device="cuda") for g, _ in W]
    lib.sssp_solve_multi([G.handle for G in Gs], [s for _, s in W], 0, None, [o.data_ptr() for o in outs],
                         _stream())
    st, _ = lib.sssp_batch_last_stats(len(W), _stream())
    assert st == 0
    for (g, s), o in zip(W, outs):
        assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s)), g.name
    for G in Gs:
        G.close()
