"""Single solves on a graph created with SSSP_GRAPH_REORDER (the device copy is
relabelled by decreasing degree; distances come back in the caller's ids),
against the oracle on the caller's graph, through the C ABI."""
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


def _s():
    return torch.cuda.current_stream().cuda_stream


def _solve(lib, G, n, s, algo, param, **kw):
    dist = torch.full((n,), 7, dtype=torch.int64, device="cuda")
    G.solve(s, algo, param, dist, _s(), lib.make_options(**kw))
    st = G.stats(_s())
    return dist.cpu().numpy().view(np.uint64).copy(), st


@pytest.mark.parametrize("shape", [0, 1])
def test_reordered_grid_all_rules(lib, shape):
    g, s = gg.workload_grid256()
    want = oracle.dijkstra(g, s)
    G = lib.Graph(g, lib.SSSP_GRAPH_REORDER)
    for algo, param in [(0, 1), (0, 1 << 10), (0, (1 << 32) - 1), (1, 1 << 13), (1, INF), (2, 0), (3, 1 << 13), (4, 0)]:
        got, st = _solve(lib, G, g.n, s, algo, param, shape=shape)
        assert st["status"] == 0 and np.array_equal(got, want), (algo, param)
    G.close()


def test_reordered_rmat_road_hubs_edge_cases(lib):
    rng = np.random.default_rng(8)
    n = 100_003
    src = np.concatenate([np.full(n - 3, i) for i in range(3)] + [rng.integers(0, n, 4000)])
    dst = np.concatenate([np.arange(3, n) for _ in range(3)] + [rng.integers(0, n, 4000)])
    graphs = [gg.rmat(16, 16, gen_seed=11, wseed=12), gg.road(300, 0.75, seed=3),
              gg.from_edges(n, src, dst, rng.integers(0, 1000, src.size), "hubs"),
              gg.from_edges(5, [0, 0, 1, 1, 3], [1, 1, 1, 2, 4], [5, 3, 0, 2 ** 32 - 1, 7], "multi_selfloop"),
              gg.chain(3000, wseed=4)]
    for g in graphs:
        for s in (gg.pick_sources(g, 2, 5) if g.name not in ("hubs", "multi_selfloop") else [0, 3]):
            want = oracle.dijkstra(g, s)
            G = lib.Graph(g, lib.SSSP_GRAPH_REORDER)
            for algo, param in ((0, 1 << 12), (1, 1 << 15), (2, 0)):
                got, st = _solve(lib, G, g.n, s, algo, param)
                assert st["status"] == 0 and np.array_equal(got, want), (g.name, s, algo)
            G.close()


def test_reordered_symmetric_bidirectional_local_and_counters(lib):
    g = gg.rmat(15, 16, gen_seed=21, wseed=22)
    s = gg.pick_sources(g, 1, 7)[0]
    want = oracle.dijkstra(g, s)
    h, depth = oracle.hops(g, s)
    G = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY | lib.SSSP_GRAPH_REORDER)
    for kw in ({"flags": lib.SSSP_SOLVE_BIDIRECTIONAL}, {"local_budget": 256}):
        got, st = _solve(lib, G, g.n, s, 0, 1 << 10, **kw)
        assert st["status"] == 0 and np.array_equal(got, want), kw
    # Lemma 5.1 on the per-vertex extraction counters, reported in the caller's ids
    ext = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    got, st = _solve(lib, G, g.n, s, 2, 0, ext_count_ptr=ext.data_ptr())
    cnt = ext.cpu().numpy().view(np.uint32)
    reach = want != np.uint64(INF)
    assert np.array_equal(got, want)
    assert np.all(cnt[reach] <= np.maximum(h[reach], 1)) and np.all(cnt[~reach] == 0)
    assert int(cnt.sum()) == st["extracted"]
    # host output and the tuned solve on the relabelled graph
    host = np.empty(g.n, np.uint64)
    lib.sssp_solve_host(G.handle, s, 0, 1 << 12, host, _s())
    assert np.array_equal(host, want)
    G.close()
