"""Full-size parity: the power-law (RMAT scale 22) and road-like (4096^2)
workloads, in the launch configuration the benchmark times, compared element
by element with the CPU oracle's Dijkstra (which finishes in seconds)."""
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


def _run(lib, g, sources, cases, flags=0, opts=None):
    G = lib.Graph(g, flags)
    dist = torch.empty(g.n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for s in sources:
        want = oracle.dijkstra(g, s)
        assert oracle.check(g, s, want)[0] == 0
        for algo, param in cases:
            dist.fill_(0)
            G.solve(s, algo, param, dist, stream, opts)
            st = G.stats(stream)
            assert st["status"] == 0, (algo, param, st)
            got = dist.cpu().numpy().view(np.uint64)
            assert np.array_equal(got, want), (g.name, s, algo, param)
    G.close()


def test_rmat22_all_rules(lib):
    g, s = gg.workload_rmat(22)
    extra = gg.pick_sources(g, 3, 77)
    cases = [(0, 1 << 18), (0, 1 << 20), (0, 1 << 22), (1, 1 << 13), (1, 1 << 15), (1, 1 << 17), (2, 0),
             (3, 1 << 15), (4, 0)]
    _run(lib, g, [s], cases)
    _run(lib, g, extra, [(0, 1 << 20)])
    # the benchmark's launch configuration: relabelled symmetric graph,
    # bidirectional relaxation, wide shape, rho in the sweep
    bench_flags = lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_REORDER
    bidir = lib.make_options(flags=lib.SSSP_SOLVE_BIDIRECTIONAL)
    _run(lib, g, [s] + extra, [(0, 1 << 18), (0, 1 << 20), (0, 1 << 22), (1, 1 << 15), (2, 0)], bench_flags, bidir)
    # ... with the benchmark's count of dense steps that use rho/10 (6) and
    # the autotuner's other choices of the count and of the degree cut-offs
    for red, sd, ch in ((6, 0, 0), (4, 64, 512), (8, 16, 128)):
        o = lib.make_options(flags=lib.SSSP_SOLVE_BIDIRECTIONAL, rho_reduced=red, small_deg=sd, chunk=ch)
        _run(lib, g, [s] + extra, [(0, 1 << 18), (0, 1 << 19)], bench_flags, o)
    # ... and the benchmark's warm-up steps (8 steps at rho = 256, then 4
    # dense steps at rho/10), and others
    for ws, wr, red in ((8, 256, 4), (6, 256, 6), (4, 1024, 2)):
        o = lib.make_options(flags=lib.SSSP_SOLVE_BIDIRECTIONAL, rho_reduced=red, rho_warmup_steps=ws, rho_warmup=wr)
        _run(lib, g, [s] + extra, [(0, 1 << 18)], bench_flags, o)


def test_road4096(lib):
    g, s = gg.workload_road(4096)
    assert g.n == 4096 * 4096
    _run(lib, g, [s], [(0, 1 << 20), (0, 1 << 14), (1, 1 << 13), (1, 1 << 15), (3, 1 << 13)])
    # the tuned road configuration: Delta*-Stepping with local relaxation in the narrow shape
    opts = lib.make_options(flags=lib.SSSP_SOLVE_BIDIRECTIONAL, local_budget=256, shape=lib.SSSP_SHAPE_NARROW)
    _run(lib, g, [s], [(1, 2111), (0, 1 << 16)], lib.SSSP_GRAPH_SYMMETRIC, opts)
    # ... with fused super-sparse steps, and a second source
    extra = gg.pick_sources(g, 1, 31, mask=gg.largest_cc(g))
    for lb in (256, 1024):
        opts = lib.make_options(flags=lib.SSSP_SOLVE_BIDIRECTIONAL | lib.SSSP_SOLVE_FUSED, local_budget=lb,
                                shape=lib.SSSP_SHAPE_NARROW)
        _run(lib, g, [s] + extra, [(1, 2111), (0, 1 << 16)], lib.SSSP_GRAPH_SYMMETRIC, opts)
