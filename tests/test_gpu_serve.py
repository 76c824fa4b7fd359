"""The query server (continuous batching): queries that arrive while others
run are admitted at the next step boundary and run alongside them; every
result equals the oracle and the single solve of the same source (the same
alone and in the mix); more queries than slots wait for a free slot; the
device loop exits when idle and restarts on the next query."""
import time

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


def _single(lib, G, n, s, algo, param):
    d = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    G.solve(s, algo, param, d, stream)
    assert G.status(stream) == 0
    return d.cpu().numpy().view(np.uint64).copy()


@pytest.mark.parametrize("mode", [1, 2])  # SSSP_BATCH_SHARED (one shared scan), SSSP_BATCH_SEPARATE
@pytest.mark.parametrize("algo,param", [(0, 2048), (1, 1 << 14), (2, 0)])
def test_overlapping_queries_equal_alone(lib, algo, param, mode):
    g = gg.road(200, 0.75, seed=3)                       # ~250 steps per query: queries overlap
    srcs = gg.pick_sources(g, 24, 17)
    G = lib.Graph(g)
    # gang=1: each query is admitted at the first step boundary after it
    # arrives (plain continuous batching; the shared-scan default waits for a
    # full gang, see test_gang_admission_of_the_shared_server)
    srv = lib.sssp_server_create(G.handle, slots=6, algo=algo, param=param, batch_mode=mode, gang=1)
    assert lib.sssp_server_mode(srv) == mode
    outs = [torch.full((g.n,), 9, dtype=torch.int64, device="cuda") for _ in srcs]
    torch.cuda.synchronize()
    tickets = []
    rng = np.random.default_rng(1)
    for s, o in zip(srcs, outs):
        tickets.append(lib.sssp_server_submit(srv, s, o.data_ptr()))
        time.sleep(float(rng.uniform(0, 0.002)))       # staggered arrivals
    infos = [lib.sssp_server_wait(srv, t, 60_000_000_000) for t in tickets]
    assert all(i["status"] == 0 and i["steps"] >= 1 for i in infos)
    for s, o in zip(srcs, outs):
        got = o.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, oracle.dijkstra(g, s))
    for j in (0, 11, 23):
        assert np.array_equal(outs[j].cpu().numpy().view(np.uint64), _single(lib, G, g.n, srcs[j], algo, param))
    # continuous batching: some query was admitted while another was running
    iv = sorted((i["device_admit_ns"], i["device_done_ns"]) for i in infos)
    joined = any(iv[b][0] > iv[a][0] and iv[b][0] < iv[a][1] for a in range(len(iv)) for b in range(a + 1, len(iv)))
    assert joined
    lib.sssp_server_destroy(srv)
    G.close()


@pytest.mark.parametrize("mode", [1, 2])
def test_backpressure_idle_restart_and_destroy(lib, mode):
    g = gg.rmat(14, 16, gen_seed=41, wseed=42)
    srcs = gg.pick_sources(g, 40, 3)
    G = lib.Graph(g)
    srv = lib.sssp_server_create(G.handle, slots=4, algo=0, param=1 << 10, idle_ns=1_000_000, batch_mode=mode)
    assert lib.sssp_server_slots(srv) == 4
    outs = [torch.empty(g.n, dtype=torch.int64, device="cuda") for _ in srcs]
    torch.cuda.synchronize()
    tickets = [lib.sssp_server_submit(srv, s, o.data_ptr()) for s, o in zip(srcs, outs)]  # 10x the slots
    for t in tickets:
        assert lib.sssp_server_wait(srv, t)["status"] == 0
    for s, o in list(zip(srcs, outs))[::7]:
        assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s))
    launches = lib.sssp_server_stats(srv)["launches"]
    time.sleep(0.05)                                    # > idle: the device loop exits
    t = lib.sssp_server_submit(srv, srcs[0], outs[0].data_ptr())
    assert lib.sssp_server_wait(srv, t)["status"] == 0
    assert lib.sssp_server_stats(srv)["launches"] > launches
    assert np.array_equal(outs[0].cpu().numpy().view(np.uint64), oracle.dijkstra(g, srcs[0]))
    # poll interface, then destroy with queries still queued
    t = lib.sssp_server_submit(srv, srcs[1], outs[1].data_ptr())
    while lib.sssp_server_poll(srv, t) is None:
        time.sleep(0.0005)
    for s, o in zip(srcs[:12], outs[:12]):
        lib.sssp_server_submit(srv, s, o.data_ptr())
    lib.sssp_server_destroy(srv)
    # the context is still usable
    assert np.array_equal(_single(lib, G, g.n, srcs[2], 2, 0), oracle.dijkstra(g, srcs[2]))
    G.close()


def test_shared_server_relabelled_graph_and_wide_slots(lib):
    """The shared-scan server on a degree-ordered symmetric graph with
    bidirectional relaxation (batch tuning) and all 64 slots: every query of
    a stream twice the slot count equals the oracle; repeated sources; a
    Delta-Stepping server falls back to separate instances."""
    g = gg.rmat(15, 16, gen_seed=43, wseed=44)
    G = lib.Graph(g, lib.SSSP_GRAPH_SYMMETRIC | lib.SSSP_GRAPH_VERIFY | lib.SSSP_GRAPH_REORDER)
    lib.sssp_graph_set_tuning(G.handle, {"algo": 0, "param": 1 << 11, "flags": 1, "rho_reduced": 6})
    srv = lib.sssp_server_create(G.handle, slots=64, algo=0, param=1 << 11)
    assert lib.sssp_server_mode(srv) == lib.SSSP_BATCH_SHARED and lib.sssp_server_slots(srv) == 64
    srcs = gg.pick_sources(g, 128, 5)
    srcs[7] = srcs[3]
    outs = [torch.full((g.n,), 1, dtype=torch.int64, device="cuda") for _ in srcs]
    torch.cuda.synchronize()
    tickets = [lib.sssp_server_submit(srv, s, o.data_ptr()) for s, o in zip(srcs, outs)]
    for t in tickets:
        assert lib.sssp_server_wait(srv, t, 60_000_000_000)["status"] == 0
    for s, o in zip(srcs, outs):
        assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s)), s
    lib.sssp_server_destroy(srv)
    srv = lib.sssp_server_create(G.handle, slots=4, algo=3, param=1 << 12)
    assert lib.sssp_server_mode(srv) == lib.SSSP_BATCH_SEPARATE
    t = lib.sssp_server_submit(srv, srcs[0], outs[0].data_ptr())
    assert lib.sssp_server_wait(srv, t)["status"] == 0
    assert np.array_equal(outs[0].cpu().numpy().view(np.uint64), oracle.dijkstra(g, srcs[0]))
    lib.sssp_server_destroy(srv)
    G.close()


def test_gang_admission_of_the_shared_server(lib):
    """The shared-scan server's default admits waiting queries as a gang (every
    slot holds one, nothing else runs, or the oldest waited gang_wait_ns), so
    queries that start together stay aligned; results equal the oracle, a
    burst of 3x the slots is admitted in gangs that start at the same device
    time, and a query arriving while a gang runs still starts once
    gang_wait_ns has passed."""
    g = gg.road(160, 0.75, seed=6)
    srcs = gg.pick_sources(g, 24, 21)
    G = lib.Graph(g)
    srv = lib.sssp_server_create(G.handle, slots=8, algo=1, param=1 << 13, batch_mode=lib.SSSP_BATCH_SHARED)
    outs = [torch.full((g.n,), 5, dtype=torch.int64, device="cuda") for _ in srcs]
    torch.cuda.synchronize()
    tickets = [lib.sssp_server_submit(srv, s, o.data_ptr()) for s, o in zip(srcs, outs)]
    infos = [lib.sssp_server_wait(srv, t, 60_000_000_000) for t in tickets]
    assert all(i["status"] == 0 for i in infos)
    for s, o in zip(srcs, outs):
        assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s))
    admits = sorted({i["device_admit_ns"] // 100_000 for i in infos})   # 0.1 ms bins
    assert len(admits) <= 6, admits                                     # gangs, not 24 single admissions
    lib.sssp_server_destroy(srv)
    # a short wait lets a late query join a running gang
    srv = lib.sssp_server_create(G.handle, slots=8, algo=1, param=1 << 13, batch_mode=lib.SSSP_BATCH_SHARED,
                                 gang_wait_ns=200_000)
    t0 = lib.sssp_server_submit(srv, srcs[0], outs[0].data_ptr())
    time.sleep(0.001)
    t1 = lib.sssp_server_submit(srv, srcs[1], outs[1].data_ptr())
    i0, i1 = lib.sssp_server_wait(srv, t0), lib.sssp_server_wait(srv, t1)
    assert i0["status"] == 0 and i1["status"] == 0
    assert i1["device_admit_ns"] < i0["device_done_ns"], (i0, i1)     # joined while the first ran
    for s, o in zip(srcs[:2], outs[:2]):
        assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.dijkstra(g, s))
    lib.sssp_server_destroy(srv)
    G.close()
