"""sssp_solve_noalloc: the solve for callers that cannot allocate device memory
when they need a solve (a plugin inside a framework that owns all device
memory through its own pool, a latency-critical loop that cannot take the
device synchronisation of cudaMalloc/cudaFree).  It takes the graph already on
the device and uses a static scratch array instead of allocating.  Its output
must equal the regular entry point's and the oracle's (bit-exact uint64
distances) on consecutive calls that share the scratch array, and a call after
the first must not change the device's free memory.  This file is collected
last on purpose."""
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


def _device_csr(g):
    """Caller-side device copies: offsets and interleaved (target, weight) pairs,
    padded to an even number of pairs as the entry point requires."""
    m_even = g.m + (g.m & 1)
    pairs = np.zeros((max(m_even, 2), 2), dtype=np.uint32)
    pairs[: g.m, 0] = g.tgt
    pairs[: g.m, 1] = g.w
    off = torch.from_numpy(g.off.view(np.int64).copy()).cuda()
    edges = torch.from_numpy(pairs.view(np.int32).copy()).cuda()
    assert edges.data_ptr() % 16 == 0
    return off, edges


def _regular(lib, g, s, algo, param):
    G = lib.Graph(g)
    d = torch.empty(g.n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    G.solve(s, algo, param, d, stream)
    assert G.status(stream) == 0
    out = d.cpu().numpy().view(np.uint64).copy()
    G.close()
    return out


def _noalloc(lib, g, s, algo, param, dev_csr):
    off, edges = dev_csr
    d = torch.full((g.n,), 3, dtype=torch.int64, device="cuda")
    stats = torch.zeros(lib.STATS_BYTES // 8, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lib.sssp_solve_noalloc(g.n, g.m, off.data_ptr(), edges.data_ptr(), s, algo, param, d.data_ptr(),
                           stats.data_ptr(), stream)
    torch.cuda.synchronize()
    st = stats.cpu().numpy().view(np.uint64)
    status = int(np.int32(st[5] & np.uint64(0xFFFFFFFF)))
    return d.cpu().numpy().view(np.uint64).copy(), status, int(st[0])


def test_noalloc_matches_regular_entry_on_consecutive_calls(lib):
    cases = [
        (gg.rmat(14, 16, gen_seed=21, wseed=22), lib.SSSP_RHO, 1 << 10),
        (gg.grid(200, 300, wseed=4), lib.SSSP_DELTA_STAR, 1 << 15),   # different n: stale scratch
        (gg.rmat(14, 16, gen_seed=21, wseed=22), lib.SSSP_BELLMAN_FORD, 0),
    ]
    for g, algo, param in cases:
        s = gg.pick_sources(g, 1, 9)[0]
        want = _regular(lib, g, s, algo, param)
        assert np.array_equal(want, oracle.dijkstra(g, s)), (g.name, algo, param)
        dev = _device_csr(g)
        for call in range(2):  # two calls in a row share the scratch array
            got, status, steps = _noalloc(lib, g, s, algo, param, dev)
            assert status == 0 and steps >= 1
            assert np.array_equal(got, want), (g.name, algo, param, call)


def test_noalloc_call_takes_no_device_memory(lib):
    """After the first call (the one-time set-up) a call changes neither the
    device's free memory nor its result."""
    g = gg.rmat(13, 16, gen_seed=5, wseed=6)
    s = gg.pick_sources(g, 1, 3)[0]
    want = oracle.dijkstra(g, s)
    dev = _device_csr(g)
    d = torch.empty(g.n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lib.sssp_solve_noalloc(g.n, g.m, dev[0].data_ptr(), dev[1].data_ptr(), s, lib.SSSP_RHO, 256, d.data_ptr(),
                           0, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        d.fill_(0)
        lib.sssp_solve_noalloc(g.n, g.m, dev[0].data_ptr(), dev[1].data_ptr(), s, lib.SSSP_RHO, 256,
                               d.data_ptr(), 0, stream)
        torch.cuda.synchronize()
        assert np.array_equal(d.cpu().numpy().view(np.uint64), want)
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_rejects_sizes_beyond_its_maximum(lib):
    dummy = torch.zeros(4, dtype=torch.int64, device="cuda")
    p = dummy.data_ptr()
    big_n = lib.NOALLOC_MAX_VERTICES + 1
    assert lib.sssp_solve_noalloc(big_n, 0, p, p, 0, 0, 1, p, 0, 0, check=False) == lib.SSSP_ERR_INVALID_ARG
    assert lib.sssp_solve_noalloc(8, lib.NOALLOC_MAX_EDGES + 1, p, p, 0, 0, 1, p, 0, 0,
                                  check=False) == lib.SSSP_ERR_INVALID_ARG
    assert lib.sssp_solve_noalloc(8, 2, p, p + 8, 0, 0, 1, p, 0, 0, check=False) == \
        lib.SSSP_ERR_INVALID_ARG  # edges not 16-byte aligned
