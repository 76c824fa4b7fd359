"""The device tournament-tree LaB-PQ (Sec. 4.2, Algorithm 2) and the stand-alone
array Extract (Sec. 4.3), through the C ABI, against the oracle's plain-set
LaB-PQ (Sec. 3.1).

Extract's output is a set (the device order is arbitrary), so each comparison
sorts both sides; Reduce (min) and the inQ flags are compared exactly.
"""
import numpy as np
import pytest

import oracle

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


def _u64(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).cuda()


def _u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


class Tree:
    def __init__(self, lib, n):
        self.lib, self.n = lib, n
        self.h = lib.sssp_tourney_create(n)
        self.out = torch.zeros(n, dtype=torch.int32, device="cuda")
        self.cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.mn = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.inq = torch.zeros((n + 31) // 32, dtype=torch.int32, device="cuda")

    def update(self, ids):
        d = _u32(ids)
        self.lib.sssp_tourney_update(self.h, d.data_ptr(), int(d.numel()), _s())

    def extract(self, keys_dev, theta):
        self.lib.sssp_tourney_extract(self.h, keys_dev.data_ptr(), theta, self.out.data_ptr(), self.cnt.data_ptr(),
                                      _s())
        c = int(self.cnt.item())
        return np.sort(self.out[:c].cpu().numpy().view(np.uint32))

    def min(self, keys_dev):
        self.lib.sssp_tourney_min(self.h, keys_dev.data_ptr(), self.mn.data_ptr(), _s())
        return int(self.mn.cpu().numpy().view(np.uint64)[0])

    def inq_flags(self):
        self.lib.sssp_tourney_inq(self.h, self.inq.data_ptr(), _s())
        w = self.inq.cpu().numpy().view(np.uint32)
        return ((w[np.arange(self.n) >> 5] >> (np.arange(self.n) & 31)) & 1).astype(np.uint8)

    def close(self):
        self.lib.sssp_tourney_destroy(self.h)


def test_the_papers_example(lib):
    key = np.array([3, 8, 4, 6, 1, 5], np.uint64)
    t = Tree(lib, 6)
    kd = _u64(key)
    assert t.min(kd) == INF
    t.update(range(6))
    assert t.min(kd) == 1
    assert sorted(key[t.extract(kd, 4)].tolist()) == [1, 3, 4]
    assert t.min(kd) == 5
    assert t.extract(kd, 4).size == 0
    t.close()


@pytest.mark.parametrize("n", [1, 2, 3, 1000, 65537, 300001])
def test_random_batches_against_the_plain_set(lib, n):
    """Interleaved batches as Algorithm 1 issues them: keys only decrease,
    every decrease is followed by an update of the record, extracts with
    thresholds at several quantiles, Reduce in between."""
    rng = np.random.default_rng(n)
    key = rng.integers(1, 1 << 40, n).astype(np.uint64)
    inq = np.zeros(n, np.uint8)
    t = Tree(lib, n)
    for rnd in range(12):
        b = int(rng.integers(1, max(2, n // 3) + 1))
        ids = rng.integers(0, n, b).astype(np.uint32)
        dec = rng.random(b) < 0.5
        key[ids[dec]] = np.minimum(key[ids[dec]], rng.integers(1, 1 << 40, int(dec.sum())).astype(np.uint64))
        inq[ids] = 1
        kd = _u64(key)
        t.update(np.concatenate([ids, [n + 5, n]]).astype(np.uint32))  # ids >= n are ignored
        assert t.min(kd) == oracle.lbpq_min(inq, key)
        q = np.flatnonzero(inq)
        theta = int(np.quantile(key[q], rng.choice([0.0, 0.1, 0.5, 0.9]))) if q.size else 0
        if rnd == 7:
            theta = INF
        want = oracle.lbpq_extract(inq, key, theta)
        got = t.extract(kd, theta)
        assert np.array_equal(got, want), (n, rnd)
        assert np.array_equal(t.inq_flags(), inq)
    t.close()


def test_array_extract_matches_the_plain_set(lib):
    rng = np.random.default_rng(9)
    n = 200_000
    key = rng.integers(0, 1 << 30, n).astype(np.uint64)
    lst = rng.permutation(n)[: n // 2].astype(np.uint32)
    kd, ld = _u64(key), _u32(lst)
    ext = torch.zeros(lst.size, dtype=torch.int32, device="cuda")
    keep = torch.zeros(lst.size, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    for theta in (0, 1 << 29, INF):
        lib.sssp_array_extract(ld.data_ptr(), lst.size, kd.data_ptr(), theta, ext.data_ptr(), cnt.data_ptr(),
                               keep.data_ptr(), cnt.data_ptr() + 4, _s())
        ce, ck = [int(x) for x in cnt.cpu().numpy()]
        inq = np.zeros(n, np.uint8)
        inq[lst] = 1
        want = oracle.lbpq_extract(inq, key, theta)
        assert np.array_equal(np.sort(ext[:ce].cpu().numpy().view(np.uint32)), want)
        assert np.array_equal(np.sort(keep[:ck].cpu().numpy().view(np.uint32)), np.flatnonzero(inq))


def test_tourney_argument_errors(lib):
    with pytest.raises(lib.SSSPError):
        lib.sssp_tourney_create(0)
    assert lib._lib.sssp_tourney_extract(None, None, 0, None, None, None) == lib.SSSP_ERR_INVALID_ARG
    assert lib._lib.sssp_array_extract(None, 4, None, 0, None, None, None, None, None) == lib.SSSP_ERR_INVALID_ARG
