"""Input generators: determinism, sizes, structure (symmetric, no self-loops or
duplicates), and the k-NN graph against brute force."""
import numpy as np

from paper_2105_06145_gb300 import graphgen as gg


def _edge_set(g):
    src = np.repeat(np.arange(g.n), np.diff(g.off.astype(np.int64)))
    return src, g.tgt.astype(np.int64), g.w


def _check_simple_symmetric(g):
    g.validate()
    src, dst, w = _edge_set(g)
    assert np.all(src != dst)                                      # no self-loops
    key = src * g.n + dst
    assert np.unique(key).size == key.size                         # no duplicates
    fwd = dict(zip(key.tolist(), w.tolist()))
    for a, b, ww in zip(src[:5000].tolist(), dst[:5000].tolist(), w[:5000].tolist()):
        assert fwd[b * g.n + a] == ww                              # symmetric weights


def test_grid_sizes_and_weights():
    g = gg.grid(256, 256, wseed=1)
    assert (g.n, g.m) == (65536, 261120)
    assert g.w.min() >= 1 and g.w.max() < (1 << 18)
    _check_simple_symmetric(g)
    h = gg.grid(256, 256, wseed=1)
    assert np.array_equal(g.w, h.w) and not np.array_equal(g.w, gg.grid(256, 256, wseed=2).w)


def test_rmat_deterministic_and_simple():
    a = gg.rmat(13, 16, gen_seed=2, wseed=3)
    b = gg.rmat(13, 16, gen_seed=2, wseed=3)
    assert np.array_equal(a.off, b.off) and np.array_equal(a.tgt, b.tgt) and np.array_equal(a.w, b.w)
    assert not np.array_equal(a.tgt, gg.rmat(13, 16, gen_seed=5, wseed=3).tgt)
    _check_simple_symmetric(a)
    assert a.w.min() >= 1 and a.w.max() < (1 << 18)
    d = a.degrees()
    assert d.max() > 20 * max(1.0, d[d > 0].mean())                  # heavy-tailed degrees


def test_rmat_n_keeps_exactly_n_vertices():
    g = gg.rmat_n(3000, 6, gen_seed=4, wseed=5)
    assert g.n == 3000 and int(g.tgt.max()) < 3000
    _check_simple_symmetric(g)


def test_road_and_jittered_grid():
    r = gg.road(64, 0.75, seed=5)
    _check_simple_symmetric(r)
    assert r.w.min() >= 201 and r.w.max() <= 1971                  # floor(1000 * [0.2, 1.97]) + 1
    deg = r.degrees()
    assert deg.max() <= 4
    full = 2 * (64 * 63 * 2)
    assert 0.70 * full < r.m < 0.80 * full                           # edges kept with p = 0.75
    u = gg.jittered_grid_uniform(64, seed=5, wseed=9)
    assert np.array_equal(u.off, r.off) and np.array_equal(u.tgt, r.tgt)  # same topology
    assert u.w.max() < (1 << 18)


def test_multi_workload_shape():
    W = gg.workload_multi(count=20, lo_log2=8, hi_log2=12, seed=3)
    assert len(W) == 20
    for g, s in W:
        assert 2 ** 8 <= g.n <= 2 ** 12 + 2 * 2 ** 6 + 1 and 0 <= s < g.n
        g.validate()


def test_knn_matches_brute_force():
    g, P = gg.knn(2500, 3, 0.02, 6, seed=2, with_points=True)
    D = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    np.fill_diagonal(D, np.inf)
    idx = np.lexsort((np.tile(np.arange(2500), (2500, 1)), D), axis=1)[:, :6]
    want = set()
    for i in range(2500):
        for j in idx[i]:
            want.add((i, int(j)))
            want.add((int(j), i))
    src, dst, w = _edge_set(g)
    assert set(zip(src.tolist(), dst.tolist())) == want
    dd = np.sqrt(((P[src] - P[dst]) ** 2).sum(-1))
    assert np.array_equal(w, (np.floor(float(1 << 20) * dd) + 1).astype(np.uint32))
    _check_simple_symmetric(g)


def test_pick_sources_in_largest_component():
    g = gg.rmat(12, 4, gen_seed=9, wseed=9)
    lab = gg.largest_cc(g)
    srcs = gg.pick_sources(g, 30, 1)
    assert len(set(srcs)) == 30 and all(lab[s] for s in srcs)


def test_generators_do_not_depend_on_the_thread_count():
    """The OpenMP generators give the same graphs with 1 thread as with the
    default count (every random number is splitmix64(seed, index)); the sizes
    are large enough (>= 2^20 edge draws) for the multi-threaded sort path."""
    import hashlib
    import os
    import subprocess
    import sys

    def digest(g):
        h = hashlib.sha256()
        for a in (g.off, g.tgt, g.w):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()

    here = {"rmat": digest(gg.rmat(17, 8, gen_seed=6, wseed=7)),
            "road": digest(gg.road(1100, 0.75, seed=8)),
            "knn": digest(gg.knn(3000, 4, 0.05, 5, float(1 << 20), seed=9))}
    code = ("import hashlib, json, numpy as np\n"
            "from paper_2105_06145_gb300 import graphgen as gg\n"
            "def digest(g):\n"
            "    h = hashlib.sha256()\n"
            "    for a in (g.off, g.tgt, g.w):\n"
            "        h.update(np.ascontiguousarray(a).tobytes())\n"
            "    return h.hexdigest()\n"
            "print(json.dumps({'rmat': digest(gg.rmat(17, 8, gen_seed=6, wseed=7)),\n"
            "                  'road': digest(gg.road(1100, 0.75, seed=8)),\n"
            "                  'knn': digest(gg.knn(3000, 4, 0.05, 5, float(1 << 20), seed=9))}))\n")
    env = dict(os.environ, OMP_NUM_THREADS="1")
    env.pop("SSSP_GRAPH_CACHE", None)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.check_output([sys.executable, "-c", code], env=env, cwd=root, text=True)
    import json
    assert json.loads(out.strip().splitlines()[-1]) == here
