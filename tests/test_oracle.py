"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: published generator
vectors, a textbook worked example, brute force (Bellman-Ford and exhaustive
simple-path enumeration), closed forms (Manhattan distance, prefix sums,
star weights), the invariants that characterise d, and the step bounds of
Lemma 5.1 and Theorems 5.3 / 5.5.  A planted mistake in any oracle function
(a dropped term, a wrong sign or index) fails at least one of these.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2105_06145_gb300 import graphgen as gg
from conftest import golden_path

INF = (1 << 64) - 1


def read_golden(name):
    rows = []
    with open(golden_path(name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# generator behind the rho sampler
# --------------------------------------------------------------------------

def test_splitmix64_published_vector():
    for idx, val in read_golden("splitmix64_state0.txt"):
        assert oracle.splitmix64(0, int(idx)) == int(val, 16)


# --------------------------------------------------------------------------
# Dijkstra: textbook example, brute force, closed forms
# --------------------------------------------------------------------------

def test_textbook_example():
    rows = read_golden("clrs_dijkstra_example.txt")
    edges = [tuple(map(int, r)) for r in rows if r[0] != "dist"]
    expect = [int(x) for x in next(r for r in rows if r[0] == "dist")[1:]]
    g = gg.from_edges(5, [e[0] for e in edges], [e[1] for e in edges], [e[2] for e in edges])
    assert oracle.dijkstra(g, 0).tolist() == expect
    assert oracle.bellman_ford(g, 0).tolist() == expect


def _tiny_cases(count, seed0=0):
    """Random tiny multigraphs: n <= 64, m <= 512, weights drawn from several
    ranges including 0 and 2^32-1, self-loops and duplicates allowed."""
    ranges = [(0, 0), (0, 3), (1, 10), (1, (1 << 18) - 1), (0xFFFFFFF0, 0xFFFFFFFF),
              (0, 0xFFFFFFFF)]
    rng = np.random.default_rng(seed0)
    for k in range(count):
        n = int(rng.integers(1, 65))
        m = int(rng.integers(0, min(512, 8 * n) + 1))
        lo, hi = ranges[k % len(ranges)]
        g = gg.random_graph(n, m, lo, hi, seed=seed0 * 1000003 + k)
        s = int(rng.integers(0, n))
        yield g, s


def test_dijkstra_matches_bellman_ford_10k_tiny_graphs():
    checked = 0
    for g, s in _tiny_cases(10000):
        d = oracle.dijkstra(g, s)
        b = oracle.bellman_ford(g, s)
        assert np.array_equal(d, b), (g.n, g.m, s)
        checked += 1
    assert checked == 10000


def _all_simple_paths_min(n, src, dst, w, s):
    """Exhaustive enumeration of every simple path from s (tiny n only)."""
    adj = [[] for _ in range(n)]
    for u, v, ww in zip(src, dst, w):
        adj[u].append((v, ww))
    best = [INF] * n
    best[s] = 0
    stack = [(s, 0, 1 << s)]
    while stack:
        u, d, seen = stack.pop()
        for v, ww in adj[u]:
            if not (seen >> v) & 1:
                nd = d + ww
                if nd < best[v]:
                    best[v] = nd
                stack.append((v, nd, seen | (1 << v)))
    return best


def test_dijkstra_matches_exhaustive_paths():
    rng = np.random.default_rng(7)
    for k in range(400):
        n = int(rng.integers(1, 8))
        m = int(rng.integers(0, 14))
        src = rng.integers(0, n, m).tolist()
        dst = rng.integers(0, n, m).tolist()
        hi = [5, 1 << 18, (1 << 32) - 1][k % 3]
        w = rng.integers(0, hi, m, endpoint=True).tolist()
        g = gg.from_edges(n, src, dst, w)
        s = int(rng.integers(0, n))
        assert oracle.dijkstra(g, s).tolist() == _all_simple_paths_min(n, src, dst, w, s)


@pytest.mark.parametrize("R,C,sr,sc", [(1, 1, 0, 0), (1, 9, 0, 4), (37, 53, 0, 0), (37, 53, 18, 26),
                                       (64, 64, 63, 0)])
def test_unit_grid_is_manhattan(R, C, sr, sc):
    g = gg.grid(R, C, wmax_excl=0)
    d = oracle.dijkstra(g, sr * C + sc).reshape(R, C)
    rr, cc = np.meshgrid(np.arange(R), np.arange(C), indexing="ij")
    assert np.array_equal(d, (np.abs(rr - sr) + np.abs(cc - sc)).astype(np.uint64))


def test_chain_is_prefix_sum_and_star_is_direct():
    g = gg.chain(500, wseed=3, wlo=0, whi=(1 << 32) - 1)
    d = oracle.dijkstra(g, 0)
    assert d.tolist() == [0] + np.cumsum(g.w.astype(object)).tolist()
    d7 = oracle.dijkstra(g, 7)
    assert d7[:7].tolist() == [INF] * 7 and d7[7] == 0
    st = gg.star(300, wseed=5)
    ds = oracle.dijkstra(st, 0)
    assert ds[0] == 0 and ds[1:].tolist() == st.w.tolist()
    assert oracle.dijkstra(st, 5).tolist() == [INF] * 5 + [0] + [INF] * 294


def test_grid256_invariants_and_symmetry():
    g, s = gg.workload_grid256()
    assert (g.n, g.m) == (65536, 261120)
    d = oracle.dijkstra(g, s)
    assert oracle.check(g, s, d) == (0, 0)
    # undirected with symmetric weights: d(s, v) == d(v, s) for a few v
    for v in (1, 255, 40000, 65535):
        assert oracle.dijkstra(g, v)[s] == d[v]


# --------------------------------------------------------------------------
# invariant checker: accepts d, rejects planted mistakes
# --------------------------------------------------------------------------

def test_check_rejects_planted_mistakes():
    g, s = gg.workload_grid256()
    d = oracle.dijkstra(g, s)
    assert oracle.check(g, s, d)[0] == 0
    bad = d.copy(); bad[s] = 1
    assert oracle.check(g, s, bad)[0] == 1
    bad = d.copy(); bad[1234] -= np.uint64(1)
    assert oracle.check(g, s, bad)[0] in (2, 3)
    bad = d.copy(); bad[1234] += np.uint64(1)  # its tight in-edge is now violated
    assert oracle.check(g, s, bad) == (2, 1234)
    bad = d.copy(); bad[999] = oracle.INF
    assert oracle.check(g, s, bad)[0] == 2
    # an unreachable vertex given a finite value: graph with an isolated vertex
    h = gg.from_edges(3, [0], [1], [4])
    dh = oracle.dijkstra(h, 0)
    assert dh.tolist() == [0, 4, INF] and oracle.check(h, 0, dh)[0] == 0
    dh2 = dh.copy(); dh2[2] = 0
    assert oracle.check(h, 0, dh2)[0] in (3, 4)


# --------------------------------------------------------------------------
# ExtDist pins
# --------------------------------------------------------------------------

def test_delta_extdist_closed_form():
    # i starts at 1 and advances every step: theta = i * Delta
    i = 1
    for k in range(1, 6):
        th, i = oracle.delta_extdist(i, 100, 0)
        assert th == 100 * k and i == k + 1
    # empty-bucket skip: qmin = 1234, Delta = 100 -> i jumps to ceil(12.34) = 13
    th, i = oracle.delta_extdist(1, 100, 1234)
    assert (th, i) == (1300, 14)
    th, i = oracle.delta_extdist(1, 100, 1300)
    assert (th, i) == (1300, 14)
    # saturation: Delta = 2^64-1 is Bellman-Ford (theta = +inf)
    assert oracle.delta_extdist(1, INF, 0)[0] == INF
    assert oracle.delta_extdist(3, 1 << 63, 0)[0] == INF
    # Delta = 1 with the skip is theta = min_Q delta (Dijkstra row of Table 2)
    assert oracle.delta_extdist(1, 1, 777)[0] == 777


def test_rho_extdist_special_cases():
    n = 10 ** 6  # keeps 20*q <= n: no dense-step adjustment
    dist = np.arange(100, dtype=np.uint64) * np.uint64(3)
    q = np.arange(100, dtype=np.uint32)
    # |Q| <= rho: every queued vertex is extracted (theta = +inf)
    assert oracle.rho_extdist(q, dist, n, 100, 1, 1, 0) == INF
    assert oracle.rho_extdist(q, dist, n, 1 << 40, 1, 1, 0) == INF
    # all keys equal: theta is that key
    same = np.full(100, 42, dtype=np.uint64)
    assert oracle.rho_extdist(q, same, n, 10, 1, 1, 0) == 42
    # theta is always the key of some queued vertex when sampling
    th = oracle.rho_extdist(q, dist, n, 10, 9, 3, 0)
    assert th in set(dist.tolist())


def test_rho_extdist_rank_within_constant_factor():
    """Appendix B: the sampled threshold ranks within a constant factor of rho
    w.h.p.  Keys are a permutation of 0..q-1, so the rank of theta is theta+1."""
    rng = np.random.default_rng(11)
    good = total = 0
    for trial in range(300):
        q = int(rng.integers(1000, 200000))
        rho = int(rng.integers(10, q // 2))
        keys = rng.permutation(q).astype(np.uint64)
        queue = rng.permutation(q).astype(np.uint32)
        th = oracle.rho_extdist(queue, keys, 10 ** 9, rho, trial, 1 + trial % 5, 0)
        rank = th + 1
        total += 1
        good += (rho / 2 <= rank <= 2 * rho)
    assert good >= 0.97 * total, (good, total)


def test_rho_extdist_dense_rule():
    """The first two dense steps (20*|Q| > n) use rho/10 (Sec. 6)."""
    q = 50000
    keys = np.arange(q, dtype=np.uint64)
    queue = np.arange(q, dtype=np.uint32)
    n = 100000  # 20*q > n: dense
    ranks_d = [oracle.rho_extdist(queue, keys, n, 5000, s, 1, 0) + 1 for s in range(40)]
    ranks_3 = [oracle.rho_extdist(queue, keys, n, 5000, s, 1, 2) + 1 for s in range(40)]
    assert 250 <= np.median(ranks_d) <= 1000
    assert 2500 <= np.median(ranks_3) <= 10000
    # a dense step with rho >= 10*q extracts everything even with the rule
    assert oracle.rho_extdist(queue, keys, n, 10 * q, 0, 1, 0) == INF


def _dense_ranks(rho, dense_before, reduced, trials=40):
    """Ranks of the sampled threshold on a dense step (20*q > n) over keys that
    are a permutation of 0..q-1 (rank = theta + 1)."""
    q, n = 50000, 100000
    keys = np.random.default_rng(5).permutation(q).astype(np.uint64)
    queue = np.arange(q, dtype=np.uint32)
    return [oracle.rho_extdist(queue, keys, n, rho, s, 1, dense_before, reduced) + 1 for s in range(trials)]


def test_rho_extdist_reduced_step_count():
    """Sec. 6 runs the first two dense steps with 10 % of rho; the count is a
    parameter: the first `reduced` dense steps use rho/10, later ones rho, and
    a count of 0 is plain rho-Stepping on every step."""
    rho = 5000
    for reduced in (0, 2, 6):
        for before in range(8):
            med = np.median(_dense_ranks(rho, before, reduced))
            if before < reduced:
                assert rho / 20 <= med <= rho / 5, (reduced, before, med)
            else:
                assert rho / 2 <= med <= 2 * rho, (reduced, before, med)
    # the same sample positions: a step below both counts, or past both, draws
    # the same threshold whatever the count
    q, n = 30000, 60000
    keys = np.random.default_rng(6).integers(0, 1 << 40, q, dtype=np.uint64)
    queue = np.random.default_rng(7).permutation(q).astype(np.uint32)
    for step in (1, 5, 9):
        a = oracle.rho_extdist(queue, keys, n, 3000, 77, step, 1, 2)
        b = oracle.rho_extdist(queue, keys, n, 3000, 77, step, 1, 6)
        c = oracle.rho_extdist(queue, keys, n, 3000, 77, step, 6, 2)
        d = oracle.rho_extdist(queue, keys, n, 3000, 77, step, 0, 0)
        assert a == b and c == d and a != c
    # a sparse step (20*q <= n) ignores the count
    for reduced in (0, 2, 6, 1000):
        assert oracle.rho_extdist(queue, keys, 10 ** 7, 3000, 77, 3, 0, reduced) == \
            oracle.rho_extdist(queue, keys, 10 ** 7, 3000, 77, 3, 0, 0)


def test_rho_extdist_rank_bound_at_reduced_rho():
    """Appendix B's guarantee holds for the reduced rho' = floor(rho/10) of a
    reduced dense step: rank within [rho'/2, 2 rho'] w.h.p."""
    rng = np.random.default_rng(13)
    good = total = 0
    for trial in range(300):
        q = int(rng.integers(2000, 200000))
        rho = int(rng.integers(100, q // 2))
        keys = rng.permutation(q).astype(np.uint64)
        queue = rng.permutation(q).astype(np.uint32)
        n = 10 * q  # 20*q > n: dense
        th = oracle.rho_extdist(queue, keys, n, rho, trial, 1 + trial % 5, trial % 4, 4)
        rank, rp = th + 1, rho // 10
        total += 1
        good += (rp / 2 <= rank <= 2 * rp)
    assert good >= 0.97 * total, (good, total)


@pytest.mark.parametrize("reduced", [0, 1, 6, 50])
def test_stepping_with_any_reduced_count(reduced):
    """The count of reduced dense steps changes thresholds only: distances equal
    Dijkstra's, Lemma 5.1's extraction bound and the partial-step bound of
    Theorem 5.3's proof hold for every count."""
    for g in _bounded_graphs():
        s = int(np.flatnonzero(gg.largest_cc(g))[0])
        d = oracle.dijkstra(g, s)
        h, kn = oracle.hops(g, s)
        for rho in (64, 1 << 10):
            ds, st, ext = oracle.stepping(g, s, oracle.RHO, rho, seed=3, want_ext=True, reduced=reduced)
            assert np.array_equal(d, ds), (g.name, rho, reduced)
            reach = d != oracle.INF
            hv = h.astype(np.int64)
            hv[s] = 1
            assert np.all(ext[reach].astype(np.int64) <= hv[reach])
            assert st["partial_steps"] <= kn + 1


@pytest.mark.parametrize("warm_steps,warm_rho", [(1, 1), (3, 4), (6, 256), (50, 16)])
def test_stepping_with_a_warm_up(warm_steps, warm_rho):
    """Warm-up steps (the first warm_steps steps use rho = warm_rho) change
    thresholds only: distances equal Dijkstra's, and Lemma 5.1's extraction
    bound and the partial-step bound of Theorem 5.3's proof still hold (every
    warm-up theta is a sampled queued key, as in any rho-Stepping step)."""
    for g in _bounded_graphs():
        s = int(np.flatnonzero(gg.largest_cc(g))[0])
        d = oracle.dijkstra(g, s)
        h, kn = oracle.hops(g, s)
        for rho in (64, 1 << 10):
            ds, st, ext = oracle.stepping(g, s, oracle.RHO, rho, seed=3, want_ext=True, reduced=6,
                                          warm_steps=warm_steps, warm_rho=warm_rho)
            assert np.array_equal(d, ds), (g.name, rho, warm_steps, warm_rho)
            reach = d != oracle.INF
            hv = h.astype(np.int64)
            hv[s] = 1
            assert np.all(ext[reach].astype(np.int64) <= hv[reach])
            assert st["partial_steps"] <= kn + 1


def test_rho_extdist_sample_cap():
    """The capped rule: a cap of 4096 (or one above the formula's count) is
    the default rule; below it, theta is the rank floor(rho' s / q) of the
    first s draws with s the cap -- checked against the draws themselves
    (positions from the published generator), sorted here with a library sort."""
    rng = np.random.default_rng(41)
    for trial in range(60):
        n = int(rng.integers(1000, 400000))
        q = int(rng.integers(1, n + 1))
        dist = rng.integers(0, 1 << 40, n, dtype=np.uint64)
        queue = rng.permutation(n)[:q].astype(np.uint32)
        rho = int([1, 7, 256, 5000][trial % 4])
        seed, step = int(rng.integers(0, 1 << 62)), int(rng.integers(1, 100))
        base = oracle.rho_extdist(queue, dist, n, rho, seed, step, 0, 0)
        assert oracle.rho_extdist(queue, dist, n, rho, seed, step, 0, 0, max_samples=4096) == base
        lg = int(math.floor(math.log2(q + 1)))
        s_formula = min(4096, 10 * (-(-q // rho) + 1 + lg))
        if q <= rho:
            assert oracle.rho_extdist(queue, dist, n, rho, seed, step, 0, 0, max_samples=64) == INF
            continue
        assert oracle.rho_extdist(queue, dist, n, rho, seed, step, 0, 0, max_samples=s_formula) == base
        for cap in (1, 100, 1024):
            s = min(cap, s_formula)
            pos = [(oracle.splitmix64(seed, (step << 32) | j) * q) >> 64 for j in range(s)]
            keys = np.sort(dist[queue[pos]])
            r = min(s - 1, rho * s // q)
            assert oracle.rho_extdist(queue, dist, n, rho, seed, step, 0, 0, max_samples=cap) == int(keys[r])


def test_rho_extdist_capped_sample_order_statistic():
    """The capped sample count, against order statistics: with distinct keys
    0..q-1, rho = 256 and q in [300k, 500k], a cap of 1024 gives rank
    floor(256 * 1024 / q) = 0, so theta is the smallest of 1024 uniform draws
    and the extracted count theta + 1 averages (q + 1) / 1025.  (The uncapped
    rule draws 4096 samples with rank 0-3 here, a wrong count or rank moves the
    mean by a factor of 1.3 or more.)"""
    rng = np.random.default_rng(5)
    ratios = []
    for _ in range(150):
        q = int(rng.integers(300000, 500001))
        dist = rng.permutation(q).astype(np.uint64)
        queue = np.arange(q, dtype=np.uint32)
        th = oracle.rho_extdist(queue, dist, 10 ** 7, 256, int(rng.integers(0, 1 << 62)), 1, 0, 0, max_samples=1024)
        ratios.append((th + 1) / ((q + 1) / 1025))
    assert 0.8 < float(np.mean(ratios)) < 1.2, np.mean(ratios)


def test_warm_up_special_cases():
    """No warm-up steps is the paper's schedule (same thresholds, so the same
    steps and work); a warm-up covering the whole solve is rho-Stepping with
    rho = warm_rho and no dense-step reduction (where its sample count stays
    under the warm-up cap of 1024); a warm-up with warm_rho = rho
    is the schedule whose reduced dense steps come only after it (with no
    reduced steps at all, the same as no warm-up)."""
    g = gg.rmat(12, 8, gen_seed=31, wseed=32)
    s = int(np.flatnonzero(gg.largest_cc(g))[0])
    d = oracle.dijkstra(g, s)
    for rho in (16, 300):
        base = oracle.stepping(g, s, oracle.RHO, rho, seed=5, reduced=2)
        same = oracle.stepping(g, s, oracle.RHO, rho, seed=5, reduced=2, warm_steps=0, warm_rho=7)
        assert np.array_equal(base[0], same[0]) and base[1] == same[1]
        # (warm-up steps draw at most 1024 samples; with rho_w >= 64 on 4,096
        # vertices the default rule draws no more: 10 (4096/64 + 1 + 12) < 1024)
        for wr in (64, 100, 300):
            all_warm = oracle.stepping(g, s, oracle.RHO, rho, seed=5, reduced=6, warm_steps=10 ** 6, warm_rho=wr)
            plain = oracle.stepping(g, s, oracle.RHO, wr, seed=5, reduced=0)
            assert np.array_equal(all_warm[0], d) and all_warm[1] == plain[1], (rho, wr)
        w_same = oracle.stepping(g, s, oracle.RHO, rho, seed=5, reduced=0, warm_steps=4, warm_rho=rho)
        no_red = oracle.stepping(g, s, oracle.RHO, rho, seed=5, reduced=0)
        assert w_same[1] == no_red[1]
    with pytest.raises(ValueError):
        oracle.stepping(g, s, oracle.RHO, 64, warm_steps=2, warm_rho=0)


# --------------------------------------------------------------------------
# Algorithm 1 run sequentially: exact distances and the paper's step bounds
# --------------------------------------------------------------------------

def _algo_cases():
    return [(oracle.RHO, 1), (oracle.RHO, 2), (oracle.RHO, 31), (oracle.RHO, 1 << 10),
            (oracle.RHO, (1 << 32) - 1), (oracle.DELTA_STAR, 1), (oracle.DELTA_STAR, 1 << 13),
            (oracle.DELTA_STAR, INF), (oracle.BELLMAN_FORD, 0), (oracle.DELTA, 1),
            (oracle.DELTA, 1 << 13), (oracle.DELTA, INF), (oracle.DIJKSTRA, 0)]


@pytest.mark.parametrize("algo,param", _algo_cases())
def test_stepping_equals_dijkstra_tiny(algo, param):
    for g, s in _tiny_cases(600, seed0=algo * 100 + (param % 97)):
        d = oracle.dijkstra(g, s)
        ds, st, _ = oracle.stepping(g, s, algo, param, seed=s)
        assert np.array_equal(d, ds)


def _bounded_graphs():
    yield gg.grid(40, 40, wseed=9)
    yield gg.rmat(12, 8, gen_seed=5, wseed=6)
    yield gg.road(48, 0.75, seed=3)
    yield gg.chain(300, wseed=1, wlo=1, whi=50, both=True)
    yield gg.random_graph(3000, 20000, 1, 1000, seed=4, drop_self_loops=True)


@pytest.mark.parametrize("algo,param", [(oracle.RHO, 1), (oracle.RHO, 64), (oracle.RHO, 1 << 12),
                                        (oracle.DELTA_STAR, 1), (oracle.DELTA_STAR, 1 << 10),
                                        (oracle.DELTA_STAR, 1 << 20), (oracle.BELLMAN_FORD, 0)])
def test_stepping_bounds(algo, param):
    """Lemma 5.1: every vertex is extracted at most h(v) times (fewest-hop
    shortest-path length; weights >= 1).  Bellman-Ford: <= k_n + 1 steps.
    Theorem 5.5: Delta* uses <= ceil(k_n L / Delta) + k_n + 1 steps.
    Theorem 5.3's proof: rho-Stepping has <= k_n + 1 partial-extract steps."""
    for g in _bounded_graphs():
        s = int(np.flatnonzero(gg.largest_cc(g))[0])
        d = oracle.dijkstra(g, s)
        h, kn = oracle.hops(g, s)
        ds, st, ext = oracle.stepping(g, s, algo, param, seed=1, want_ext=True)
        assert np.array_equal(d, ds)
        reach = d != oracle.INF
        assert np.all(ext[~reach] == 0)
        hv = h.astype(np.int64)
        hv[s] = 1
        assert np.all(ext[reach].astype(np.int64) <= hv[reach]), g.name
        L = int(g.w.max())
        if algo == oracle.BELLMAN_FORD:
            assert st["steps"] <= kn + 1
        elif algo == oracle.DELTA_STAR:
            assert st["steps"] <= math.ceil(kn * L / param) + kn + 1
        else:
            assert st["partial_steps"] <= kn + 1


def test_hops_pins():
    # chain: h(v) = v; unit grid: h = Manhattan distance
    g = gg.chain(50, wseed=2)
    h, k = oracle.hops(g, 0)
    assert h.tolist() == list(range(50)) and k == 49
    gu = gg.grid(9, 11, wmax_excl=0)
    hu, ku = oracle.hops(gu, 0)
    rr, cc = np.meshgrid(np.arange(9), np.arange(11), indexing="ij")
    assert np.array_equal(hu.reshape(9, 11), (rr + cc).astype(np.uint32)) and ku == 18
    # fewest hops among equal-length paths: 0->1->2 (1+1) vs 0->2 (2)
    t = gg.from_edges(3, [0, 1, 0], [1, 2, 2], [1, 1, 2])
    assert oracle.hops(t, 0)[0].tolist() == [0, 1, 1]


def test_bruteforce_hops_tiny():
    """h(v) by exhaustive enumeration of simple paths on tiny graphs."""
    rng = np.random.default_rng(5)
    for _ in range(200):
        n = int(rng.integers(1, 7))
        m = int(rng.integers(0, 12))
        src = rng.integers(0, n, m).tolist()
        dst = rng.integers(0, n, m).tolist()
        w = rng.integers(1, 4, m).tolist()
        g = gg.from_edges(n, src, dst, w)
        d = oracle.dijkstra(g, 0)
        best = {}
        adj = [[] for _ in range(n)]
        for u, v, ww in zip(src, dst, w):
            adj[u].append((v, ww))
        stack = [(0, 0, 0, 1)]
        while stack:
            u, dd, hh, seen = stack.pop()
            if dd == d[u]:
                best[u] = min(best.get(u, 1 << 30), hh)
            for v, ww in adj[u]:
                if not (seen >> v) & 1:
                    stack.append((v, dd + ww, hh + 1, seen | (1 << v)))
        h, _ = oracle.hops(g, 0)
        for v in range(n):
            if d[v] == oracle.INF:
                assert h[v] == 0xFFFFFFFF
            else:
                assert h[v] == best[v]


def test_delta_finishcheck_closed_form():
    # theta = i * Delta; the jump past empty buckets
    assert oracle.delta_theta(1, 100, 0) == (100, 1)
    assert oracle.delta_theta(1, 100, 1234) == (1300, 13)
    # FinishCheck: stay while the step wrote a value below theta, else advance
    assert oracle.delta_finish(3, 300, 299) == 3
    assert oracle.delta_finish(3, 300, 300) == 4
    assert oracle.delta_finish(3, 300, oracle.INF) == 4


def test_dijkstra_in_framework_settles_one_distance_per_step():
    """theta = min_Q delta (Table 2, Dijkstra row): with positive weights every
    step extracts exactly the vertices at the smallest queued distance, each
    vertex once, so the step count is the number of distinct finite distances."""
    for g in (gg.grid(30, 30, wseed=4), gg.rmat(11, 8, gen_seed=3, wseed=4),
              gg.random_graph(800, 5000, 1, 50, seed=2, drop_self_loops=True)):
        s = int(np.flatnonzero(gg.largest_cc(g))[0])
        d = oracle.dijkstra(g, s)
        ds, st, ext = oracle.stepping(g, s, oracle.DIJKSTRA, 0, want_ext=True)
        fin = d[d != oracle.INF]
        assert np.array_equal(ds, d)
        assert st["steps"] == np.unique(fin).size
        assert np.all(ext[d != oracle.INF] == 1) and st["extracted"] == fin.size


def test_delta_stepping_distances_and_extraction_bound():
    """Original Delta-Stepping reaches d, and Lemma 5.1 (each vertex extracted
    at most h(v) times) holds for it as for every stepping algorithm."""
    g = gg.road(40, 0.75, seed=2)
    s = int(np.flatnonzero(gg.largest_cc(g))[0])
    d = oracle.dijkstra(g, s)
    h, kn = oracle.hops(g, s)
    hv = h.astype(np.int64)
    hv[s] = 1
    reach = d != oracle.INF
    for delta in (1, 200, 5000, 1 << 20):
        ds, st, ext = oracle.stepping(g, s, oracle.DELTA, delta, want_ext=True)
        assert np.array_equal(ds, d)
        assert np.all(ext[reach].astype(np.int64) <= hv[reach])


def _golden_tree():
    from conftest import golden_path
    vals = {}
    for line in open(golden_path("tournament_tree_figure.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        vals[k] = [int(x) for x in v]
    return np.array(vals["keys"], dtype=np.uint64), vals["root"][0]


def test_lbpq_oracle_on_the_papers_tournament_tree_example():
    """Sec. 4.2: the tree of the figure holds records with keys 3,8,4,6,1,5 and
    its root keeps the smallest key, 1."""
    key, root = _golden_tree()
    inq = np.ones(key.size, np.uint8)
    assert oracle.lbpq_min(inq, key) == root
    got = oracle.lbpq_extract(inq, key, 4)
    assert sorted(key[got].tolist()) == [1, 3, 4]
    assert oracle.lbpq_min(inq, key) == 5 and oracle.lbpq_extract(inq, key, 4).size == 0
    assert sorted(oracle.lbpq_extract(inq, key, (1 << 64) - 1).tolist()) == [1, 3, 5]
    assert oracle.lbpq_min(inq, key) == (1 << 64) - 1


def test_lbpq_oracle_against_sorting():
    """Extract(theta) returns exactly the queued records that come first in key
    order up to theta (an order-statistics view, computed here by sorting), and
    Reduce is the first key in that order."""
    rng = np.random.default_rng(3)
    for trial in range(200):
        n = int(rng.integers(1, 300))
        key = rng.integers(0, 50, n).astype(np.uint64)
        inq = (rng.random(n) < 0.6).astype(np.uint8)
        q = np.flatnonzero(inq)
        order = q[np.argsort(key[q], kind="stable")]
        if q.size:
            assert oracle.lbpq_min(inq, key) == int(key[order[0]])
        else:
            assert oracle.lbpq_min(inq, key) == (1 << 64) - 1
        theta = int(rng.integers(0, 60))
        kcount = int(np.searchsorted(key[order], theta, side="right"))
        got = oracle.lbpq_extract(inq, key, theta)
        assert sorted(got.tolist()) == sorted(order[:kcount].tolist())
        assert np.array_equal(np.flatnonzero(inq), np.sort(order[kcount:]))
