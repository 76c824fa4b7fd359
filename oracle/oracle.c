/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded CPU implementation of what the stepping-SSSP
 * library computes.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg may load this file; the library's solve path never does.  It
 * shares no code, header or constant table with the CUDA sources.
 *
 * Paper: Dong, Gu, Sun, Zhang, "Efficient Stepping Algorithms and
 * Implementations for Parallel Shortest Paths", SPAA'21 (arXiv 2105.06145).
 *
 * Contents (each function cites the passage it follows):
 *   oracle_dijkstra      -- d(s,v), the plain definition of the SSSP output
 *                           (Sec. 1 problem statement; Sec. 2 graph notation),
 *                           computed by textbook binary-heap Dijkstra.
 *   oracle_bellman_ford  -- brute-force Bellman-Ford (n-1 full passes), used
 *                           to pin oracle_dijkstra on tiny graphs.
 *   oracle_stepping      -- Algorithm 1 (the stepping framework) run
 *                           sequentially over the array-based LaB-PQ
 *                           (Sec. 4.3), with the ExtDist rules of Table 2 for
 *                           Bellman-Ford, Delta*-Stepping and rho-Stepping.
 *   oracle_rho_extdist   -- the sampling-based rho-th smallest threshold of
 *                           Sec. 6 ("Threshold estimation") and Appendix B.
 *   oracle_delta_extdist -- theta = i*Delta of Table 2 (Delta*-Stepping).
 *   oracle_splitmix64    -- the counter-based generator the rho sampler draws
 *                           from (Steele, Lea, Flood, OOPSLA 2014).
 *   oracle_check         -- invariants that characterise d (Sec. 2).
 *   oracle_lbpq_extract / oracle_lbpq_min -- the LaB-PQ interface on a plain
 *                           set (Sec. 3.1, Table 1), the definition the device
 *                           tournament tree (Sec. 4.2) must reproduce.
 *   oracle_hops          -- fewest-hop shortest-path depth h(v) (Sec. 2,
 *                           "hop distance"), used for the step bounds of
 *                           Lemma 5.1 and Theorems 5.3 / 5.5.
 *
 * Graph convention: directed CSR.  off[0..n], off[0]=0, off[n]=m; the edges of
 * u are tgt[off[u]..off[u+1]) with weights w[...].  Weights are unsigned
 * 32-bit integers; distances are unsigned 64-bit, UINT64_MAX = unreachable.
 *
 * Parity status: every distance returned here is pinned (brute-force
 * Bellman-Ford, closed forms, invariants, a textbook example).  Step counts
 * and thresholds of oracle_stepping are pinned only by the bounds of
 * Lemma 5.1 / Theorems 5.3, 5.5 and by the exact sampling definition.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF UINT64_MAX

/* ------------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea, Flood 2014): output k (0-based) of the generator */
/* started at state `seed` is mix(seed + (k+1)*golden_gamma).                */
/* ------------------------------------------------------------------------ */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------------------------ */
/* Binary min-heap of (key, vertex) pairs, lazy deletion (no decrease-key).  */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t v; } heap_item;
typedef struct { heap_item* a; size_t size, cap; } heap;

static int heap_push(heap* h, uint64_t key, uint32_t v)
{
    if (h->size == h->cap) {
        size_t nc = h->cap ? 2 * h->cap : 1024;
        heap_item* na = (heap_item*)realloc(h->a, nc * sizeof(heap_item));
        if (!na) return -1;
        h->a = na;
        h->cap = nc;
    }
    size_t i = h->size++;
    while (i > 0) {
        size_t p = (i - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].key = key;
    h->a[i].v = v;
    return 0;
}

static heap_item heap_pop(heap* h)
{
    heap_item top = h->a[0];
    heap_item last = h->a[--h->size];
    size_t i = 0;
    for (;;) {
        size_t l = 2 * i + 1, r = l + 1, c;
        if (l >= h->size) break;
        c = (r < h->size && h->a[r].key < h->a[l].key) ? r : l;
        if (h->a[c].key >= last.key) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->size > 0) h->a[i] = last;
    return top;
}

/*
 * d(s, v) for every v: the minimum over s->v paths of the sum of edge
 * weights, UINT64_MAX when no path exists (Sec. 1 problem statement; Sec. 2
 * graph notation).  Textbook Dijkstra with a binary heap and lazy deletion;
 * correct for any non-negative integer weights.  Returns 0, or -1 on a bad
 * source / allocation failure.
 */
int oracle_dijkstra(uint32_t n, const uint64_t* off, const uint32_t* tgt,
                    const uint32_t* w, uint32_t s, uint64_t* dist)
{
    if (s >= n) return -1;
    for (uint32_t v = 0; v < n; ++v) dist[v] = ORC_INF;
    heap h = {0, 0, 0};
    dist[s] = 0;
    if (heap_push(&h, 0, s)) return -1;
    while (h.size > 0) {
        heap_item it = heap_pop(&h);
        if (it.key != dist[it.v]) continue; /* stale entry */
        uint32_t u = it.v;
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint64_t cand = dist[u] + (uint64_t)w[e];
            uint32_t v = tgt[e];
            if (cand < dist[v]) {
                dist[v] = cand;
                if (heap_push(&h, cand, v)) { free(h.a); return -1; }
            }
        }
    }
    free(h.a);
    return 0;
}

/*
 * Brute-force Bellman-Ford: up to n-1 passes relaxing every edge, stopping
 * early when a pass changes nothing.  O(n m); used only on tiny graphs to pin
 * oracle_dijkstra.
 */
int oracle_bellman_ford(uint32_t n, const uint64_t* off, const uint32_t* tgt,
                        const uint32_t* w, uint32_t s, uint64_t* dist)
{
    if (s >= n) return -1;
    for (uint32_t v = 0; v < n; ++v) dist[v] = ORC_INF;
    dist[s] = 0;
    for (uint32_t pass = 0; pass + 1 < n; ++pass) {
        int changed = 0;
        for (uint32_t u = 0; u < n; ++u) {
            if (dist[u] == ORC_INF) continue;
            for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
                uint64_t cand = dist[u] + (uint64_t)w[e];
                if (cand < dist[tgt[e]]) { dist[tgt[e]] = cand; changed = 1; }
            }
        }
        if (!changed) break;
    }
    return 0;
}

/*
 * Reachability from s by breadth-first search (ignores weights).
 * reach[v] = 1 iff some path s->v exists.
 */
int oracle_reach(uint32_t n, const uint64_t* off, const uint32_t* tgt,
                 uint32_t s, uint8_t* reach)
{
    if (s >= n) return -1;
    uint32_t* q = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    if (!q) return -1;
    memset(reach, 0, n);
    size_t head = 0, tail = 0;
    reach[s] = 1;
    q[tail++] = s;
    while (head < tail) {
        uint32_t u = q[head++];
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t v = tgt[e];
            if (!reach[v]) { reach[v] = 1; q[tail++] = v; }
        }
    }
    free(q);
    return 0;
}

/*
 * Invariants that together characterise the distance function d (Sec. 2):
 *   1  dist[s] == 0
 *   2  every edge (u,v) with finite dist[u] satisfies dist[v] <= dist[u]+w
 *   3  every finite dist[v], v != s, is tight on some in-edge
 *      (dist[v] == dist[u]+w for some edge (u,v) with finite dist[u])
 *   4  dist[v] == UINT64_MAX exactly when v is unreachable from s
 * Returns 0 when all hold, otherwise the number of the first violated
 * invariant; *bad (if non-null) receives the offending vertex.  Invariants
 * 1-3 and non-negative weights imply dist == d (the standard certificate).
 */
int oracle_check(uint32_t n, const uint64_t* off, const uint32_t* tgt,
                 const uint32_t* w, uint32_t s, const uint64_t* dist,
                 uint32_t* bad)
{
    if (s >= n) return -1;
    if (dist[s] != 0) { if (bad) *bad = s; return 1; }
    uint8_t* tight = (uint8_t*)calloc(n ? n : 1, 1);
    uint8_t* reach = (uint8_t*)malloc(n ? n : 1);
    if (!tight || !reach) { free(tight); free(reach); return -1; }
    tight[s] = 1;
    int rc = 0;
    for (uint32_t u = 0; u < n && !rc; ++u) {
        if (dist[u] == ORC_INF) continue;
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint64_t cand = dist[u] + (uint64_t)w[e];
            uint32_t v = tgt[e];
            if (dist[v] > cand) { if (bad) *bad = v; rc = 2; break; }
            if (dist[v] == cand) tight[v] = 1;
        }
    }
    if (!rc) {
        for (uint32_t v = 0; v < n; ++v) {
            if (dist[v] != ORC_INF && !tight[v]) { if (bad) *bad = v; rc = 3; break; }
        }
    }
    if (!rc) {
        oracle_reach(n, off, tgt, s, reach);
        for (uint32_t v = 0; v < n; ++v) {
            if ((dist[v] == ORC_INF) == (reach[v] != 0)) { if (bad) *bad = v; rc = 4; break; }
        }
    }
    free(tight);
    free(reach);
    return rc;
}

/*
 * Hop distance h(v): the number of edges on the shortest (weighted) s->v path
 * that uses the fewest edges (Sec. 2, "hop distance"); UINT32_MAX when v is
 * unreachable.  Computed by Dijkstra on the lexicographic key (distance,
 * hops).  Returns max_v h(v) over reachable v (the fewest-hop shortest-path
 * tree depth from s, the k_n of Lemma 5.1 for this source), or -1 on error.
 */
int64_t oracle_hops(uint32_t n, const uint64_t* off, const uint32_t* tgt,
                    const uint32_t* w, uint32_t s, uint32_t* hops)
{
    if (s >= n) return -1;
    uint64_t* dist = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n);
    if (!dist) return -1;
    for (uint32_t v = 0; v < n; ++v) { dist[v] = ORC_INF; hops[v] = UINT32_MAX; }
    /* heap key: we order by (dist, hops); hops < 2^32 so pack into a pair of
     * comparisons by pushing dist and keeping hops in a side array.  Ties in
     * dist are broken by hops through a second heap key. */
    typedef struct { uint64_t d; uint32_t h, v; } it2;
    it2* a = NULL;
    size_t size = 0, cap = 0;
    int64_t depth = 0;
#define IT_LESS(x, y) ((x).d < (y).d || ((x).d == (y).d && (x).h < (y).h))
#define PUSH2(D, H, V) do {                                                   \
        if (size == cap) {                                                    \
            size_t nc = cap ? 2 * cap : 1024;                                 \
            it2* na = (it2*)realloc(a, nc * sizeof(it2));                     \
            if (!na) { free(a); free(dist); return -1; }                      \
            a = na; cap = nc;                                                 \
        }                                                                     \
        it2 x_; x_.d = (D); x_.h = (H); x_.v = (V);                           \
        size_t i_ = size++;                                                   \
        while (i_ > 0) {                                                      \
            size_t p_ = (i_ - 1) / 2;                                         \
            if (!IT_LESS(x_, a[p_])) break;                                   \
            a[i_] = a[p_]; i_ = p_;                                           \
        }                                                                     \
        a[i_] = x_;                                                           \
    } while (0)
    dist[s] = 0;
    hops[s] = 0;
    PUSH2(0, 0, s);
    while (size > 0) {
        it2 top = a[0], last = a[--size];
        size_t i = 0;
        for (;;) {
            size_t l = 2 * i + 1, r = l + 1, c;
            if (l >= size) break;
            c = (r < size && IT_LESS(a[r], a[l])) ? r : l;
            if (!IT_LESS(a[c], last)) break;
            a[i] = a[c];
            i = c;
        }
        if (size > 0) a[i] = last;
        if (top.d != dist[top.v] || top.h != hops[top.v]) continue; /* stale */
        if ((int64_t)top.h > depth) depth = top.h;
        uint32_t u = top.v;
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t v = tgt[e];
            uint64_t cd = dist[u] + (uint64_t)w[e];
            uint32_t ch = hops[u] + 1;
            if (cd < dist[v] || (cd == dist[v] && ch < hops[v])) {
                dist[v] = cd;
                hops[v] = ch;
                PUSH2(cd, ch, v);
            }
        }
    }
#undef PUSH2
#undef IT_LESS
    free(a);
    free(dist);
    return depth;
}

/* ------------------------------------------------------------------------ */
/* ExtDist rules (Table 2 and Sec. 6).                                        */
/* ------------------------------------------------------------------------ */

/* Upper bound on the rho-sampler's sample count (a reading: the paper only
 * says s = O(n/rho + log n); the cap bounds the sort). */
#define ORC_MAX_SAMPLES 4096u
#define ORC_WARM_SAMPLES 1024u  /* sample cap of the warm-up steps of oracle_stepping */

static uint64_t floor_log2_u64(uint64_t x) /* x >= 1 */
{
    uint64_t r = 0;
    while (x > 1) { x >>= 1; ++r; }
    return r;
}

static int cmp_u64(const void* a, const void* b)
{
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

/*
 * rho-Stepping threshold (Table 2: theta <- the rho-th smallest delta in Q;
 * Sec. 6 "Threshold estimation" and Appendix B: sample s = c(n/rho + log n)
 * uniformly random frontier elements, sort them, pick the (rho*s/n)-th; c=10;
 * when the frontier holds fewer than rho vertices theta is the largest key;
 * 10% of rho in the first two dense rounds).
 *
 * queue[0..q) lists the ids in Q in list order; dist is the key array; n is
 * the vertex count; step is the 1-based step number; dense_before is the
 * number of dense steps that came before this one; reduced is how many dense
 * steps use 10% of rho (the paper's choice is 2; Sec. 6 gives it as a tuning
 * made on its machine, so the count is a parameter here).  Readings:
 *   - a step is dense when 20*q > n; the first `reduced` dense steps use
 *     rho' = max(1, floor(rho/10)), every other step rho' = rho;
 *   - "n" inside s and the rank is the frontier size q (samples come from the
 *     current frontier), "log n" is the paper's 1 + log2(n+1) taken as
 *     1 + floor(log2(q+1)), and n/rho is rounded up:
 *         s = min(4096, 10 * (ceil(q/rho') + 1 + floor(log2(q+1))));
 *   - sample j (0 <= j < s) reads position floor(h_j * q / 2^64) of the list,
 *     h_j = splitmix64 output number (step * 2^32 + j) from state `seed`
 *     (uniform, with replacement);
 *   - theta = sorted_samples[min(s-1, floor(rho' * s / q))] (0-based rank);
 *   - when q <= rho' every queued vertex is extracted; theta = UINT64_MAX
 *     selects exactly the same set as the largest queued key.
 */
uint64_t oracle_rho_extdist_capped(const uint32_t* queue, uint32_t q, const uint64_t* dist,
                                   uint32_t n, uint64_t rho, uint64_t seed, uint64_t step,
                                   uint32_t dense_before, uint32_t reduced, uint32_t max_samples);

uint64_t oracle_rho_extdist(const uint32_t* queue, uint32_t q, const uint64_t* dist,
                            uint32_t n, uint64_t rho, uint64_t seed, uint64_t step,
                            uint32_t dense_before, uint32_t reduced)
{
    return oracle_rho_extdist_capped(queue, q, dist, n, rho, seed, step, dense_before, reduced,
                                     ORC_MAX_SAMPLES);
}

/*
 * The same rule with the sample count capped at max_samples (1 ..
 * ORC_MAX_SAMPLES) instead of 4096: s = min(max_samples, 10 * (ceil(q/rho')
 * + 1 + floor(log2(q+1)))), the rank taken from that s.  The warm-up steps of
 * oracle_stepping use 1024 (a reading of this library, see oracle_stepping).
 */
uint64_t oracle_rho_extdist_capped(const uint32_t* queue, uint32_t q, const uint64_t* dist,
                                   uint32_t n, uint64_t rho, uint64_t seed, uint64_t step,
                                   uint32_t dense_before, uint32_t reduced, uint32_t max_samples)
{
    if (max_samples < 1 || max_samples > ORC_MAX_SAMPLES) max_samples = ORC_MAX_SAMPLES;
    uint64_t rho_eff = rho;
    if ((uint64_t)q * 20u > (uint64_t)n && dense_before < reduced) {
        rho_eff = rho / 10u;
        if (rho_eff < 1) rho_eff = 1;
    }
    if ((uint64_t)q <= rho_eff) return ORC_INF;
    uint64_t s = 10u * ((q + rho_eff - 1) / rho_eff + 1u + floor_log2_u64((uint64_t)q + 1u));
    if (s > max_samples) s = max_samples;
    uint64_t keys[ORC_MAX_SAMPLES];
    for (uint64_t j = 0; j < s; ++j) {
        uint64_t h = oracle_splitmix64(seed, (step << 32) | j);
        uint64_t pos = (uint64_t)(((unsigned __int128)h * (unsigned __int128)q) >> 64);
        keys[j] = dist[queue[pos]];
    }
    qsort(keys, (size_t)s, sizeof(uint64_t), cmp_u64);
    uint64_t r = rho_eff * s / (uint64_t)q;
    if (r > s - 1) r = s - 1;
    return keys[r];
}

/*
 * Delta*-Stepping threshold (Table 2: theta <- i*Delta, no FinishCheck, so i
 * advances every step).  Readings: i starts at 1; when no queued key is
 * <= i*Delta, i jumps to ceil(qmin/Delta) so that no step is empty; the
 * product saturates at UINT64_MAX.  *i is updated to the value for the next
 * step.  qmin is the smallest key in Q.
 */
uint64_t oracle_delta_extdist(uint64_t* i, uint64_t delta, uint64_t qmin)
{
    uint64_t cur = *i;
    uint64_t theta = (cur > UINT64_MAX / delta) ? ORC_INF : cur * delta;
    if (qmin > theta) {
        cur = qmin / delta + ((qmin % delta) != 0);
        theta = (cur > UINT64_MAX / delta) ? ORC_INF : cur * delta;
    }
    *i = cur + 1;
    return theta;
}

/*
 * Original Delta-Stepping (Table 2: theta <- i*Delta; FinishCheck: if no new
 * delta[v] < i*Delta, i <- i+1).  Readings: i starts at 1; "new delta[v]" are
 * the values written by successful WriteMin calls of the step just finished;
 * when i advances past an empty bucket it jumps to ceil(qmin/Delta) at the
 * next ExtDist (as for Delta*).  oracle_delta_theta returns theta for the
 * current i (applying the jump); oracle_delta_finish applies FinishCheck.
 */
uint64_t oracle_delta_theta(uint64_t* i, uint64_t delta, uint64_t qmin)
{
    uint64_t cur = *i;
    uint64_t theta = (cur > UINT64_MAX / delta) ? ORC_INF : cur * delta;
    if (qmin > theta) {
        cur = qmin / delta + ((qmin % delta) != 0);
        theta = (cur > UINT64_MAX / delta) ? ORC_INF : cur * delta;
    }
    *i = cur;
    return theta;
}

void oracle_delta_finish(uint64_t* i, uint64_t theta, uint64_t min_new)
{
    if (!(min_new < theta)) *i += 1;
}

/* Statistics of one oracle_stepping run. */
typedef struct {
    uint64_t steps;          /* iterations of the while loop of Algorithm 1 */
    uint64_t extracted;      /* total ids returned by Extract over all steps */
    uint64_t edges;          /* total out-edges scanned by extracted ids      */
    uint64_t updates;        /* successful WriteMin calls                     */
    uint64_t full_steps;     /* rho: steps with |Q| > rho' (sampled theta)    */
    uint64_t partial_steps;  /* rho: steps with |Q| <= rho' (extract all)     */
    uint32_t max_ext;        /* max over v of the times v was extracted       */
    uint32_t pad;
} oracle_stats;

enum { ORC_RHO = 0, ORC_DELTA_STAR = 1, ORC_BELLMAN_FORD = 2, ORC_DELTA = 3, ORC_DIJKSTRA = 4 };

/*
 * Algorithm 1 (the stepping framework), executed sequentially on the
 * array-based LaB-PQ of Sec. 4.3 (a flag per vertex; Update sets the flag and
 * appends the id, Extract scans the queued ids and packs those with key <=
 * theta).  algo selects the ExtDist (and FinishCheck) of Table 2:
 *   ORC_RHO          theta from oracle_rho_extdist (param = rho >= 1;
 *                    rho_reduced = dense steps that use rho/10, the paper's 2;
 *                    the first warm_steps steps use rho = warm_rho instead,
 *                    without the reduction, from at most 1024 samples, and
 *                    are not counted as dense steps -- warm_steps = 0 is the
 *                    paper's schedule)
 *   ORC_DELTA_STAR   theta from oracle_delta_extdist (param = Delta >= 1)
 *   ORC_BELLMAN_FORD theta = +infinity (param ignored)
 *   ORC_DELTA        theta = i*Delta with FinishCheck (oracle_delta_theta /
 *                    oracle_delta_finish; param = Delta >= 1)
 *   ORC_DIJKSTRA     theta = min over Q of delta (param ignored)
 * Only ORC_DELTA has a FinishCheck.  The relaxation reads delta[u] when it
 * relaxes (Algorithm 1's WriteMin line), and WriteMin succeeds only on a
 * strictly smaller value (Sec. 2, the WriteMin definition).
 * ext_count (optional, n entries) receives how often each vertex was
 * extracted.  Returns 0, or -1 on bad arguments.
 */
int oracle_stepping(uint32_t n, const uint64_t* off, const uint32_t* tgt,
                    const uint32_t* w, uint32_t s, int algo, uint64_t param,
                    uint64_t seed, uint32_t rho_reduced, uint32_t warm_steps, uint64_t warm_rho,
                    uint64_t* dist, uint32_t* ext_count, oracle_stats* st)
{
    if (s >= n) return -1;
    if (algo == ORC_RHO && warm_steps > 0 && warm_rho == 0) return -1;
    if (algo != ORC_BELLMAN_FORD && algo != ORC_DIJKSTRA && param == 0) return -1;
    if (algo < 0 || algo > 4) return -1;
    uint8_t* inq = (uint8_t*)calloc(n, 1);
    uint32_t* Q = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t* F = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t* cnt = (uint32_t*)calloc(n, sizeof(uint32_t));
    if (!inq || !Q || !F || !cnt) { free(inq); free(Q); free(F); free(cnt); return -1; }
    oracle_stats z;
    memset(&z, 0, sizeof z);

    /* delta <- +inf; delta[s] <- 0; Q.Update(s) */
    for (uint32_t v = 0; v < n; ++v) dist[v] = ORC_INF;
    dist[s] = 0;
    uint32_t qlen = 0;
    inq[s] = 1;
    Q[qlen++] = s;

    uint64_t delta_i = 1;
    uint32_t dense_seen = 0;
    while (qlen > 0) {
        z.steps++;
        /* ExtDist */
        uint64_t theta;
        uint64_t qmin = ORC_INF;
        for (uint32_t i = 0; i < qlen; ++i)
            if (dist[Q[i]] < qmin) qmin = dist[Q[i]];
        if (algo == ORC_BELLMAN_FORD) {
            theta = ORC_INF;
        } else if (algo == ORC_DELTA_STAR) {
            theta = oracle_delta_extdist(&delta_i, param, qmin);
        } else if (algo == ORC_DELTA) {
            theta = oracle_delta_theta(&delta_i, param, qmin);
        } else if (algo == ORC_DIJKSTRA) {
            theta = qmin;
        } else if (z.steps <= warm_steps) {
            /* warm-up step: rho = warm_rho, no dense-step reduction */
            theta = oracle_rho_extdist_capped(Q, qlen, dist, n, warm_rho, seed, z.steps, 0, 0, ORC_WARM_SAMPLES);
            if ((uint64_t)qlen <= warm_rho) z.partial_steps++; else z.full_steps++;
        } else {
            int dense = (uint64_t)qlen * 20u > (uint64_t)n;
            uint64_t rho_eff = param;
            if (dense && dense_seen < rho_reduced) { rho_eff = param / 10u; if (rho_eff < 1) rho_eff = 1; }
            theta = oracle_rho_extdist(Q, qlen, dist, n, param, seed, z.steps, dense_seen, rho_reduced);
            if ((uint64_t)qlen <= rho_eff) z.partial_steps++; else z.full_steps++;
            if (dense) dense_seen++;
        }
        /* Extract(theta): ids with key <= theta leave Q (flag cleared) */
        uint32_t flen = 0, keep = 0;
        for (uint32_t i = 0; i < qlen; ++i) {
            uint32_t v = Q[i];
            if (dist[v] <= theta) { inq[v] = 0; F[flen++] = v; }
            else Q[keep++] = v;
        }
        qlen = keep;
        z.extracted += flen;
        uint64_t min_new = ORC_INF;
        /* relax the out-edges of every extracted id */
        for (uint32_t i = 0; i < flen; ++i) {
            uint32_t u = F[i];
            cnt[u]++;
            z.edges += off[u + 1] - off[u];
            for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
                uint32_t v = tgt[e];
                uint64_t cand = dist[u] + (uint64_t)w[e];
                if (cand < dist[v]) {           /* WriteMin succeeded */
                    dist[v] = cand;
                    z.updates++;
                    if (cand < min_new) min_new = cand;
                    if (!inq[v]) { inq[v] = 1; Q[qlen++] = v; } /* Update(v) */
                }
            }
        }
        if (algo == ORC_DELTA) oracle_delta_finish(&delta_i, theta, min_new); /* FinishCheck */
    }
    for (uint32_t v = 0; v < n; ++v) if (cnt[v] > z.max_ext) z.max_ext = cnt[v];
    if (ext_count) memcpy(ext_count, cnt, sizeof(uint32_t) * (size_t)n);
    if (st) *st = z;
    free(inq); free(Q); free(F); free(cnt);
    return 0;
}

/*
 * The LaB-PQ interface as a plain set (Sec. 3.1, Table 1): Q holds the ids
 * with inq[id] = 1; the key of id is key[id].  Extract(theta) returns every id
 * in Q whose key is <= theta, in increasing id order, and removes it from Q;
 * Reduce returns the smallest key in Q (UINT64_MAX for an empty Q).  This is
 * the definition that any implementation -- the array of Sec. 4.3 or the
 * tournament tree of Sec. 4.2 -- must reproduce; O(n) per call.
 */
uint32_t oracle_lbpq_extract(uint32_t n, uint8_t* inq, const uint64_t* key, uint64_t theta, uint32_t* out)
{
    uint32_t c = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (inq[v] && key[v] <= theta) { inq[v] = 0; out[c++] = v; }
    return c;
}

uint64_t oracle_lbpq_min(uint32_t n, const uint8_t* inq, const uint64_t* key)
{
    uint64_t m = ORC_INF;
    for (uint32_t v = 0; v < n; ++v)
        if (inq[v] && key[v] < m) m = key[v];
    return m;
}
