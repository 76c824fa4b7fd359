/*
 * graphgen.c -- seeded synthetic graph generators (input side only).
 *
 * These build the CSR inputs that stand in for the paper's workloads: the
 * power-law social/web graphs (RMAT), the road networks (a jittered,
 * bond-percolated grid) and plain grids (Sec. 7 "Experimental setup": social
 * and web weights uniform in [1, 2^18), road weights derived from geometry).
 * No SSSP arithmetic lives here.  Every random choice is a pure function of
 * (seed, index) through splitmix64 (Steele, Lea, Flood 2014), so results do
 * not depend on thread count or platform.  Floating point (road geometry) is
 * compiled with -ffp-contract=off so x86-64 and AArch64 agree bit for bit.
 *
 * Output CSR: off[n+1] (uint64), tgt[m] and w[m] (uint32); the out-edges of
 * every vertex are sorted by target id; every graph produced here is
 * symmetric (each undirected edge stored in both directions with one weight)
 * and has no self-loops or duplicate edges.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static inline uint64_t gg_sm64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t gg_mulhi(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* Weight of the undirected edge {u,v}: uniform in [1, wmax_excl) via the
 * multiply-high reduction of a 64-bit hash of the ordered pair (min, max). */
static inline uint32_t gg_pair_weight(uint64_t seed, uint32_t u, uint32_t v, uint32_t wmax_excl)
{
    uint32_t a = u < v ? u : v, b = u < v ? v : u;
    uint64_t h = gg_sm64(seed, ((uint64_t)a << 32) | b);
    return 1u + (uint32_t)gg_mulhi(h, (uint64_t)(wmax_excl - 1u));
}

void graphgen_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* 4-neighbour R x C grid, id = r*C + c, both directions stored.            */
/* ------------------------------------------------------------------------ */
uint64_t graphgen_grid_edges(uint32_t R, uint32_t C)
{
    return 2ull * ((uint64_t)R * (C ? C - 1 : 0) + (uint64_t)C * (R ? R - 1 : 0));
}

/* Fills caller arrays (off: R*C+1, tgt/w: graphgen_grid_edges).  wmax_excl=0
 * gives unit weights. */
int graphgen_grid(uint32_t R, uint32_t C, uint64_t wseed, uint32_t wmax_excl,
                  uint64_t* off, uint32_t* tgt, uint32_t* w)
{
    uint64_t e = 0;
    for (uint32_t r = 0; r < R; ++r) {
        for (uint32_t c = 0; c < C; ++c) {
            uint32_t id = r * C + c;
            off[id] = e;
            uint32_t nb[4];
            int k = 0;
            if (r > 0) nb[k++] = id - C;
            if (c > 0) nb[k++] = id - 1;
            if (c + 1 < C) nb[k++] = id + 1;
            if (r + 1 < R) nb[k++] = id + C;
            for (int j = 0; j < k; ++j) {
                tgt[e] = nb[j];
                w[e] = wmax_excl ? gg_pair_weight(wseed, id, nb[j], wmax_excl) : 1u;
                ++e;
            }
        }
    }
    off[(uint64_t)R * C] = e;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sorting helpers: LSD radix sort of 64-bit keys on their low `bits` bits. */
/* ------------------------------------------------------------------------ */
static int gg_radix_sort(uint64_t* keys, uint64_t count, int bits)
{
    uint64_t* tmp = (uint64_t*)malloc(sizeof(uint64_t) * (count ? count : 1));
    if (!tmp) return -1;
    const int D = 11;
    uint64_t* src = keys;
    uint64_t* dst = tmp;
#ifdef _OPENMP
    int T = omp_get_max_threads();
#else
    int T = 1;
#endif
    if (count < (1u << 20)) T = 1;
    uint64_t* hist = (uint64_t*)malloc(sizeof(uint64_t) * 2048u * (size_t)T);
    if (!hist) { free(tmp); return -1; }
    for (int shift = 0; shift < bits; shift += D) {
        /* stable LSD pass: thread t owns the contiguous chunk [lo_t, hi_t) */
        memset(hist, 0, sizeof(uint64_t) * 2048u * (size_t)T);
#ifdef _OPENMP
#pragma omp parallel num_threads(T)
#endif
        {
#ifdef _OPENMP
            int t = omp_get_thread_num();
#else
            int t = 0;
#endif
            uint64_t lo = count * (uint64_t)t / (uint64_t)T, hi = count * (uint64_t)(t + 1) / (uint64_t)T;
            uint64_t* h = hist + 2048u * (size_t)t;
            for (uint64_t i = lo; i < hi; ++i) h[(src[i] >> shift) & 2047u]++;
#ifdef _OPENMP
#pragma omp barrier
#pragma omp single
#endif
            {
                uint64_t sum = 0;
                for (int d = 0; d < 2048; ++d)
                    for (int tt = 0; tt < T; ++tt) {
                        uint64_t c = hist[2048u * (size_t)tt + d];
                        hist[2048u * (size_t)tt + d] = sum;
                        sum += c;
                    }
            }
            for (uint64_t i = lo; i < hi; ++i) dst[h[(src[i] >> shift) & 2047u]++] = src[i];
        }
        uint64_t* t = src; src = dst; dst = t;
    }
    if (src != keys) memcpy(keys, src, sizeof(uint64_t) * count);
    free(hist);
    free(tmp);
    return 0;
}

/* Turns a sorted, unique list of directed pairs key = (u << sh) | v into CSR
 * with pair weights.  Allocates *off, *tgt, *w. */
static int gg_keys_to_csr(const uint64_t* keys, uint64_t m, uint32_t n, int sh,
                          uint64_t wseed, uint32_t wmax_excl,
                          uint64_t** off_out, uint32_t** tgt_out, uint32_t** w_out)
{
    uint64_t* off = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    uint32_t* tgt = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* w = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!off || !tgt || !w) { free(off); free(tgt); free(w); return -1; }
    uint64_t mask = (sh >= 64) ? ~0ull : ((1ull << sh) - 1u);
    for (uint64_t i = 0; i < m; ++i) off[(uint32_t)(keys[i] >> sh) + 1]++;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t u = (uint32_t)(keys[i] >> sh), v = (uint32_t)(keys[i] & mask);
        tgt[i] = v;
        w[i] = wmax_excl ? gg_pair_weight(wseed, u, v, wmax_excl) : 1u;
    }
    for (uint32_t u = 0; u < n; ++u) off[u + 1] += off[u];
    *off_out = off; *tgt_out = tgt; *w_out = w;
    return 0;
}

/* Symmetrise `cnt` pairs held as key=(u<<sh)|v in keys[0..cnt), keys having
 * room for 2*cnt entries: drop self-loops, add reversed copies, sort, unique.
 * Returns the final count. */
static int64_t gg_symmetrise(uint64_t* keys, uint64_t cnt, int sh)
{
    uint64_t mask = (1ull << sh) - 1u;
    uint64_t k = 0;
    for (uint64_t i = 0; i < cnt; ++i) {
        uint64_t u = keys[i] >> sh, v = keys[i] & mask;
        if (u != v) keys[k++] = keys[i];
    }
    uint64_t half = k;
    for (uint64_t i = 0; i < half; ++i) {
        uint64_t u = keys[i] >> sh, v = keys[i] & mask;
        keys[k++] = (v << sh) | u;
    }
    if (gg_radix_sort(keys, k, 2 * sh)) return -1;
    uint64_t out = 0;
    for (uint64_t i = 0; i < k; ++i)
        if (out == 0 || keys[i] != keys[out - 1]) keys[out++] = keys[i];
    return (int64_t)out;
}

/* ------------------------------------------------------------------------ */
/* RMAT (Chakrabarti, Zhan, Faloutsos 2004), Graph500-style: ef * 2^scale   */
/* edge draws, `scale` quadrant choices each with probabilities (a,b,c,d),  */
/* no noise, then a seeded random relabelling of the vertices, then         */
/* symmetrise, drop self-loops, sort, unique.                                */
/* ------------------------------------------------------------------------ */
int graphgen_rmat_n(uint32_t scale, uint32_t edgefactor, double a, double b, double c,
                    uint64_t gen_seed, uint64_t wseed, uint32_t wmax_excl, uint32_t n_keep,
                    uint32_t* n_out, uint64_t* m_out,
                    uint64_t** off, uint32_t** tgt, uint32_t** w);

int graphgen_rmat(uint32_t scale, uint32_t edgefactor, double a, double b, double c,
                  uint64_t gen_seed, uint64_t wseed, uint32_t wmax_excl,
                  uint32_t* n_out, uint64_t* m_out,
                  uint64_t** off, uint32_t** tgt, uint32_t** w)
{
    return graphgen_rmat_n(scale, edgefactor, a, b, c, gen_seed, wseed, wmax_excl, 0,
                           n_out, m_out, off, tgt, w);
}

/* As graphgen_rmat; when 0 < n_keep < 2^scale, edges with an endpoint >= n_keep
 * (after the relabelling) are rejected and the graph has n_keep vertices. */
int graphgen_rmat_n(uint32_t scale, uint32_t edgefactor, double a, double b, double c,
                    uint64_t gen_seed, uint64_t wseed, uint32_t wmax_excl, uint32_t n_keep,
                    uint32_t* n_out, uint64_t* m_out,
                    uint64_t** off, uint32_t** tgt, uint32_t** w)
{
    if (scale < 1 || scale > 30) return -1;
    uint32_t n = 1u << scale;
    uint64_t E = (uint64_t)edgefactor << scale;
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (2 * E ? 2 * E : 1));
    uint32_t* perm = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    if (!keys || !perm) { free(keys); free(perm); return -1; }
    const uint64_t two32 = 4294967296ull;
    uint64_t ta = (uint64_t)(a * (double)two32);
    uint64_t tb = ta + (uint64_t)(b * (double)two32);
    uint64_t tc = tb + (uint64_t)(c * (double)two32);
    uint64_t per_edge = (scale + 1) / 2;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint64_t e = 0; e < E; ++e) {
        uint32_t u = 0, v = 0;
        uint64_t h = 0;
        for (uint32_t lvl = 0; lvl < scale; ++lvl) {
            if ((lvl & 1u) == 0) h = gg_sm64(gen_seed, e * per_edge + lvl / 2);
            uint64_t r = (lvl & 1u) ? (h >> 32) : (h & 0xFFFFFFFFull);
            uint32_t bu, bv;
            if (r < ta) { bu = 0; bv = 0; }
            else if (r < tb) { bu = 0; bv = 1; }
            else if (r < tc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        keys[e] = ((uint64_t)u << scale) | v;
    }
    /* random relabelling: Fisher-Yates driven by a second splitmix stream */
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    uint64_t pseed = gen_seed ^ 0xA5A5A5A55A5A5A5AULL;
    for (uint32_t i = n - 1; i > 0; --i) {
        uint32_t j = (uint32_t)gg_mulhi(gg_sm64(pseed, i), (uint64_t)i + 1u);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    uint64_t mask = ((uint64_t)1 << scale) - 1u;
    uint32_t nk = (n_keep > 0 && n_keep < n) ? n_keep : n;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint64_t e = 0; e < E; ++e) {
        uint32_t u = perm[keys[e] >> scale], v = perm[keys[e] & mask];
        keys[e] = (u >= nk || v >= nk) ? ~0ull : (((uint64_t)u << scale) | v);
    }
    uint64_t kept = 0;
    for (uint64_t e = 0; e < E; ++e)
        if (keys[e] != ~0ull) keys[kept++] = keys[e];
    free(perm);
    int64_t m = gg_symmetrise(keys, kept, (int)scale);
    if (m < 0) { free(keys); return -1; }
    int rc = gg_keys_to_csr(keys, (uint64_t)m, nk, (int)scale, wseed, wmax_excl, off, tgt, w);
    free(keys);
    if (rc) return rc;
    n = nk;
    *n_out = n;
    *m_out = (uint64_t)m;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Road-like graph: side x side grid of points, each jittered uniformly      */
/* within +-jitter of its cell centre; every right/down neighbour edge kept  */
/* with probability keep_num/2^64 (one draw per undirected edge); weight =   */
/* floor(scale * Euclidean length) + 1.                                     */
/* ------------------------------------------------------------------------ */
static inline double gg_unit(uint64_t h) { return (double)(h >> 11) * (1.0 / 9007199254740992.0); }

int graphgen_road_w(uint32_t side, uint64_t keep_num, double jitter, double wscale,
                    uint64_t seed, uint32_t wmax_excl, uint64_t wseed, uint32_t* n_out, uint64_t* m_out,
                    uint64_t** off_out, uint32_t** tgt_out, uint32_t** w_out);

int graphgen_road(uint32_t side, uint64_t keep_num, double jitter, double wscale,
                  uint64_t seed, uint32_t* n_out, uint64_t* m_out,
                  uint64_t** off_out, uint32_t** tgt_out, uint32_t** w_out)
{
    return graphgen_road_w(side, keep_num, jitter, wscale, seed, 0, 0, n_out, m_out, off_out, tgt_out, w_out);
}

/* As graphgen_road; wmax_excl > 0 replaces the geometric weights by weights
 * uniform in [1, wmax_excl) drawn from wseed (same topology). */
int graphgen_road_w(uint32_t side, uint64_t keep_num, double jitter, double wscale,
                    uint64_t seed, uint32_t wmax_excl, uint64_t wseed, uint32_t* n_out, uint64_t* m_out,
                    uint64_t** off_out, uint32_t** tgt_out, uint32_t** w_out)
{
    uint64_t n64 = (uint64_t)side * side;
    if (side == 0 || n64 > 0xFFFFFFFFull) return -1;
    uint32_t n = (uint32_t)n64;
    double* px = (double*)malloc(sizeof(double) * n64);
    double* py = (double*)malloc(sizeof(double) * n64);
    uint8_t* keep = (uint8_t*)malloc(n64); /* bit0: right edge, bit1: down edge */
    uint64_t* off = (uint64_t*)calloc(n64 + 1, sizeof(uint64_t));
    if (!px || !py || !keep || !off) { free(px); free(py); free(keep); free(off); return -1; }
    uint64_t pseed = seed, eseed = seed ^ 0x5DEECE66DULL;
    for (uint32_t r = 0; r < side; ++r)
        for (uint32_t c = 0; c < side; ++c) {
            uint64_t id = (uint64_t)r * side + c;
            double jx = -jitter + 2.0 * jitter * gg_unit(gg_sm64(pseed, 2 * id));
            double jy = -jitter + 2.0 * jitter * gg_unit(gg_sm64(pseed, 2 * id + 1));
            px[id] = (double)c + jx;
            py[id] = (double)r + jy;
            uint8_t k = 0;
            if (c + 1 < side && gg_sm64(eseed, 2 * id) < keep_num) k |= 1;
            if (r + 1 < side && gg_sm64(eseed, 2 * id + 1) < keep_num) k |= 2;
            keep[id] = k;
        }
    /* degrees */
    for (uint32_t r = 0; r < side; ++r)
        for (uint32_t c = 0; c < side; ++c) {
            uint64_t id = (uint64_t)r * side + c;
            if (keep[id] & 1) { off[id + 1]++; off[id + 2]++; }
            if (keep[id] & 2) { off[id + 1]++; off[id + side + 1]++; }
        }
    for (uint64_t i = 0; i < n64; ++i) off[i + 1] += off[i];
    uint64_t m = off[n64];
    uint32_t* tgt = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* w = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!tgt || !w) { free(px); free(py); free(keep); free(off); free(tgt); free(w); return -1; }
    for (uint32_t r = 0; r < side; ++r)
        for (uint32_t c = 0; c < side; ++c) {
            uint64_t id = (uint64_t)r * side + c;
            uint64_t e = off[id];
            uint64_t nb[4];
            int k = 0;
            if (r > 0 && (keep[id - side] & 2)) nb[k++] = id - side;
            if (c > 0 && (keep[id - 1] & 1)) nb[k++] = id - 1;
            if (keep[id] & 1) nb[k++] = id + 1;
            if (keep[id] & 2) nb[k++] = id + side;
            for (int j = 0; j < k; ++j) {
                double dx = px[nb[j]] - px[id];
                double dy = py[nb[j]] - py[id];
                double len = sqrt(dx * dx + dy * dy);
                tgt[e] = (uint32_t)nb[j];
                w[e] = wmax_excl ? gg_pair_weight(wseed, (uint32_t)id, (uint32_t)nb[j], wmax_excl)
                                 : (uint32_t)floor(wscale * len) + 1u;
                ++e;
            }
        }
    free(px); free(py); free(keep);
    *n_out = n; *m_out = m;
    *off_out = off; *tgt_out = tgt; *w_out = w;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Uniform random multigraph for tests: m directed edges (u,v) with u, v     */
/* uniform, weights uniform in [wlo, whi] (inclusive); self-loops and       */
/* duplicates are kept unless the flags drop them.  Not symmetric.           */
/* ------------------------------------------------------------------------ */
int graphgen_random(uint32_t n, uint64_t m, uint32_t wlo, uint32_t whi, uint64_t seed,
                    int drop_self_loops, uint64_t* m_out,
                    uint64_t** off_out, uint32_t** tgt_out, uint32_t** w_out)
{
    if (n == 0 || whi < wlo) return -1;
    uint64_t* us = (uint64_t*)malloc(sizeof(uint64_t) * (m ? m : 1));
    uint64_t* off = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    uint32_t* tgt = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* w = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    if (!us || !off || !tgt || !w) { free(us); free(off); free(tgt); free(w); return -1; }
    uint64_t k = 0;
    for (uint64_t e = 0; e < m; ++e) {
        uint32_t u = (uint32_t)gg_mulhi(gg_sm64(seed, 3 * e), n);
        uint32_t v = (uint32_t)gg_mulhi(gg_sm64(seed, 3 * e + 1), n);
        uint64_t span = (uint64_t)whi - wlo + 1u;
        uint32_t ww = wlo + (uint32_t)gg_mulhi(gg_sm64(seed, 3 * e + 2), span);
        if (drop_self_loops && u == v) continue;
        us[k] = ((uint64_t)u << 32) | v;
        tgt[k] = ww; /* weight parked in tgt for the bucket pass */
        ++k;
    }
    /* bucket by source, stable */
    for (uint64_t i = 0; i < k; ++i) off[(us[i] >> 32) + 1]++;
    for (uint32_t u = 0; u < n; ++u) off[u + 1] += off[u];
    uint64_t* pos = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint32_t* t2 = (uint32_t*)malloc(sizeof(uint32_t) * (k ? k : 1));
    if (!pos || !t2) { free(us); free(off); free(tgt); free(w); free(pos); free(t2); return -1; }
    memcpy(pos, off, sizeof(uint64_t) * ((size_t)n + 1));
    for (uint64_t i = 0; i < k; ++i) {
        uint64_t p = pos[us[i] >> 32]++;
        t2[p] = (uint32_t)(us[i] & 0xFFFFFFFFu);
        w[p] = tgt[i];
    }
    free(tgt); free(us); free(pos);
    *m_out = k; *off_out = off; *tgt_out = t2; *w_out = w;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Connected components of the undirected view (union-find), used to draw   */
/* sources from the largest component.  label[v] = 1 for v in the largest   */
/* component, else 0.  Returns the largest component's size.                */
/* ------------------------------------------------------------------------ */
static uint32_t gg_find(uint32_t* p, uint32_t x)
{
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

int64_t graphgen_largest_cc(uint32_t n, const uint64_t* off, const uint32_t* tgt, uint8_t* label)
{
    uint32_t* p = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n ? n : 1));
    uint32_t* sz = (uint32_t*)calloc(n ? n : 1, sizeof(uint32_t));
    if (!p || !sz) { free(p); free(sz); return -1; }
    for (uint32_t v = 0; v < n; ++v) p[v] = v;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t a = gg_find(p, u), b = gg_find(p, tgt[e]);
            if (a != b) { if (a < b) p[b] = a; else p[a] = b; }
        }
    uint32_t best = 0, bestsz = 0;
    for (uint32_t v = 0; v < n; ++v) sz[gg_find(p, v)]++;
    for (uint32_t v = 0; v < n; ++v)
        if (sz[v] > bestsz) { bestsz = sz[v]; best = v; }
    for (uint32_t v = 0; v < n; ++v) label[v] = (gg_find(p, v) == best);
    free(p); free(sz);
    return (int64_t)bestsz;
}

/* The k-th vertex (0-based, in id order) among those with label[v] != 0. */
int64_t graphgen_kth_labelled(uint32_t n, const uint8_t* label, uint64_t k)
{
    for (uint32_t v = 0; v < n; ++v)
        if (label[v]) { if (k == 0) return v; --k; }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* k-nearest-neighbour graph of points from a 3-D mixture of `clusters`      */
/* clusters: centres uniform in the unit cube, offsets sigma * z per         */
/* coordinate with z the Irwin-Hall sum of 12 uniforms minus 6 (an           */
/* approximately standard normal variate built from uniforms only, so the    */
/* points are bit-identical on every platform); a point outside the cube is  */
/* redrawn.  Each point links to its k nearest other points (Euclidean,      */
/* ties by index); the union is symmetrised; w = floor(wscale * d) + 1.      */
/* ------------------------------------------------------------------------ */
static double gg_irwin_hall(uint64_t seed, uint64_t base)
{
    double s = 0.0;
    for (int j = 0; j < 12; ++j) s += gg_unit(gg_sm64(seed, base + (uint64_t)j));
    return s - 6.0;
}

int graphgen_knn(uint32_t npts, uint32_t clusters, double sigma, uint32_t k, double wscale, uint64_t seed,
                 uint64_t* m_out, uint64_t** off_out, uint32_t** tgt_out, uint32_t** w_out, double* xyz_out)
{
    if (npts < 2 || clusters == 0 || k == 0 || k >= npts) return -1;
    const uint32_t n = npts;
    double* P = xyz_out ? xyz_out : (double*)malloc(sizeof(double) * 3 * (size_t)n);
    double* C = (double*)malloc(sizeof(double) * 3 * (size_t)clusters);
    if (!P || !C) { if (!xyz_out) free(P); free(C); return -1; }
    const uint64_t cseed = seed ^ 0x1234567887654321ULL;
    for (uint32_t j = 0; j < clusters; ++j)
        for (int d = 0; d < 3; ++d) C[3 * j + d] = gg_unit(gg_sm64(cseed, 3ull * j + d));
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (uint32_t i = 0; i < n; ++i) {
        const uint32_t cl = (uint32_t)gg_mulhi(gg_sm64(seed, (uint64_t)i << 20), clusters);
        for (uint64_t attempt = 0;; ++attempt) {
            const uint64_t base = ((uint64_t)i << 20) + 1 + attempt * 36;
            double x = C[3 * cl] + sigma * gg_irwin_hall(seed, base);
            double y = C[3 * cl + 1] + sigma * gg_irwin_hall(seed, base + 12);
            double z = C[3 * cl + 2] + sigma * gg_irwin_hall(seed, base + 24);
            if (x >= 0.0 && x < 1.0 && y >= 0.0 && y < 1.0 && z >= 0.0 && z < 1.0) {
                P[3 * (size_t)i] = x; P[3 * (size_t)i + 1] = y; P[3 * (size_t)i + 2] = z;
                break;
            }
        }
    }
    free(C);
    /* uniform grid, G^3 cells; points sorted by cell */
    const uint32_t G = 128;
    const double h = 1.0 / G;
    uint64_t ncell = (uint64_t)G * G * G;
    uint32_t* cstart = (uint32_t*)calloc(ncell + 1, sizeof(uint32_t));
    uint32_t* order = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    uint32_t* cellof = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n);
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (size_t)n * k);
    if (!cstart || !order || !cellof || !keys) {
        free(cstart); free(order); free(cellof); free(keys); if (!xyz_out) free(P); return -1;
    }
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t cx = (uint32_t)(P[3 * (size_t)i] * G), cy = (uint32_t)(P[3 * (size_t)i + 1] * G),
                 cz = (uint32_t)(P[3 * (size_t)i + 2] * G);
        if (cx >= G) cx = G - 1;
        if (cy >= G) cy = G - 1;
        if (cz >= G) cz = G - 1;
        cellof[i] = (cz * G + cy) * G + cx;
        cstart[cellof[i] + 1]++;
    }
    for (uint64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
    {
        uint32_t* pos = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)ncell);
        if (!pos) { free(cstart); free(order); free(cellof); free(keys); if (!xyz_out) free(P); return -1; }
        memcpy(pos, cstart, sizeof(uint32_t) * (size_t)ncell);
        for (uint32_t i = 0; i < n; ++i) order[pos[cellof[i]]++] = i;  /* ascending index within a cell */
        free(pos);
    }
    const int scale = 1 + (int)(63 - __builtin_clzll((unsigned long long)n));  /* bits for an id */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (uint32_t i = 0; i < n; ++i) {
        /* k best (d2, index) kept sorted ascending */
        double bd[64];
        uint32_t bi[64];
        uint32_t cnt = 0;
        const double px = P[3 * (size_t)i], py = P[3 * (size_t)i + 1], pz = P[3 * (size_t)i + 2];
        const int cx = (int)(cellof[i] % G), cy = (int)((cellof[i] / G) % G), cz = (int)(cellof[i] / G / G);
        for (int r = 0; r < (int)G; ++r) {
            for (int dz = -r; dz <= r; ++dz)
                for (int dy = -r; dy <= r; ++dy)
                    for (int dx = -r; dx <= r; ++dx) {
                        if (dx != -r && dx != r && dy != -r && dy != r && dz != -r && dz != r) continue;
                        const int x = cx + dx, y = cy + dy, z = cz + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= (int)G || y >= (int)G || z >= (int)G) continue;
                        const uint32_t c = ((uint32_t)z * G + (uint32_t)y) * G + (uint32_t)x;
                        for (uint32_t t = cstart[c]; t < cstart[c + 1]; ++t) {
                            const uint32_t j = order[t];
                            if (j == i) continue;
                            const double ex = P[3 * (size_t)j] - px, ey = P[3 * (size_t)j + 1] - py,
                                         ez = P[3 * (size_t)j + 2] - pz;
                            const double d2 = ex * ex + ey * ey + ez * ez;
                            if (cnt == k && (d2 > bd[k - 1] || (d2 == bd[k - 1] && j > bi[k - 1]))) continue;
                            uint32_t q = cnt < k ? cnt++ : k - 1;
                            while (q > 0 && (bd[q - 1] > d2 || (bd[q - 1] == d2 && bi[q - 1] > j))) {
                                bd[q] = bd[q - 1]; bi[q] = bi[q - 1]; --q;
                            }
                            bd[q] = d2; bi[q] = j;
                        }
                    }
            /* every point beyond ring r is at least r*h away */
            if (cnt == k && bd[k - 1] <= ((double)r * h) * ((double)r * h)) break;
        }
        for (uint32_t q = 0; q < k; ++q)
            keys[(size_t)i * k + q] = ((uint64_t)i << scale) | (q < cnt ? bi[q] : i);
    }
    free(order); free(cellof); free(cstart);
    int64_t m = gg_symmetrise(keys, (uint64_t)n * k, scale);
    if (m < 0) { free(keys); if (!xyz_out) free(P); return -1; }
    uint64_t* off = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    uint32_t* tgt = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    uint32_t* w = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(m ? m : 1));
    if (!off || !tgt || !w) { free(off); free(tgt); free(w); free(keys); if (!xyz_out) free(P); return -1; }
    const uint64_t mask = (1ull << scale) - 1u;
    for (int64_t e = 0; e < m; ++e) off[(keys[e] >> scale) + 1]++;
    for (uint32_t u = 0; u < n; ++u) off[u + 1] += off[u];
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t e = 0; e < m; ++e) {
        const uint32_t u = (uint32_t)(keys[e] >> scale), v = (uint32_t)(keys[e] & mask);
        const uint32_t a = u < v ? u : v, b = u < v ? v : u;
        const double ex = P[3 * (size_t)a] - P[3 * (size_t)b], ey = P[3 * (size_t)a + 1] - P[3 * (size_t)b + 1],
                     ez = P[3 * (size_t)a + 2] - P[3 * (size_t)b + 2];
        tgt[e] = v;
        w[e] = (uint32_t)floor(wscale * sqrt(ex * ex + ey * ey + ez * ez)) + 1u;
    }
    free(keys);
    if (!xyz_out) free(P);
    *m_out = (uint64_t)m; *off_out = off; *tgt_out = tgt; *w_out = w;
    return 0;
}
