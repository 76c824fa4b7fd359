// sssp_tune.cu -- the autotuner of libsssp (host code).
//
// The paper fixes the parameter per graph family (rho = 2^21 for social and
// web graphs, 2^15 for road networks; Sec. 7) and reports the best rho of a
// sweep beside it.  This library measures instead: sssp_autotune times
// candidate configurations of the one persistent solve kernel on sample
// sources of the graph itself and keeps the fastest.  A configuration is an
// ExtDist rule with its parameter (rho-Stepping or Delta*-Stepping, Table 2),
// the kernel shape (SSSP_SHAPE_*), bidirectional relaxation (symmetric graphs,
// Sec. 6) and the local-relaxation budget of super-sparse steps (Sec. 6).  The
// distances never depend on the choice, only the time does.
//
// Search (every solve timed with CUDA events on the caller's stream):
//   1. every rule/parameter candidate (rho = n/4 ... n/1024 and Delta = mean
//      weight x 1/8 ... 8, factors of 2 apart), wide shape, no local
//      relaxation, on the first sample source;
//   2. the two fastest of (1) in both shapes, on up to three sources (as
//      every later stage);
//   3. sparse graphs (mean out-degree < 20): the three fastest of (1) of each
//      rule, in the winning shape with local budgets 64, 256 and 1024, and in
//      the narrow shape with fused super-sparse steps (SSSP_SOLVE_FUSED) with
//      local budgets 0, 64, 256 and 1024;
//   4. rho-Stepping winner: the number of dense steps that use rho/10 (the
//      paper's 2, then 4, 6, 8 and none), then 4, 6 or 8 warm-up steps at
//      rho = 256 (sssp_options.rho_warmup_steps), each with the count found,
//      2, 4 or 6 reduced dense steps after it;
//   5. the degree-bin cut-offs: small-degree bound 16 and 64 (default 32),
//      then chunk records of 128 and 512 edges (default 256);
//   6. the winner on every sample source (sssp_tuning.ms).
// The result is kept on the graph handle and in a per-class table (graph class
// = size, mean degree, degree skew and symmetry; sssp_graph_class), which
// sssp_solve_tuned and the batched and serving calls consult for graphs that
// were not tuned themselves.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>

#include "sssp_internal.h"

namespace {

std::mutex g_class_mu;
std::map<uint64_t, sssp_tuning> g_class_table;

int fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? SSSP_ERR_OUT_OF_MEMORY : SSSP_ERR_CUDA; }

uint32_t ceil_log2(uint64_t x)
{
    uint32_t l = 0;
    while ((1ull << l) < x && l < 63) ++l;
    return l;
}

struct Candidate {
    sssp_algo algo;
    uint64_t param;
    uint32_t shape;
    uint32_t local;
    double ms;
    uint32_t rho_reduced;   // sssp_options encoding (0 = the paper's 2)
    uint32_t small_deg;     // 0 = default
    uint32_t chunk;         // 0 = default
    uint32_t fused;         // 1 = SSSP_SOLVE_FUSED
    uint32_t warm_steps;    // sssp_options.rho_warmup_steps / rho_warmup
    uint32_t warm_rho;
};

// Mean time of one solve per source (ms); a failed solve is reported as rc.
int time_config(const sssp_graph* g, const Candidate& c, const uint32_t* srcs, uint32_t ns, uint64_t* dist,
                cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, double* ms_out)
{
    sssp_options o;
    memset(&o, 0, sizeof o);
    o.flags = ((g->flags & SSSP_GRAPH_SYMMETRIC) ? SSSP_SOLVE_BIDIRECTIONAL : 0u) | (c.fused ? SSSP_SOLVE_FUSED : 0u);
    o.shape = c.shape;
    o.local_budget = c.local;
    o.rho_reduced = c.rho_reduced;
    o.rho_warmup_steps = c.warm_steps;
    o.rho_warmup = c.warm_rho;
    o.small_deg = c.small_deg;
    o.chunk = c.chunk;
    double total = 0;
    for (uint32_t i = 0; i < ns; ++i) {
        cudaError_t e = cudaEventRecord(e0, st);
        if (e != cudaSuccess) return fail(e);
        int rc = sssp_solve_ex(g, srcs[i], c.algo, c.param, dist, &o, st);
        if (rc != SSSP_OK) return rc;
        if ((e = cudaEventRecord(e1, st)) != cudaSuccess) return fail(e);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) return fail(e);
        rc = sssp_last_status(g, st);
        if (rc != SSSP_OK) return rc;
        float t = 0;
        if ((e = cudaEventElapsedTime(&t, e0, e1)) != cudaSuccess) return fail(e);
        total += t;
    }
    *ms_out = total / ns;
    return SSSP_OK;
}

}  // namespace

uint64_t sssp_class_key(const sssp_graph* g)
{
    const double avg = g->n ? (double)g->m / (double)g->n : 0.0;
    const uint32_t lg_n = ceil_log2(g->n);
    const uint32_t lg_avg4 = avg > 1.0 ? (uint32_t)std::lround(4.0 * std::log2(avg)) : 0u;
    const uint32_t skew = (avg > 0.0 && g->max_deg > avg) ? (uint32_t)std::floor(std::log2((double)g->max_deg / avg)) : 0u;
    return (uint64_t)(lg_n & 0xFF) | ((uint64_t)(lg_avg4 & 0xFF) << 8) | ((uint64_t)(skew & 0xFF) << 16) |
           ((uint64_t)((g->flags & SSSP_GRAPH_SYMMETRIC) ? 1 : 0) << 24);
}

bool sssp_lookup_tuning(const sssp_graph* g, sssp_tuning* out)
{
    if (g->tuned) {
        *out = g->tuning;
        return true;
    }
    std::lock_guard<std::mutex> lk(g_class_mu);
    auto it = g_class_table.find(sssp_class_key(g));
    if (it == g_class_table.end()) return false;
    *out = it->second;
    return true;
}

uint64_t sssp_graph_param(const sssp_graph* g, sssp_algo algo)
{
    sssp_tuning t;
    if (sssp_lookup_tuning(g, &t) && t.algo == algo) return t.param;
    return sssp_default_param(g->n, g->m, algo, g->mean_w);
}

bool sssp_lookup_batch_tuning(const sssp_graph* g, sssp_tuning* out)
{
    if (g->batch_tuned) {
        *out = g->batch_tuning;
        return true;
    }
    return sssp_lookup_tuning(g, out);
}

uint64_t sssp_graph_batch_param(const sssp_graph* g, sssp_algo algo)
{
    sssp_tuning t;
    if (sssp_lookup_batch_tuning(g, &t) && t.algo == algo) return t.param;
    return sssp_default_param(g->n, g->m, algo, g->mean_w);
}

extern "C" {

int sssp_graph_class(const sssp_graph* g, uint64_t* key)
{
    if (!g || !key) return SSSP_ERR_INVALID_ARG;
    *key = sssp_class_key(g);
    return SSSP_OK;
}

int sssp_autotune(sssp_graph* g, const uint32_t* sources, uint32_t k, sssp_tuning* out, void* stream)
{
    return sssp_autotune_ex(g, sources, k, (1u << SSSP_RHO) | (1u << SSSP_DELTA_STAR), out, stream);
}

int sssp_autotune_ex(sssp_graph* g, const uint32_t* sources, uint32_t k, uint32_t rules, sssp_tuning* out,
                     void* stream)
{
    if (!g || !sources || k == 0) return SSSP_ERR_INVALID_ARG;
    if (rules == 0 || (rules & ~((1u << SSSP_RHO) | (1u << SSSP_DELTA_STAR)))) return SSSP_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < k; ++i)
        if (sources[i] >= g->n) return SSSP_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(g->device);
    if (e != cudaSuccess) return fail(e);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint64_t* dist = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&dist), sizeof(uint64_t) * (size_t)g->n)) != cudaSuccess) return fail(e);
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaFree(dist);
        if (e0) cudaEventDestroy(e0);
        return fail(e);
    }
    int rc = SSSP_OK;
    uint32_t timed = 0;
    Candidate best{SSSP_RHO, 0, SSSP_SHAPE_WIDE, 0, 0, 0, 0, 0, 0, 0, 0};
    do {
        // rule / parameter candidates: rho = n/4 ... n/1024 (>= 64) and Delta =
        // mean weight x {1/8 ... 8}, each a factor of 2 apart
        std::vector<Candidate> cand;
        for (uint32_t j = 2; j <= 10 && (rules & (1u << SSSP_RHO)); ++j) {
            uint64_t rho = (uint64_t)g->n >> j;
            if (rho < 64) rho = 64;
            bool dup = false;
            for (const Candidate& c : cand) dup = dup || (c.algo == SSSP_RHO && c.param == rho);
            if (!dup) cand.push_back({SSSP_RHO, rho, SSSP_SHAPE_WIDE, 0, 0, 0, 0, 0, 0, 0, 0});
        }
        for (double f : {0.125, 0.25, 0.5, 1.0, 2.0, 4.0, 8.0}) {
            if (!(rules & (1u << SSSP_DELTA_STAR))) break;
            const double d = g->mean_w * f;
            cand.push_back({SSSP_DELTA_STAR, d > 1.0 ? (uint64_t)d : 1ull, SSSP_SHAPE_WIDE, 0, 0, 0, 0, 0, 0, 0, 0});
        }
        // one warm-up solve (first launch of the kernel, lazy allocations)
        double ignore;
        if ((rc = time_config(g, cand[0], sources, 1, dist, st, e0, e1, &ignore)) != SSSP_OK) break;
        // (1)
        for (Candidate& c : cand) {
            if ((rc = time_config(g, c, sources, 1, dist, st, e0, e1, &c.ms)) != SSSP_OK) break;
            ++timed;
        }
        if (rc != SSSP_OK) break;
        std::vector<Candidate> sorted = cand;
        for (size_t i = 0; i < sorted.size(); ++i)
            for (size_t j = i + 1; j < sorted.size(); ++j)
                if (sorted[j].ms < sorted[i].ms) std::swap(sorted[i], sorted[j]);
        // (2) (and the later stages) on up to three sources: one or two sources
        //     let the source's own cost decide between close candidates
        const uint32_t ns2 = k < 3 ? k : 3;
        best.ms = INFINITY;
        for (size_t i = 0; i < 2 && i < sorted.size(); ++i)
            for (uint32_t shape : {SSSP_SHAPE_WIDE, SSSP_SHAPE_NARROW}) {
                Candidate c = sorted[i];
                c.shape = shape;
                if ((rc = time_config(g, c, sources, ns2, dist, st, e0, e1, &c.ms)) != SSSP_OK) break;
                ++timed;
                if (c.ms < best.ms) best = c;
            }
        if (rc != SSSP_OK) break;
        // (3) local relaxation changes which rule and parameter win (it makes
        //     multi-hop steps), so it is tried on the two best of (1) of each
        //     rule, in the shape that won (2)
        if (g->n && (double)g->m / (double)g->n < 20.0) {
            // (the ranking of (1) -- wide, unfused, no local relaxation -- is a
            // rough guide here, so the three best of each rule are taken)
            std::vector<Candidate> base;
            for (sssp_algo a : {SSSP_RHO, SSSP_DELTA_STAR}) {
                int taken = 0;
                for (const Candidate& c : sorted)
                    if (c.algo == a && taken < 3) { base.push_back(c); ++taken; }
            }
            // ... and, since fused super-sparse steps change the ranking as
            // much, the same in the narrow shape with fused steps (also
            // without local relaxation)
            const uint32_t win_shape = best.shape;
            for (size_t i = 0; i < base.size() && rc == SSSP_OK; ++i)
                for (uint32_t fused : {0u, 1u})
                    for (uint32_t local : {0u, 64u, 256u, 1024u}) {
                        if (local == 0 && !fused) continue;  // timed in (1)/(2)
                        Candidate c = base[i];
                        c.shape = fused ? SSSP_SHAPE_NARROW : win_shape;
                        c.fused = fused;
                        c.local = local;
                        if ((rc = time_config(g, c, sources, ns2, dist, st, e0, e1, &c.ms)) != SSSP_OK) break;
                        ++timed;
                        if (c.ms < best.ms) best = c;
                    }
            if (rc != SSSP_OK) break;
        }
        // (4) rho-Stepping: how many dense steps use rho/10 (Sec. 6 uses two)
        if (best.algo == SSSP_RHO) {
            const Candidate base = best;
            for (uint32_t red : {4u, 6u, 8u, (uint32_t)SSSP_RHO_REDUCED_NONE}) {
                Candidate c = base;
                c.rho_reduced = red;
                if ((rc = time_config(g, c, sources, ns2, dist, st, e0, e1, &c.ms)) != SSSP_OK) break;
                ++timed;
                if (c.ms < best.ms) best = c;
            }
            if (rc != SSSP_OK) break;
            // ... and warm-up steps at a small rho (the first, sparse waves in
            // small groups); each count of reduced dense steps again after it
            const Candidate base2 = best;
            for (uint32_t ws : {4u, 6u, 8u}) {
                for (uint32_t red : {base2.rho_reduced, 2u, 4u, 6u}) {
                    Candidate c = base2;
                    c.warm_steps = ws;
                    c.warm_rho = 256;
                    c.rho_reduced = red == 2u ? 0u : red;
                    if ((rc = time_config(g, c, sources, ns2, dist, st, e0, e1, &c.ms)) != SSSP_OK) break;
                    ++timed;
                    if (c.ms < best.ms) best = c;
                }
                if (rc != SSSP_OK) break;
            }
            if (rc != SSSP_OK) break;
        }
        // (5) degree-bin cut-offs: the small-degree bound, then the chunk length
        {
            Candidate base = best;
            for (uint32_t sd : {16u, 64u}) {
                Candidate c = base;
                c.small_deg = sd;
                if ((rc = time_config(g, c, sources, ns2, dist, st, e0, e1, &c.ms)) != SSSP_OK) break;
                ++timed;
                if (c.ms < best.ms) best = c;
            }
            if (rc != SSSP_OK) break;
            base = best;
            for (uint32_t ch : {128u, 512u}) {
                Candidate c = base;
                c.chunk = ch;
                if ((rc = time_config(g, c, sources, ns2, dist, st, e0, e1, &c.ms)) != SSSP_OK) break;
                ++timed;
                if (c.ms < best.ms) best = c;
            }
            if (rc != SSSP_OK) break;
        }
        // (6)
        if ((rc = time_config(g, best, sources, k, dist, st, e0, e1, &best.ms)) != SSSP_OK) break;
    } while (false);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dist);
    if (rc != SSSP_OK) return rc;
    sssp_tuning t;
    memset(&t, 0, sizeof t);
    t.algo = best.algo;
    t.shape = best.shape;
    t.param = best.param;
    t.flags = ((g->flags & SSSP_GRAPH_SYMMETRIC) ? SSSP_SOLVE_BIDIRECTIONAL : 0u) | (best.fused ? SSSP_SOLVE_FUSED : 0u);
    t.local_budget = best.local;
    t.ms = best.ms;
    t.candidates = timed;
    t.rho_reduced = best.rho_reduced;
    t.rho_warmup_steps = best.warm_steps;
    t.rho_warmup = best.warm_rho;
    t.small_deg = best.small_deg;
    t.chunk = best.chunk;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        g->tuning = t;
        g->tuned = true;
    }
    {
        std::lock_guard<std::mutex> lk(g_class_mu);
        g_class_table[sssp_class_key(g)] = t;
    }
    if (out) *out = t;
    return SSSP_OK;
}

// Batched launches have their own best configuration (the device is shared by
// k instances, so a rule or parameter that is fastest alone is not always
// fastest in a batch).  Candidates as in sssp_autotune's first stage, each
// timed as one sssp_solve_sources launch over up to 8 of the sources (with the
// local budget the batch would use); the two best of each rule re-timed on all
// k sources (separate instances, SSSP_BATCH_SEPARATE) and, for k <= 64, with
// one shared edge scan per step (SSSP_BATCH_SHARED); then local budgets 0, 64
// and 256 for every separate-instance finalist on graphs where batched
// launches use local relaxation, and for a rho-Stepping winner 4, 6, 8 or no dense steps
// with rho/10 (the paper's 2 is the starting point).  The result is kept as the graph's batch tuning,
// which the batched and serving calls prefer.
int sssp_autotune_batch(sssp_graph* g, const uint32_t* sources, uint32_t k, uint32_t rules, sssp_tuning* out,
                        void* stream)
{
    if (!g || !sources || k == 0 || k > sssp::kMaxBatch) return SSSP_ERR_INVALID_ARG;
    if (rules == 0 || (rules & ~((1u << SSSP_RHO) | (1u << SSSP_DELTA_STAR)))) return SSSP_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < k; ++i)
        if (sources[i] >= g->n) return SSSP_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(g->device);
    if (e != cudaSuccess) return fail(e);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint64_t* dist = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&dist), sizeof(uint64_t) * (size_t)g->n * k)) != cudaSuccess)
        return fail(e);
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaFree(dist);
        if (e0) cudaEventDestroy(e0);
        return fail(e);
    }
    const bool sym = (g->flags & SSSP_GRAPH_SYMMETRIC) != 0;
    sssp_tuning single;
    const uint32_t local0 = sssp_lookup_tuning(g, &single) ? single.local_budget : 0u;
    // candidates are compared on up to kSweep of the sources; the winner is
    // timed on all k
    constexpr uint32_t kSweep = 8;
    uint32_t kk = k < kSweep ? k : kSweep;
    auto time_batch = [&](const sssp_tuning& t, double* ms) -> int {
        {
            std::lock_guard<std::mutex> lk(g->mu);
            g->batch_tuning = t;
            g->batch_tuned = true;
        }
        cudaError_t ee = cudaEventRecord(e0, st);
        if (ee != cudaSuccess) return fail(ee);
        int r = sssp_solve_sources(g, sources, kk, t.algo, nullptr, dist, stream);
        if (r != SSSP_OK) return r;
        if ((ee = cudaEventRecord(e1, st)) != cudaSuccess) return fail(ee);
        if ((ee = cudaEventSynchronize(e1)) != cudaSuccess) return fail(ee);
        sssp_stats s0;
        r = sssp_batch_last_stats(&s0, 1, stream);
        if (r != SSSP_OK) return r;
        float tm = 0;
        if ((ee = cudaEventElapsedTime(&tm, e0, e1)) != cudaSuccess) return fail(ee);
        *ms = tm;
        return SSSP_OK;
    };
    std::vector<sssp_tuning> cand;
    auto add = [&](sssp_algo a, uint64_t prm) {
        sssp_tuning t;
        memset(&t, 0, sizeof t);
        t.algo = a;
        t.param = prm;
        t.flags = sym ? SSSP_SOLVE_BIDIRECTIONAL : 0u;
        t.local_budget = local0;
        t.batch_mode = SSSP_BATCH_SEPARATE;
        for (const sssp_tuning& c : cand) if (c.algo == a && c.param == prm) return;
        cand.push_back(t);
    };
    if (rules & (1u << SSSP_RHO))
        for (uint32_t j = 2; j <= 10; j += 2) add(SSSP_RHO, ((uint64_t)g->n >> j) < 64 ? 64 : ((uint64_t)g->n >> j));
    if (rules & (1u << SSSP_DELTA_STAR))
        for (double f : {0.125, 0.5, 2.0, 8.0}) {
            const double d = g->mean_w * f;
            add(SSSP_DELTA_STAR, d > 1.0 ? (uint64_t)d : 1ull);
        }
    int rc = SSSP_OK;
    uint32_t timed = 0;
    sssp_tuning best = cand[0];
    double best_ms = INFINITY, ms = 0;
    rc = time_batch(cand[0], &ms);  // warm-up (first launch, workspace growth)
    std::vector<double> sweep(cand.size(), INFINITY);
    for (size_t i = 0; i < cand.size() && rc == SSSP_OK; ++i) {
        if ((rc = time_batch(cand[i], &sweep[i])) != SSSP_OK) break;
        ++timed;
    }
    // the two best of each rule on the small sweep, re-timed on all k sources
    // (a few instances are latency-bound and can rank configurations
    // differently from a full batch)
    kk = k;
    std::vector<sssp_tuning> finalists;
    for (sssp_algo a : {SSSP_RHO, SSSP_DELTA_STAR}) {
        for (int r = 0; r < 2 && rc == SSSP_OK; ++r) {
            size_t bi = cand.size();
            for (size_t i = 0; i < cand.size(); ++i)
                if (cand[i].algo == a && sweep[i] < INFINITY && (bi == cand.size() || sweep[i] < sweep[bi])) bi = i;
            if (bi == cand.size()) break;
            sweep[bi] = INFINITY;  // taken
            finalists.push_back(cand[bi]);
            if ((rc = time_batch(cand[bi], &ms)) != SSSP_OK) break;
            ++timed;
            if (ms < best_ms) { best_ms = ms; best = cand[bi]; }
        }
    }
    // the same finalists with one shared edge scan per step (k <= 64): no
    // local or bidirectional relaxation there; rho-Stepping also with six
    // dense steps at rho/10
    if (rc == SSSP_OK && sssp::ms_batch_supported(SSSP_RHO, k)) {
        for (const sssp_tuning& f : finalists) {
            for (uint32_t variant = 0; variant < 3; ++variant) {
                // the paper's 2 reduced dense steps, 6, and 8 warm-up steps at
                // rho 256 followed by 4
                if (variant && f.algo != SSSP_RHO) continue;
                sssp_tuning t = f;
                t.batch_mode = SSSP_BATCH_SHARED;
                t.local_budget = 0;
                t.rho_reduced = variant == 0 ? 0u : variant == 1 ? 6u : 4u;
                t.rho_warmup_steps = variant == 2 ? 8u : 0u;
                t.rho_warmup = variant == 2 ? 256u : 0u;
                if ((rc = time_batch(t, &ms)) != SSSP_OK) break;
                ++timed;
                if (ms < best_ms) { best_ms = ms; best = t; }
            }
            if (rc != SSSP_OK) break;
        }
    }
    // local budgets for every finalist of the separate-instance kernel (the
    // budget changes which rule and parameter win, as in single solves)
    if (rc == SSSP_OK && g->n >= (1u << 20) && (double)g->m / (double)g->n < 20.0) {
        for (const sssp_tuning& f : finalists) {
            for (uint32_t local : {0u, 64u, 256u}) {
                if (local == f.local_budget) continue;
                sssp_tuning t = f;
                t.local_budget = local;
                if ((rc = time_batch(t, &ms)) != SSSP_OK) break;
                ++timed;
                if (ms < best_ms) { best_ms = ms; best = t; }
            }
            if (rc != SSSP_OK) break;
        }
    }
    if (rc == SSSP_OK && best.algo == SSSP_RHO) {  // dense steps with rho/10 (Sec. 6 uses two)
        const sssp_tuning base = best;
        for (uint32_t red : {4u, 6u, 8u, (uint32_t)SSSP_RHO_REDUCED_NONE}) {
            if (red == base.rho_reduced) continue;
            sssp_tuning t = base;
            t.rho_reduced = red;
            if ((rc = time_batch(t, &ms)) != SSSP_OK) break;
            ++timed;
            if (ms < best_ms) { best_ms = ms; best = t; }
        }
    }
    if (rc == SSSP_OK) rc = time_batch(best, &best_ms);
    // throughput of the winner with fewer concurrent sources: on a graph where
    // one solve already keeps the device busy, fewer queries at once are faster
    uint32_t slots = k;
    double best_rate = best_ms > 0 ? (double)k / best_ms : 0.0;
    for (uint32_t kc : {16u, 4u, 1u}) {
        if (rc != SSSP_OK || kc >= k) continue;
        kk = kc;
        double t2 = 0;
        if ((rc = time_batch(best, &t2)) != SSSP_OK) break;
        // a smaller batch of kc queries: compare queries per ms
        if (t2 > 0 && (double)kc / t2 > best_rate) { best_rate = (double)kc / t2; slots = kc; }
    }
    kk = k;
    best.slots = slots;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(dist);
    best.ms = best_ms;
    best.candidates = timed;
    best.slots = slots;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (rc == SSSP_OK) g->batch_tuning = best;
        g->batch_tuned = rc == SSSP_OK;
    }
    if (rc != SSSP_OK) return rc;
    if (out) *out = best;
    return SSSP_OK;
}

int sssp_graph_get_tuning(const sssp_graph* g, sssp_tuning* out)
{
    if (!g || !out) return SSSP_ERR_INVALID_ARG;
    return sssp_lookup_tuning(g, out) ? SSSP_OK : SSSP_ERR_INVALID_ARG;
}

int sssp_graph_set_tuning(sssp_graph* g, const sssp_tuning* t)
{
    if (!g || !t) return SSSP_ERR_INVALID_ARG;
    if (t->algo != SSSP_RHO && t->algo != SSSP_DELTA_STAR && t->algo != SSSP_BELLMAN_FORD) return SSSP_ERR_INVALID_ARG;
    if (algo_needs_param(t->algo) && t->param == 0) return SSSP_ERR_INVALID_ARG;
    if (t->shape > SSSP_SHAPE_NARROW || (t->flags & ~(SSSP_SOLVE_BIDIRECTIONAL | SSSP_SOLVE_FUSED)))
        return SSSP_ERR_INVALID_ARG;
    if ((t->flags & SSSP_SOLVE_BIDIRECTIONAL) && !(g->flags & SSSP_GRAPH_SYMMETRIC)) return SSSP_ERR_INVALID_ARG;
    if (t->local_budget != 0 && t->algo == SSSP_BELLMAN_FORD) return SSSP_ERR_INVALID_ARG;
    if (t->small_deg != 0 && (t->small_deg < sssp::kSmallDegMin || t->small_deg > sssp::kSmallDegMax))
        return SSSP_ERR_INVALID_ARG;
    if (t->chunk != 0 && t->chunk != 128 && t->chunk != 256 && t->chunk != 512 && t->chunk != 1024)
        return SSSP_ERR_INVALID_ARG;
    if (t->batch_mode > SSSP_BATCH_SEPARATE) return SSSP_ERR_INVALID_ARG;
    if ((t->rho_warmup_steps == 0) != (t->rho_warmup == 0)) return SSSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    g->tuning = *t;
    g->tuned = true;
    return SSSP_OK;
}

int sssp_solve_tuned(const sssp_graph* g, uint32_t source, uint64_t* dist_out, void* stream)
{
    if (!g) return SSSP_ERR_INVALID_ARG;
    sssp_tuning t;
    if (!sssp_lookup_tuning(g, &t)) {
        memset(&t, 0, sizeof t);
        t.algo = SSSP_RHO;
        t.param = sssp_default_param(g->n, g->m, SSSP_RHO, g->mean_w);
        t.flags = (g->flags & SSSP_GRAPH_SYMMETRIC) ? SSSP_SOLVE_BIDIRECTIONAL : 0u;
        t.shape = SSSP_SHAPE_WIDE;
    }
    sssp_options o;
    memset(&o, 0, sizeof o);
    o.flags = t.flags;
    o.shape = t.shape;
    o.local_budget = t.local_budget;
    o.rho_reduced = t.rho_reduced;
    o.rho_warmup_steps = t.rho_warmup_steps;
    o.rho_warmup = t.rho_warmup;
    o.small_deg = t.small_deg;
    o.chunk = t.chunk;
    return sssp_solve_ex(g, source, t.algo, t.param, dist_out, &o, stream);
}

}  // extern "C"
