// sssp_api.cu -- host side of the C ABI declared in include/sssp.h.
//
// Owns the device copy of the graph and the solver scratch (queue bitmap,
// queue lists, extraction lists, control block), validates arguments, and
// launches the persistent cooperative solve kernel (sssp_kernels.cu).

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <new>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "sssp_internal.h"

using namespace sssp;

// struct sssp_graph is defined in sssp_internal.h


namespace {

int cuda_fail(cudaError_t e)
{
    if (e == cudaErrorMemoryAllocation) return SSSP_ERR_OUT_OF_MEMORY;
    return SSSP_ERR_CUDA;
}

template <typename T>
cudaError_t dalloc(T** p, uint64_t count)
{
    return cudaMalloc(reinterpret_cast<void**>(p), (size_t)(count ? count : 1) * sizeof(T));
}

void free_graph(sssp_graph* g)
{
    if (!g) return;
    cudaFree(g->d_off);
    cudaFree(g->d_edges);
    cudaFree(g->d_inq);
    cudaFree(g->d_qa);
    cudaFree(g->d_qb);
    cudaFree(g->d_fsmall);
    cudaFree(g->d_items);
    cudaFree(g->d_ctrl);
    cudaFree(g->d_dist_internal);
    cudaFree(g->d_lrel);
    cudaFree(g->d_fre);
    cudaFree(g->d_off2);
    cudaFree(g->d_edges2);
    cudaFree(g->d_perm);
    cudaFree(g->d_iperm);
    cudaFree(g->d_dist2);
    if (g->h_ctrl) cudaFreeHost(g->h_ctrl);
    delete g;
}

// The relabelled copy of SSSP_GRAPH_REORDER: new id = rank by decreasing
// out-degree (ties by id), each adjacency sorted by (new target, weight).
// Adjacencies are rebuilt in parallel over ranges of new ids.
void relabel_graph(uint32_t n, const uint64_t* off, const uint32_t* tgt, const uint32_t* w, std::vector<uint32_t>& perm,
                   std::vector<uint32_t>& iperm, std::vector<uint64_t>& off2, std::vector<uint32_t>& tgt2,
                   std::vector<uint32_t>& w2)
{
    const uint64_t m = off[n];
    iperm.resize(n);
    for (uint32_t i = 0; i < n; ++i) iperm[i] = i;
    std::sort(iperm.begin(), iperm.end(), [off](uint32_t a, uint32_t b) {
        const uint64_t da = off[a + 1] - off[a], db = off[b + 1] - off[b];
        return da != db ? da > db : a < b;
    });
    perm.resize(n);
    for (uint32_t i = 0; i < n; ++i) perm[iperm[i]] = i;
    off2.resize((size_t)n + 1);
    off2[0] = 0;
    for (uint32_t i = 0; i < n; ++i) off2[i + 1] = off2[i] + (off[iperm[i] + 1] - off[iperm[i]]);
    tgt2.resize(m);
    w2.resize(m);
    unsigned nt = std::thread::hardware_concurrency();
    nt = nt < 1 ? 1 : (nt > 64 ? 64 : nt);
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) {
        th.emplace_back([&, t]() {
            std::vector<uint64_t> key;
            const uint32_t lo = (uint32_t)((uint64_t)n * t / nt), hi = (uint32_t)((uint64_t)n * (t + 1) / nt);
            for (uint32_t u = lo; u < hi; ++u) {
                const uint32_t o = iperm[u];
                const uint64_t b = off[o], d = off[o + 1] - b;
                key.resize(d);
                for (uint64_t j = 0; j < d; ++j) key[j] = ((uint64_t)perm[tgt[b + j]] << 32) | w[b + j];
                std::sort(key.begin(), key.end());
                for (uint64_t j = 0; j < d; ++j) {
                    tgt2[off2[u] + j] = (uint32_t)(key[j] >> 32);
                    w2[off2[u] + j] = (uint32_t)key[j];
                }
            }
        });
    }
    for (std::thread& x : th) x.join();
}

// The two builds of the solve kernel (sssp_kernels.cu compiled twice): the
// wide shape (1024 threads, 64 registers each: the most loads in flight, for
// edge-heavy steps) and the narrow one (512 threads, up to 128 registers:
// cheaper block-wide phases, for graphs whose solves take many small steps).
struct SolveShape {
    const void* (*kernel)();
    int (*threads)();
    unsigned int (*smem)();
};
const SolveShape kShapes[2] = {
    {sssp::solve_kernel_ptr, sssp::solve_kernel_threads, sssp::solve_kernel_smem},
    {sssp_narrow::solve_kernel_ptr, sssp_narrow::solve_kernel_threads, sssp_narrow::solve_kernel_smem},
};

// blocks per SM of a shape of the solve kernel (its dynamic shared memory is fixed)
int solve_blocks_per_sm(int shape, int* out)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    const SolveShape& sh = kShapes[shape];
    const void* fn = sh.kernel();
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.smem());
    if (e != cudaSuccess) return cuda_fail(e);
    int bps = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, sh.threads(), sh.smem());
    if (e != cudaSuccess) return cuda_fail(e);
    *out = bps;
    return SSSP_OK;
}

}  // namespace

extern "C" {

const char* sssp_status_string(int status)
{
    switch (status) {
        case SSSP_OK: return "ok";
        case SSSP_ERR_INVALID_ARG: return "invalid argument";
        case SSSP_ERR_OUT_OF_MEMORY: return "out of memory";
        case SSSP_ERR_CUDA: return "CUDA runtime error";
        case SSSP_ERR_TIMEOUT: return "device-wide wait timed out";
        case SSSP_ERR_INTERNAL: return "internal capacity or step guard";
        default: return "unknown status";
    }
}

int sssp_graph_create(uint32_t n, uint64_t m, const uint64_t* offsets, const uint32_t* targets,
                      const uint32_t* weights, sssp_graph** out)
{
    return sssp_graph_create_ex(n, m, offsets, targets, weights, 0, out);
}

namespace {

// Every edge (u,v,w) has a reverse (v,u,w): each adjacency is sorted by
// (target, weight) in a copy and searched.
bool verify_symmetric(uint32_t n, const uint64_t* off, const uint32_t* tgt, const uint32_t* w)
{
    const uint64_t m = off[n];
    std::vector<uint64_t> key(m);
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) key[e] = ((uint64_t)tgt[e] << 32) | w[e];
        std::sort(key.begin() + (ptrdiff_t)off[u], key.begin() + (ptrdiff_t)off[u + 1]);
    }
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            const uint32_t v = tgt[e];
            const uint64_t want = ((uint64_t)u << 32) | w[e];
            if (!std::binary_search(key.begin() + (ptrdiff_t)off[v], key.begin() + (ptrdiff_t)off[v + 1], want))
                return false;
        }
    return true;
}

}  // namespace

int sssp_graph_create_ex(uint32_t n, uint64_t m, const uint64_t* offsets, const uint32_t* targets,
                         const uint32_t* weights, uint32_t flags, sssp_graph** out)
{
    if (!out) return SSSP_ERR_INVALID_ARG;
    *out = nullptr;
    if (n == 0 || !offsets || (m > 0 && (!targets || !weights))) return SSSP_ERR_INVALID_ARG;
    if (m >= (1ull << 40)) return SSSP_ERR_INVALID_ARG;
    if (offsets[0] != 0 || offsets[n] != m) return SSSP_ERR_INVALID_ARG;
    for (uint32_t u = 0; u < n; ++u)
        if (offsets[u + 1] < offsets[u]) return SSSP_ERR_INVALID_ARG;
    for (uint64_t e = 0; e < m; ++e)
        if (targets[e] >= n) return SSSP_ERR_INVALID_ARG;
    if (flags & ~(SSSP_GRAPH_SYMMETRIC | SSSP_GRAPH_VERIFY | SSSP_GRAPH_REORDER)) return SSSP_ERR_INVALID_ARG;
    if ((flags & SSSP_GRAPH_VERIFY) && (flags & SSSP_GRAPH_SYMMETRIC) &&
        !verify_symmetric(n, offsets, targets, weights))
        return SSSP_ERR_INVALID_ARG;

    // exact capacities of the relaxation records one Extract can produce:
    // each vertex is queued at most once, so at most every vertex at once.
    // Two sets: at the default degree-bin cut-offs (batched and serving
    // launches) and the largest over every cut-off a single solve may take
    // (small_deg in [kSmallDegMin, kSmallDegMax], chunks of >= 2^kChunkLog2Min
    // edges) -- the single solve's record arrays are sized for the latter.
    uint64_t small_cap = 0, item_cap = 0, small_any = 0, item_any = 0, ms_rec = 0;
    unsigned __int128 wsum = 0;
    for (uint64_t e = 0; e < m; ++e) wsum += weights[e];
    uint64_t max_deg = 0;
    for (uint32_t u = 0; u < n; ++u) {
        const uint64_t deg = offsets[u + 1] - offsets[u];
        max_deg = deg > max_deg ? deg : max_deg;
        if (deg == 0) continue;
        if (deg <= kSmallDeg) ++small_cap;
        else item_cap += chunk_count(offsets[u], offsets[u + 1]);
        if (deg <= kSmallDegMax) ++small_any;
        ms_rec += (deg + kMsRecEdges - 1) / kMsRecEdges;
        if (deg > kSmallDegMin) item_any += chunk_count(offsets[u], offsets[u + 1], kChunkLog2Min);
    }

    // relabelled copy for single solves (its chunk records are counted too:
    // the record arrays serve both layouts)
    std::vector<uint32_t> perm, iperm, tgt2, w2;
    std::vector<uint64_t> off2;
    if (flags & SSSP_GRAPH_REORDER) {
        relabel_graph(n, offsets, targets, weights, perm, iperm, off2, tgt2, w2);
        uint64_t item_cap2 = 0, item_any2 = 0;
        for (uint32_t u = 0; u < n; ++u) {
            const uint64_t deg = off2[u + 1] - off2[u];
            if (deg > kSmallDeg) item_cap2 += chunk_count(off2[u], off2[u + 1]);
            if (deg > kSmallDegMin) item_any2 += chunk_count(off2[u], off2[u + 1], kChunkLog2Min);
        }
        item_cap = item_cap2 > item_cap ? item_cap2 : item_cap;
        item_any = item_any2 > item_any ? item_any2 : item_any;
    }

    sssp_graph* g = new (std::nothrow) sssp_graph();
    if (!g) return SSSP_ERR_OUT_OF_MEMORY;
    g->n = n;
    g->m = m;
    g->flags = flags & SSSP_GRAPH_SYMMETRIC;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) { free_graph(g); return cuda_fail(e); }

    const uint64_t m_pad = (m + 1) & ~1ull;  // even, so 16-byte pair loads stay in bounds
    const uint64_t m_alloc = m_pad < 2 ? 2 : m_pad;
    uint32_t* d_tgt = nullptr;
    uint32_t* d_w = nullptr;
    g->fsmall_cap = small_cap + 1;
    g->mean_w = m ? (double)wsum / (double)m : 1.0;
    g->max_deg = max_deg;
    g->item_cap = item_cap + 1;
    g->fsmall_cap_any = small_any + 1;
    g->item_cap_any = item_any + 1;
    g->ms_rec_cap = ms_rec + 1;
    if ((e = dalloc(&g->d_off, (uint64_t)n + 1)) != cudaSuccess ||
        (e = dalloc(&g->d_edges, m_alloc)) != cudaSuccess ||
        (e = dalloc(&g->d_inq, ((uint64_t)n + 31) / 32)) != cudaSuccess ||
        (e = dalloc(&g->d_qa, n)) != cudaSuccess || (e = dalloc(&g->d_qb, n)) != cudaSuccess ||
        (e = dalloc(&g->d_fsmall, g->fsmall_cap_any)) != cudaSuccess ||
        (e = dalloc(&g->d_items, g->item_cap_any)) != cudaSuccess ||
        (e = dalloc(&g->d_ctrl, 1)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void**>(&g->h_ctrl), sizeof(Ctrl))) != cudaSuccess ||
        (e = dalloc(&d_tgt, m)) != cudaSuccess || (e = dalloc(&d_w, m)) != cudaSuccess) {
        cudaFree(d_tgt);
        cudaFree(d_w);
        free_graph(g);
        return cuda_fail(e);
    }
    memset(g->h_ctrl, 0, sizeof(Ctrl));
    e = cudaMemcpy(g->d_off, offsets, sizeof(uint64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m) e = cudaMemcpy(d_tgt, targets, sizeof(uint32_t) * m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && m) e = cudaMemcpy(d_w, weights, sizeof(uint32_t) * m, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_pack_edges(d_tgt, d_w, g->d_edges, m, m_alloc, 0);
    if (e == cudaSuccess) e = cudaMemset(g->d_ctrl, 0, sizeof(Ctrl));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && (flags & SSSP_GRAPH_REORDER)) {
        g->reordered = true;
        g->h_perm = std::move(perm);
        if ((e = dalloc(&g->d_off2, (uint64_t)n + 1)) == cudaSuccess && (e = dalloc(&g->d_edges2, m_alloc)) == cudaSuccess &&
            (e = dalloc(&g->d_perm, n)) == cudaSuccess && (e = dalloc(&g->d_iperm, n)) == cudaSuccess &&
            (e = dalloc(&g->d_dist2, n)) == cudaSuccess)
            e = cudaMemcpy(g->d_off2, off2.data(), sizeof(uint64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_perm, g->h_perm.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g->d_iperm, iperm.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && m) e = cudaMemcpy(d_tgt, tgt2.data(), sizeof(uint32_t) * m, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && m) e = cudaMemcpy(d_w, w2.data(), sizeof(uint32_t) * m, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = launch_pack_edges(d_tgt, d_w, g->d_edges2, m, m_alloc, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(d_tgt);
    cudaFree(d_w);
    if (e != cudaSuccess) { free_graph(g); return cuda_fail(e); }
    *out = g;
    return SSSP_OK;
}

int sssp_graph_destroy(sssp_graph* g)
{
    if (!g) return SSSP_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    free_graph(g);
    return SSSP_OK;
}

int sssp_graph_info(const sssp_graph* g, uint32_t* n, uint64_t* m)
{
    if (!g) return SSSP_ERR_INVALID_ARG;
    if (n) *n = g->n;
    if (m) *m = g->m;
    return SSSP_OK;
}

int sssp_solve_ex(const sssp_graph* gc, uint32_t source, sssp_algo algo, uint64_t param, uint64_t* dist_out,
                  const sssp_options* opt, void* stream)
{
    sssp_graph* g = const_cast<sssp_graph*>(gc);
    if (!g || !dist_out) return SSSP_ERR_INVALID_ARG;
    if (source >= g->n) return SSSP_ERR_INVALID_ARG;
    if (!algo_valid(algo)) return SSSP_ERR_INVALID_ARG;
    if (algo_needs_param(algo) && param == 0) return SSSP_ERR_INVALID_ARG;
    sssp_options o;
    memset(&o, 0, sizeof o);
    if (opt) o = *opt;
    if (o.trace && o.trace_cap == 0) o.trace = nullptr;

    SolveParams p;
    memset(&p, 0, sizeof p);
    p.off = g->d_off;
    p.edges = g->d_edges;
    p.n = g->n;
    p.m = g->m;
    p.dist = dist_out;
    p.inq = g->d_inq;
    p.qa = g->d_qa;
    p.qb = g->d_qb;
    p.fsmall = g->d_fsmall;
    p.fsmall_cap = g->fsmall_cap_any;
    p.items = g->d_items;
    p.item_cap = g->item_cap_any;
    p.ctrl = g->d_ctrl;
    p.source = source;
    p.algo = (int)algo;
    p.param = param;
    p.seed = o.seed ? o.seed : (0x2105061450000000ull ^ (uint64_t)source);
    p.timeout_ns = o.timeout_ns ? o.timeout_ns : 2000000000ull;
    p.solve_timeout_ns = o.solve_timeout_ns ? o.solve_timeout_ns : 60000000000ull;
    p.max_steps = o.max_steps;
    p.ext_count = o.ext_count;
    p.trace = o.trace;
    p.trace_cap = o.trace_cap;
    p.exit_block = o.test_exit_block;
    p.stats_out = o.stats_out;
    if (o.flags & ~(SSSP_SOLVE_BIDIRECTIONAL | SSSP_SOLVE_FUSED)) return SSSP_ERR_INVALID_ARG;
    if ((o.flags & SSSP_SOLVE_BIDIRECTIONAL) && !(g->flags & SSSP_GRAPH_SYMMETRIC)) return SSSP_ERR_INVALID_ARG;
    p.bidir = (o.flags & SSSP_SOLVE_BIDIRECTIONAL) ? 1 : 0;
    if (o.local_budget != 0 && algo != SSSP_RHO && algo != SSSP_DELTA_STAR) return SSSP_ERR_INVALID_ARG;
    p.local_budget = o.local_budget;
    if (o.local_budget != 0) {
        // per-vertex record of local relaxations (allocated by the first solve
        // that uses local relaxation on this graph)
        std::lock_guard<std::mutex> lk(g->mu);
        if (!g->d_lrel) {
            cudaError_t e = dalloc(&g->d_lrel, g->n);
            if (e != cudaSuccess) { g->d_lrel = nullptr; return cuda_fail(e); }
        }
        p.lrel = g->d_lrel;
    }
    p.rho_reduced = o.rho_reduced == 0 ? kRhoReducedDefault
                    : o.rho_reduced == SSSP_RHO_REDUCED_NONE ? 0u : o.rho_reduced;
    if (o.small_deg != 0 && (o.small_deg < kSmallDegMin || o.small_deg > kSmallDegMax)) return SSSP_ERR_INVALID_ARG;
    p.small_deg = o.small_deg ? o.small_deg : kSmallDeg;
    p.chunk_log2 = kChunkLog2;
    if (o.chunk != 0) {
        uint32_t lg = 0;
        while ((1u << lg) < o.chunk && lg < 31) ++lg;
        if ((1u << lg) != o.chunk || lg < kChunkLog2Min || lg > kChunkLog2Max) return SSSP_ERR_INVALID_ARG;
        p.chunk_log2 = lg;
    }
    if (g->reordered) {  // the relabelled copy; distances back in the caller's ids at the end
        p.off = g->d_off2;
        p.edges = g->d_edges2;
        p.dist = g->d_dist2;
        p.dist_out = dist_out;
        p.perm = g->d_perm;
        p.iperm = g->d_iperm;
        p.source = g->h_perm[source];
    }
    if (o.rho_warmup_steps != 0 && o.rho_warmup == 0) return SSSP_ERR_INVALID_ARG;
    if (o.rho_warmup_steps == 0 && o.rho_warmup != 0) return SSSP_ERR_INVALID_ARG;
    p.sample_cap = (algo == SSSP_RHO) ? rho_sample_bound(g->n, param) : 0;
    if (algo == SSSP_RHO && o.rho_warmup_steps != 0) {
        p.warm_steps = o.rho_warmup_steps;
        p.warm_rho = o.rho_warmup;
        // warm-up steps sample at rho_warmup itself (the bound assumes rho/10)
        const uint32_t wcap = rho_sample_bound(g->n, 10ull * o.rho_warmup);
        if (wcap > p.sample_cap) p.sample_cap = wcap;
    }
    if (o.shape > SSSP_SHAPE_NARROW) return SSSP_ERR_INVALID_ARG;
    const int shape = o.shape == SSSP_SHAPE_NARROW ? 1 : 0;
    const size_t dyn_smem = kShapes[shape].smem();
    int bps = 0;
    int rc;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        cudaError_t e = cudaSetDevice(g->device);
        if (e != cudaSuccess) return cuda_fail(e);
        rc = solve_blocks_per_sm(shape, &bps);
    }
    if (rc != SSSP_OK) return rc;
    if (bps < 1) return SSSP_ERR_CUDA;
    uint32_t grid = (uint32_t)(bps * g->num_sms);
    if (o.grid_limit && o.grid_limit < grid) grid = o.grid_limit;
    if (p.exit_block > grid) return SSSP_ERR_INVALID_ARG;
    g->last_grid = grid;
    if ((o.flags & SSSP_SOLVE_FUSED) && shape == 1) {
        // per block two step-parity buffers of one Extract round's entries
        const uint64_t need = (uint64_t)grid * 2ull * (uint64_t)kShapes[shape].threads() * (uint64_t)kExtractPer;
        std::lock_guard<std::mutex> lk(g->mu);
        if (g->fre_cap < need) {
            cudaFree(g->d_fre);
            g->fre_cap = 0;
            cudaError_t e = dalloc(&g->d_fre, need);
            if (e != cudaSuccess) { g->d_fre = nullptr; return cuda_fail(e); }
            g->fre_cap = need;
        }
        p.fre = g->d_fre;
    }

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(g->d_ctrl, 0, sizeof(Ctrl), st);
    if (e != cudaSuccess) return cuda_fail(e);
    void* args[] = {&p};
    e = cudaLaunchCooperativeKernel(kShapes[shape].kernel(), dim3(grid), dim3(kShapes[shape].threads()), args,
                                    dyn_smem, st);
    if (e != cudaSuccess) return cuda_fail(e);
    return SSSP_OK;
}

int sssp_solve(const sssp_graph* g, uint32_t source, sssp_algo algo, uint64_t param, uint64_t* dist_out,
               void* stream)
{
    return sssp_solve_ex(g, source, algo, param, dist_out, nullptr, stream);
}

int sssp_last_stats(const sssp_graph* gc, sssp_stats* out, void* stream)
{
    sssp_graph* g = const_cast<sssp_graph*>(gc);
    if (!g || !out) return SSSP_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(g->h_ctrl, g->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    const Ctrl& c = *g->h_ctrl;
    out->steps = c.steps;
    out->queued = c.queued;
    out->extracted = c.extracted;
    out->edges = c.edges;
    out->updates = c.updates_total;
    out->status = c.status;
    out->grid = g->last_grid;
    return SSSP_OK;
}

int sssp_last_status(const sssp_graph* g, void* stream)
{
    sssp_stats s;
    int rc = sssp_last_stats(g, &s, stream);
    if (rc != SSSP_OK) return rc;
    return s.status;
}

int sssp_solve_host(const sssp_graph* g, uint32_t source, sssp_algo algo, uint64_t param,
                    uint64_t* host_dist_out, void* stream)
{
    return sssp_solve_host_ex(g, source, algo, param, host_dist_out, nullptr, stream);
}

int sssp_solve_host_ex(const sssp_graph* gc, uint32_t source, sssp_algo algo, uint64_t param,
                       uint64_t* host_dist_out, const sssp_options* opt, void* stream)
{
    sssp_graph* g = const_cast<sssp_graph*>(gc);
    if (!g || !host_dist_out) return SSSP_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (!g->d_dist_internal) {
            cudaError_t e = dalloc(&g->d_dist_internal, g->n);
            if (e != cudaSuccess) { g->d_dist_internal = nullptr; return cuda_fail(e); }
        }
    }
    int rc = sssp_solve_ex(g, source, algo, param, g->d_dist_internal, opt, stream);
    if (rc != SSSP_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(host_dist_out, g->d_dist_internal, sizeof(uint64_t) * (size_t)g->n,
                                    cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e);
    return sssp_last_status(g, stream);
}

int sssp_rho_threshold(const uint32_t* queue, uint32_t q, const uint64_t* dist, uint32_t n, uint64_t rho,
                       uint64_t seed, uint64_t step, uint32_t dense_before, uint32_t reduced,
                       uint32_t max_samples, uint64_t* theta_out, void* stream)
{
    if ((q > 0 && !queue) || !dist || !theta_out || n == 0 || rho == 0 || q > n) return SSSP_ERR_INVALID_ARG;
    if (max_samples > kMaxSamples) return SSSP_ERR_INVALID_ARG;
    if (max_samples == 0) max_samples = kMaxSamples;
    static uint32_t* d_err = nullptr;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!d_err) {
            cudaError_t e = dalloc(&d_err, 1);
            if (e != cudaSuccess) { d_err = nullptr; return cuda_fail(e); }
        }
    }
    cudaError_t e = launch_rho_threshold(queue, q, dist, n, rho, seed, step, dense_before, reduced, max_samples,
                                         theta_out, d_err, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SSSP_OK : cuda_fail(e);
}

}  // extern "C"
