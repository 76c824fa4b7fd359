// sssp_internal.h -- types shared by the host ABI (sssp_api.cu) and the
// device code (sssp_kernels.cu) of libsssp.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/sssp.h"

namespace sssp {

constexpr int kBlock = 512;                 // threads per block of the persistent kernel
constexpr int kWarps = kBlock / 32;
constexpr uint32_t kSmallDeg = 32;          // degree <= this: warp-flattened relaxation groups
constexpr uint32_t kChunk = 256;            // edges per relaxation chunk item (even)
constexpr int kExtractItems = 4;            // queue entries per thread per extract tile
constexpr int kStage = 512;                 // per-warp staging slots for re-queued ids
constexpr uint32_t kMaxSamples = 4096;      // cap on the rho sampler's sample count
constexpr uint64_t kInf = ~0ull;

// Device control block of one solve.  Zeroed by the host before each launch.
// Per-step counters live in a ring of three slots indexed by step % 3: slot
// k%3 holds |Q_k| (qsize, qmin: appended during step k-1) and the Extract
// output of step k (fsmall, fchunk, fcount, fedges, updates).
struct Ctrl {
    unsigned long long bar;       // grid-barrier arrival counter (monotone)
    int status;                   // sssp_status of the solve (0 = OK)
    unsigned int pad0;
    unsigned int qsize[3];
    unsigned int fsmall[3];
    unsigned int fchunk[3];
    unsigned int fcount[3];
    unsigned long long qmin[3];
    unsigned long long fedges[3];
    unsigned long long updates[3];
    // totals, written by block 0 when the solve ends
    unsigned long long steps, queued, extracted, edges, updates_total;
};

struct SolveParams {
    const uint64_t* off;          // CSR offsets [n+1]
    const uint2* edges;           // packed (target, weight) [m rounded up to even]
    uint32_t n;
    uint64_t m;
    uint64_t* dist;               // delta / output [n]
    uint32_t* inq;                // LaB-PQ membership bitmap [ceil(n/32)]
    uint32_t* qa;                 // queue lists (alternating) [n]
    uint32_t* qb;
    uint32_t* fsmall;             // extracted ids with 1 <= degree <= kSmallDeg [n]
    uint2* items;                 // (id, chunk) relaxation items of larger vertices
    uint64_t item_cap;
    Ctrl* ctrl;
    uint32_t source;
    int algo;
    uint64_t param;
    uint64_t seed;
    uint64_t timeout_ns;          // bound on each device-wide wait
    uint64_t solve_timeout_ns;    // bound on the whole solve
    uint64_t max_steps;
    uint32_t* ext_count;          // optional [n]
    sssp_step_trace* trace;       // optional [trace_cap]
    uint32_t trace_cap;
    uint32_t exit_block;          // testing: 1 + block that leaves before the first wait
    uint32_t sample_cap;          // power of two >= the largest sample count, or 0
    sssp_stats* stats_out;        // optional device copy of the totals
};

// Upper bound on items produced by one Extract: each extracted vertex of
// degree > kSmallDeg yields at most deg/kChunk + 2 chunk items.
inline uint64_t item_capacity(uint32_t n, uint64_t m) { return m / kChunk + 2ull * n + 64; }

// Launch helpers implemented in sssp_kernels.cu.
cudaError_t launch_pack_edges(const uint32_t* tgt, const uint32_t* w, uint2* edges, uint64_t m,
                              uint64_t m_pad, cudaStream_t st);
const void* solve_kernel_ptr();
cudaError_t launch_rho_threshold(const uint32_t* queue, uint32_t q, const uint64_t* dist,
                                 uint32_t n, uint64_t rho, uint64_t seed, uint64_t step,
                                 uint32_t dense_before, uint64_t* theta_out, uint32_t* err_out,
                                 cudaStream_t st);
uint32_t rho_sample_bound(uint32_t n, uint64_t rho);   // power-of-two smem keys needed

}  // namespace sssp
