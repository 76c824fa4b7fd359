// sssp_internal.h -- types shared by the host ABI (sssp_api.cu) and the
// device code (sssp_kernels.cu) of libsssp.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/sssp.h"

namespace sssp {

#ifndef SSSP_BLOCK
#define SSSP_BLOCK 1024
#endif
#ifndef SSSP_MIN_BLOCKS
#define SSSP_MIN_BLOCKS 1
#endif
constexpr int kBlock = SSSP_BLOCK;                // threads per block of the persistent kernels
constexpr int kMinBlocks = SSSP_MIN_BLOCKS;       // resident blocks per SM the solve kernel is built for
constexpr int kWarps = kBlock / 32;
#ifndef SSSP_SMALL_DEG
#define SSSP_SMALL_DEG 32
#endif
#ifndef SSSP_EXTRACT_ITEMS
#define SSSP_EXTRACT_ITEMS 4
#endif
constexpr uint32_t kSmallDeg = SSSP_SMALL_DEG;  // default cut-off: degree <= this -> warp-flattened groups
constexpr int kSmallRounds = 4;             // 32-edge rounds per batch in the flattened path
constexpr uint32_t kChunk = 256;            // default edges per relaxation chunk record (even)
constexpr uint32_t kChunkLog2 = 8;
// Range of the single solve's runtime degree-bin cut-offs (sssp_options
// small_deg / chunk); the batched kernels use the defaults above.
constexpr uint32_t kSmallDegMin = 8, kSmallDegMax = 128;
constexpr uint32_t kChunkLog2Min = 7, kChunkLog2Max = 10;   // 128 .. 1024 edges
constexpr uint32_t kRhoReducedDefault = 2;  // dense steps with rho/10 (Sec. 6)
constexpr int kExtractItems = SSSP_EXTRACT_ITEMS;  // batched kernels: queue entries per thread per extract tile
constexpr int kStage = 512;                 // per-warp staging slots for re-queued ids
constexpr uint32_t kMaxSamples = 4096;      // cap on the rho sampler's sample count
constexpr uint32_t kWarmSamples = 1024;     // ... in rho-Stepping's warm-up steps
constexpr uint64_t kInf = ~0ull;

// Dynamic shared memory.  Per warp kStage re-queue staging slots (relaxation
// phase); the rho sampler's keys reuse the same region at the start of a step
// (the staging slots are empty between steps).
constexpr uint32_t kStageBytes = kWarps * (uint32_t)kStage * 4u;        // 64 KB
// Batched / serving kernels: staging (and the sampler's keys).
constexpr uint32_t kBatchDynSmem = kStageBytes > kMaxSamples * 8u ? kStageBytes : kMaxSamples * 8u;
// Single solve: Extract stages one round of up to kExtractCap queue entries
// of one of the block's runs (a 16-byte record and a kind byte each) in the same
// region (Extract, the sampler and the relaxation never overlap in time).
#ifndef SSSP_EXTRACT_PER
#define SSSP_EXTRACT_PER 4
#endif
constexpr int kExtractPer = SSSP_EXTRACT_PER;                           // entries per thread per round
constexpr uint32_t kExtractCap = (uint32_t)kBlock * kExtractPer;        // 4096
constexpr uint32_t kExtractBytes = kExtractCap * 16u + kExtractCap;     // 68 KB
constexpr uint32_t kSolveDynSmem = kExtractBytes > kBatchDynSmem ? kExtractBytes : kBatchDynSmem;

// Relaxation records written by Extract and read by the relaxation (16 bytes,
// make_rec / rec_start / rec_len): x,y = first edge index | (edge count << 40);
// z,w = delta[u] at extraction for a low-degree record (all of u's <= kSmallDeg
// edges), z = u for a chunk record (at most kChunk edges of u within one
// kChunk-aligned block of the edge array).

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
    unsigned long long umin[3];   // smallest distance written by the relaxation of the step (slot of Q_{k+1})
    unsigned long long ledges[3]; // edges relaxed by the local relaxation of super-sparse steps
    // totals, written by block 0 when the solve ends
    unsigned long long steps, queued, extracted, edges, updates_total;
    unsigned long long t0;        // solve start on the device clock (block 0), the origin of trace times
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
    uint4* fsmall;                // records of extracted vertices with 1 <= degree <= kSmallDeg
    uint64_t fsmall_cap;
    uint4* items;                 // chunk records of extracted vertices with degree > kSmallDeg
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
    uint32_t sample_cap;          // power of two >= the largest sample count (<= kMaxSamples)
    sssp_stats* stats_out;        // optional device copy of the totals
    int bidir;                    // bidirectional relaxation of chunk records (symmetric graphs)
    uint32_t local_budget;        // local relaxation of super-sparse steps: vertices per warp and step (0 = off)
    uint32_t rho_reduced;         // rho-Stepping: dense steps that use rho/10
    uint64_t* lrel;               // [n] distance each vertex was last locally relaxed with, or null
    uint32_t small_deg;           // degree-bin cut-off: 1..small_deg -> low-degree records
    uint32_t chunk_log2;          // chunk records cover at most 2^chunk_log2 edges (aligned)
    // SSSP_SOLVE_FUSED: per block two step-parity buffers of kExtractCap
    // (vertex, -, distance it was relaxed with) -- the vertices the block
    // extracted in a fused step, re-checked after the step; null = no fused steps
    uint4* fre;
    // rho-Stepping warm-up: steps 1..warm_steps use rho = warm_rho (no
    // dense-step reduction, not counted as dense steps); 0 = none
    uint32_t warm_steps;
    uint64_t warm_rho;
    // relabelled graph (SSSP_GRAPH_REORDER): the solve runs on the relabelled
    // copy with dist = internal distances in the new ids; at the end
    // dist_out[v] = dist[perm[v]] for every caller id v; ext_count is indexed
    // through iperm (new -> caller id).  All null without relabelling.
    const uint32_t* perm;
    const uint32_t* iperm;
    uint64_t* dist_out;
};

// Chunk records of one vertex: its edge range [b, e) cut at multiples of 2^lg.
inline uint64_t chunk_count(uint64_t b, uint64_t e, uint32_t lg = kChunkLog2)
{
    return e > b ? ((e - 1) >> lg) - (b >> lg) + 1 : 0;
}

// Upper bound on chunk records of one Extract when only n and m are known:
// each vertex of degree > kSmallDeg yields at most deg/kChunk + 2 records and
// there are at most m/(kSmallDeg+1) such vertices.
inline uint64_t item_capacity_bound(uint64_t n, uint64_t m)
{
    uint64_t heavy = m / (kSmallDeg + 1);
    if (heavy > n) heavy = n;
    return m / kChunk + 2ull * heavy + 64;
}

// Launch helpers implemented in sssp_kernels.cu.
cudaError_t launch_pack_edges(const uint32_t* tgt, const uint32_t* w, uint2* edges, uint64_t m,
                              uint64_t m_pad, cudaStream_t st);
const void* solve_kernel_ptr();
int solve_kernel_threads();             // threads per block of this build of the solve kernel
unsigned int solve_kernel_smem();       // its dynamic shared memory per block
cudaError_t launch_rho_threshold(const uint32_t* queue, uint32_t q, const uint64_t* dist,
                                 uint32_t n, uint64_t rho, uint64_t seed, uint64_t step,
                                 uint32_t dense_before, uint32_t reduced, uint32_t max_samples, uint64_t* theta_out,
                                 uint32_t* err_out, cudaStream_t st);
uint32_t rho_sample_bound(uint32_t n, uint64_t rho);   // power-of-two smem keys needed

// Batched solves (sssp_batch.cu).
constexpr uint32_t kMaxBatch = 2048;        // instances per batched launch
const void* batch_kernel_ptr();
const void* serve_kernel_ptr();

// Query servers: one command and one completion record per slot in
// host-mapped memory, and the host's submission counter / stop flag.
struct SlotCmd {                  // written by the host
    unsigned long long ticket;
    unsigned long long dist_ptr;  // caller-owned device uint64[n]
    unsigned int source;
    unsigned int seq;             // written last
};
struct SlotDone {                 // written by the device
    unsigned long long ticket;
    unsigned long long t_admit_ns, t_done_ns;
    unsigned long long edges, extracted;
    unsigned int steps;
    int status;
    unsigned int seq;             // written last
    unsigned int pad;
};
struct ServeShared {              // host-mapped
    unsigned long long submitted; // host: commands written so far (monotone)
    unsigned int stop;            // host: leave the loop
    unsigned int pad;
};

// The shared-scan server's device state (sssp_msbatch.cu): a persistent loop
// over S <= 64 query slots that are the instances of the shared-scan kernel.
struct MsServer;
size_t ms_server_bytes(const sssp_graph* g, uint32_t S);
int ms_server_create(const sssp_graph* g, uint32_t S, sssp_algo algo, uint64_t param, uint32_t rho_reduced,
                     uint32_t warm_steps, uint64_t warm_rho, bool bidir, SlotCmd* d_cmd, SlotDone* d_done, ServeShared* d_shared, uint64_t idle_ns,
                     uint32_t gang, uint64_t gang_wait_ns, MsServer** out);
int ms_server_launch(MsServer* s, cudaStream_t st);
int ms_server_status(MsServer* s);      // device status after the loop returned (synchronous)
void ms_server_destroy(MsServer* s);

// Batched solves of k <= 64 sources on one graph with one shared edge scan
// per step (sssp_msbatch.cu): outs[i] receives instance i's distances.
bool ms_batch_supported(sssp_algo algo, uint32_t k);
int ms_solve_sources(const sssp_graph* g, const uint32_t* sources, uint32_t k, sssp_algo algo,
                     const uint64_t* params, uint64_t* const* outs, uint32_t rho_reduced, uint32_t warm_steps,
                     uint64_t warm_rho, bool bidir, void* stream);
int ms_last_stats(int dev, sssp_stats* out, uint32_t k, cudaStream_t st);
constexpr uint32_t kMsRecEdges = 32;        // edges per relaxation record of the shared-scan kernel

}  // namespace sssp

// The narrow build of the solve kernel (sssp_kernels.cu compiled with
// SSSP_BLOCK=512 into this namespace; SolveParams and Ctrl have the same layout).
namespace sssp_narrow {
const void* solve_kernel_ptr();
int solve_kernel_threads();
unsigned int solve_kernel_smem();
}

// Library-side state of one graph handle (host ABI and batched solves).
struct sssp_graph {
    uint32_t n = 0;
    uint64_t m = 0;
    int device = 0;
    int num_sms = 0;
    uint64_t* d_off = nullptr;
    uint2* d_edges = nullptr;
    // scratch
    uint32_t* d_inq = nullptr;
    uint32_t* d_qa = nullptr;
    uint32_t* d_qb = nullptr;
    uint4* d_fsmall = nullptr;
    uint64_t fsmall_cap = 0;               // records of one Extract at the default cut-offs
    uint4* d_items = nullptr;
    uint64_t item_cap = 0;
    uint64_t fsmall_cap_any = 0;           // ... at any allowed cut-offs (single-solve scratch)
    uint64_t item_cap_any = 0;
    uint64_t ms_rec_cap = 0;               // shared-scan batch: per-warp records of one Extract (sum of ceil(deg/32))
    sssp::Ctrl* d_ctrl = nullptr;
    uint64_t* d_dist_internal = nullptr;   // lazily allocated for sssp_solve_host
    uint64_t* d_lrel = nullptr;            // lazily allocated for solves with local relaxation
    uint4* d_fre = nullptr;                // lazily allocated for solves with SSSP_SOLVE_FUSED
    uint64_t fre_cap = 0;                  // its entries
    // SSSP_GRAPH_REORDER: relabelled copy for single solves (new id = rank by
    // decreasing out-degree, ties by id; adjacencies sorted by new target)
    bool reordered = false;
    uint64_t* d_off2 = nullptr;
    uint2* d_edges2 = nullptr;
    uint32_t* d_perm = nullptr;            // caller id -> new id
    uint32_t* d_iperm = nullptr;           // new id -> caller id
    uint64_t* d_dist2 = nullptr;           // distances in the new ids
    std::vector<uint32_t> h_perm;          // caller id -> new id (source mapping)
    sssp::Ctrl* h_ctrl = nullptr;                // pinned readback
    uint32_t last_grid = 0;
    double mean_w = 1.0;                   // mean edge weight (default Delta)
    uint64_t max_deg = 0;                  // largest out-degree (graph class)
    uint32_t flags = 0;                    // SSSP_GRAPH_* flags given at creation
    bool tuned = false;                    // tuning holds an autotuner result (or a set one)
    sssp_tuning tuning = {};
    bool batch_tuned = false;              // batch_tuning holds a result of sssp_autotune_batch
    sssp_tuning batch_tuning = {};
    std::mutex mu;                         // guards lazy allocations / attributes
};

// Parameter used when a batched call passes no per-instance parameters: for
// rho-Stepping rho = max(64, n/16) (the best of the rho sweep on the RMAT
// scale-22 workload is 2^18 = n/16), for Delta*-Stepping Delta = max(1,
// mean weight / 4) (best of the Delta sweep there), 0 for Bellman-Ford.
inline uint64_t sssp_default_param(uint32_t n, uint64_t /*m*/, sssp_algo algo, double mean_w = 4.0)
{
    if (algo == SSSP_RHO) return n / 16 > 64 ? n / 16 : 64;
    if (algo == SSSP_DELTA_STAR || algo == SSSP_DELTA) { const double d = mean_w / 4.0; return d > 1.0 ? (uint64_t)d : 1; }
    return 0;
}

// The ExtDist rules that need the smallest queued distance each step.
inline __host__ __device__ bool algo_tracks_qmin(int algo)
{
    return algo == SSSP_DELTA_STAR || algo == SSSP_DELTA || algo == SSSP_DIJKSTRA;
}
inline __host__ __device__ bool algo_valid(int algo) { return algo >= SSSP_RHO && algo <= SSSP_DIJKSTRA; }
inline __host__ __device__ bool algo_needs_param(int algo)
{
    return algo == SSSP_RHO || algo == SSSP_DELTA_STAR || algo == SSSP_DELTA;
}

// Autotuner results (sssp_tune.cu): the class key of a graph (log2 n, mean
// degree, degree skew, symmetry), the tuning that applies to a graph (its own,
// else its class's), and the parameter a call that passes none uses.
uint64_t sssp_class_key(const sssp_graph* g);
bool sssp_lookup_tuning(const sssp_graph* g, sssp_tuning* out);
uint64_t sssp_graph_param(const sssp_graph* g, sssp_algo algo);
// The tuning batched and serving launches use: the graph's batch tuning
// (sssp_autotune_batch), else sssp_lookup_tuning's.
bool sssp_lookup_batch_tuning(const sssp_graph* g, sssp_tuning* out);
uint64_t sssp_graph_batch_param(const sssp_graph* g, sssp_algo algo);
