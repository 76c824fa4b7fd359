// sssp_noalloc.cu -- a solve entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need a
// solve: a plugin whose enqueue step runs inside a framework that owns all
// device memory through its own pool, or a latency-critical loop that cannot
// afford the implicit device synchronisation of cudaMalloc/cudaFree.
// sssp_solve_noalloc serves them: the caller passes the graph, already in
// device memory, and the output buffer; the solver's working memory (queue
// bitmap, queue lists, extraction lists, control block) comes from the
// file-scope array below, which every GPU that loads this module holds until
// the process exits.  No cudaMalloc, cudaFree or allocating library routine
// is called on this path.
//
// The array is shared by every call on a device and keeps the previous
// call's contents; the solve itself re-initialises what must start from a
// known state (the control block is cleared before each launch, the queue
// bitmap and distances at the start of the kernel).  Calls that overlap on
// the GPU (two streams, or two host threads without ordering) race on it.

#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "sssp_internal.h"

using namespace sssp;

namespace {

constexpr uint64_t align256(uint64_t x) { return (x + 255ull) & ~255ull; }

constexpr uint64_t kNaVertices = SSSP_NOALLOC_MAX_VERTICES;
constexpr uint64_t kNaEdges = SSSP_NOALLOC_MAX_EDGES;
constexpr uint64_t kNaHeavy = kNaEdges / (kSmallDeg + 1) < kNaVertices ? kNaEdges / (kSmallDeg + 1) : kNaVertices;
constexpr uint64_t kNaItems = kNaEdges / kChunk + 2ull * kNaHeavy + 64ull;  // chunk-record bound

// byte offsets of the regions inside the scratch array
constexpr uint64_t kOffCtrl = 0;
constexpr uint64_t kOffInq = align256(kOffCtrl + sizeof(Ctrl));
constexpr uint64_t kOffQa = align256(kOffInq + 4ull * ((kNaVertices + 31) / 32));
constexpr uint64_t kOffQb = align256(kOffQa + 4ull * kNaVertices);
constexpr uint64_t kOffFsmall = align256(kOffQb + 4ull * kNaVertices);
constexpr uint64_t kOffItems = align256(kOffFsmall + 16ull * kNaVertices);
constexpr uint64_t kScratchBytes = align256(kOffItems + 16ull * kNaItems);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
uint32_t g_grid[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// scratch array (its host-side name is only a stand-in, not a device
// address) and the cooperative grid of the solve kernel (blocks per SM x SMs,
// with the kernel's shared-memory attribute set).  Later calls reuse both, so
// a call does no host-side set-up work.
int setup_device(int dev, unsigned char** scratch, uint32_t* grid)
{
    if (dev < 0 || dev >= kMaxDevices) return SSSP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) return SSSP_ERR_CUDA;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || sms <= 0) return SSSP_ERR_CUDA;
        const void* fn = solve_kernel_ptr();
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveDynSmem);
        if (e != cudaSuccess) return SSSP_ERR_CUDA;
        int bps = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlock, kSolveDynSmem);
        if (e != cudaSuccess || bps < 1) return SSSP_ERR_CUDA;
        g_grid[dev] = (uint32_t)(bps * sms);
        g_scratch_addr[dev] = ptr;
    }
    *scratch = static_cast<unsigned char*>(g_scratch_addr[dev]);
    *grid = g_grid[dev];
    return SSSP_OK;
}

}  // namespace

extern "C" int sssp_solve_noalloc(uint32_t n, uint64_t m, const uint64_t* offsets, const uint32_t* edges,
                                  uint32_t source, sssp_algo algo, uint64_t param, uint64_t* dist_out,
                                  sssp_stats* stats_out, void* stream)
{
    if (n == 0 || n > kNaVertices || m > kNaEdges) return SSSP_ERR_INVALID_ARG;
    if (!offsets || !dist_out || (m > 0 && !edges)) return SSSP_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(edges) & 15u) != 0) return SSSP_ERR_INVALID_ARG;
    if (source >= n) return SSSP_ERR_INVALID_ARG;
    if (!algo_valid(algo)) return SSSP_ERR_INVALID_ARG;
    if (algo_needs_param(algo) && param == 0) return SSSP_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SSSP_ERR_CUDA;
    unsigned char* base = nullptr;
    uint32_t grid = 0;
    int rc = setup_device(dev, &base, &grid);
    if (rc != SSSP_OK) return rc;

    SolveParams p;
    memset(&p, 0, sizeof p);
    p.off = offsets;
    p.edges = reinterpret_cast<const uint2*>(edges ? edges : reinterpret_cast<const uint32_t*>(base + kOffItems));
    p.n = n;
    p.m = m;
    p.dist = dist_out;
    p.inq = reinterpret_cast<uint32_t*>(base + kOffInq);
    p.qa = reinterpret_cast<uint32_t*>(base + kOffQa);
    p.qb = reinterpret_cast<uint32_t*>(base + kOffQb);
    p.fsmall = reinterpret_cast<uint4*>(base + kOffFsmall);
    p.fsmall_cap = kNaVertices;
    p.items = reinterpret_cast<uint4*>(base + kOffItems);
    p.item_cap = kNaItems;
    p.ctrl = reinterpret_cast<Ctrl*>(base + kOffCtrl);
    p.source = source;
    p.algo = (int)algo;
    p.param = param;
    p.seed = 0x2105061450000000ull ^ (uint64_t)source;
    p.timeout_ns = 2000000000ull;
    p.solve_timeout_ns = 60000000000ull;
    p.stats_out = stats_out;
    p.sample_cap = (algo == SSSP_RHO) ? rho_sample_bound(n, param) : 0;
    p.rho_reduced = kRhoReducedDefault;
    p.small_deg = kSmallDeg;
    p.chunk_log2 = kChunkLog2;

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), st);  // the control block must start at zero
    if (e != cudaSuccess) return SSSP_ERR_CUDA;
    void* args[] = {&p};
    e = cudaLaunchCooperativeKernel(solve_kernel_ptr(), dim3(grid), dim3(kBlock), args, kSolveDynSmem, st);
    return e == cudaSuccess ? SSSP_OK : SSSP_ERR_CUDA;
}
