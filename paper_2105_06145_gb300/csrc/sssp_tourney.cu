// sssp_tourney.cu -- the tournament-tree LaB-PQ of Sec. 4.2 (Algorithm 2) on
// the device, as a stand-alone data structure behind its own C ABI calls.
//
// A complete binary tree over N = 2^L leaves (N >= n; leaf N + id holds record
// id, leaves beyond n are never in Q) in heap order: node t has children 2t and
// 2t + 1, node 1 is the root.  Interior node t keeps key[t], the smallest key of
// the records in its subtree that are in Q (as of the last Sync), and a
// "renewed" flag (bit t of a bitmap) set when a leaf below changed since.  A
// record's key is delta[id] (the key array is passed by pointer, as in Sec. 3.1).
//
//   Mark(id, f)    inQ(id) <- f, then test-and-set the renewed flags from the
//                  leaf's parent upward, stopping at the first flag that was
//                  already set (Algorithm 2, Mark).  A flag that is newly set
//                  also appends its node to the list of its level, so that Sync
//                  visits only renewed nodes.
//   Sync           level by level from the deepest interior level to the root:
//                  every renewed node takes the smaller key of its children and
//                  clears its flag (Algorithm 2, Update; bottom-up instead of the
//                  recursive top-down order: same keys, one pass per level).
//   Traverse(th)   level by level from the root: nodes whose key is <= th are
//                  expanded; a leaf whose record is in Q with key <= th is
//                  output and Marked out of Q (Algorithm 2, Traverse).
//   Extract(th)    Sync, then Traverse (Algorithm 2, Extract).
//   LazyInsert(id) Mark(id, 1).  Reduce (min over Q) = key[1] after a Sync.
//
// Every level is one kernel launch on the caller's stream (the launches order
// the levels); the level lists and the traversal frontiers hold at most 2^l
// entries at level l.
#include <cstdint>
#include <cstring>
#include <new>
#include <cuda_runtime.h>

#include "sssp_internal.h"
#include "sssp_device.cuh"

struct sssp_tourney {
    uint32_t n = 0;
    uint32_t L = 0;                  // levels of interior nodes: 0 (root) .. L-1
    uint64_t N = 0;                  // leaves, 2^L
    uint64_t* d_key = nullptr;       // [N] interior keys (index 0 unused)
    uint32_t* d_renew = nullptr;     // [N/32] renewed flags of interior nodes
    uint32_t* d_inq = nullptr;       // [ceil(n/32)] inQ flags of the records
    uint32_t* d_lists = nullptr;     // level lists: level l at offset 2^l - 1, capacity 2^l
    uint32_t* d_cnt = nullptr;       // [L] list lengths; [L .. L+1] frontier counters
    uint32_t* d_front = nullptr;     // two traversal frontiers, N entries each
};

namespace {

constexpr int kTBlock = 256;
constexpr uint64_t kTInf = ~0ull;

int fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? SSSP_ERR_OUT_OF_MEMORY : SSSP_ERR_CUDA; }

unsigned int grid_for(uint64_t items)
{
    uint64_t b = (items + kTBlock - 1) / kTBlock;
    if (b < 1) b = 1;
    if (b > 4096) b = 4096;
    return (unsigned int)b;
}

// Mark(id, flag) for a batch: thread per id (grid-strided).
__global__ void tt_mark_kernel(const uint32_t* __restrict__ ids, uint32_t b, uint32_t flag, uint32_t n, uint64_t N,
                               uint32_t L, uint32_t* inq, uint32_t* renew, uint32_t* lists, uint32_t* cnt)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < b; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t id = ids[i];
        if (id >= n) continue;
        if (flag) atomicOr(&inq[id >> 5], 1u << (id & 31u));
        else atomicAnd(&inq[id >> 5], ~(1u << (id & 31u)));
        uint64_t t = (N + id) >> 1;
        uint32_t level = L - 1;
        while (t >= 1) {
            const uint32_t bit = 1u << (t & 31u);
            const uint32_t prev = atomicOr(&renew[t >> 5], bit);
            if (prev & bit) break;  // another Mark owns the rest of the path
            const uint32_t pos = atomicAdd(&cnt[level], 1u);
            lists[((1ull << level) - 1) + pos] = (uint32_t)t;
            t >>= 1;
            if (level == 0) break;
            --level;
        }
    }
}

__device__ __forceinline__ uint64_t leaf_key(uint64_t c, uint64_t N, uint32_t n, const uint32_t* inq,
                                             const uint64_t* keys)
{
    const uint64_t id = c - N;
    if (id >= n) return kTInf;
    const bool in = (__ldcg(&inq[id >> 5]) >> (id & 31u)) & 1u;
    return in ? __ldcg(reinterpret_cast<const unsigned long long*>(&keys[id])) : kTInf;
}

// Sync of one level: every renewed node on the level's list takes the smaller
// key of its children and clears its flag; the list is emptied.
__global__ void tt_sync_level_kernel(uint32_t level, uint32_t L, uint64_t N, uint32_t n, const uint64_t* keys,
                                     uint64_t* key, uint32_t* renew, const uint32_t* inq, const uint32_t* lists,
                                     uint32_t* cnt)
{
    const uint32_t c = __ldcg(&cnt[level]);
    const uint32_t* lst = lists + ((1ull << level) - 1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = lst[i];
        uint64_t a, b;
        if (level == L - 1) {
            a = leaf_key(2 * t, N, n, inq, keys);
            b = leaf_key(2 * t + 1, N, n, inq, keys);
        } else {
            a = __ldcg(reinterpret_cast<const unsigned long long*>(&key[2 * t]));
            b = __ldcg(reinterpret_cast<const unsigned long long*>(&key[2 * t + 1]));
        }
        key[t] = a < b ? a : b;
        atomicAnd(&renew[t >> 5], ~(1u << (t & 31u)));
    }
}

__global__ void tt_reset_count_kernel(uint32_t* cnt, uint32_t i) { cnt[i] = 0; }

// Traverse of one level: expand the frontier nodes (key <= theta) into the
// next frontier, or, below the last interior level, output the records in Q
// with key <= theta and Mark them out of Q.
__global__ void tt_traverse_level_kernel(uint32_t level, uint32_t L, uint64_t N, uint32_t n, uint64_t theta,
                                         const uint64_t* keys, const uint64_t* key, uint32_t* inq, uint32_t* renew,
                                         uint32_t* lists, uint32_t* cnt, const uint32_t* front_in,
                                         uint32_t* front_out, uint32_t in_slot, uint32_t out_slot, uint32_t* out,
                                         uint32_t* out_count)
{
    // level 0: the frontier is the root when its key <= theta (count 0 or 1)
    const uint32_t c = __ldcg(&cnt[L + in_slot]);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2ull * c;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t t = level == 0 ? 1ull : front_in[i >> 1];
        const uint64_t ch = 2 * t + (i & 1u);
        if (level < L - 1) {
            if (__ldcg(reinterpret_cast<const unsigned long long*>(&key[ch])) <= theta)
                front_out[atomicAdd(&cnt[L + out_slot], 1u)] = (uint32_t)ch;
        } else {
            const uint64_t id = ch - N;
            // a record must be in Q (its key may be UINT64_MAX = theta)
            const bool in = id < n && ((__ldcg(&inq[id >> 5]) >> (id & 31u)) & 1u);
            if (in && __ldcg(reinterpret_cast<const unsigned long long*>(&keys[id])) <= theta) {
                out[atomicAdd(out_count, 1u)] = (uint32_t)id;
                // Mark(id, 0): leave Q, renew the path
                atomicAnd(&inq[id >> 5], ~(1u << (id & 31u)));
                uint64_t u = ch >> 1;
                uint32_t lv = L - 1;
                while (u >= 1) {
                    const uint32_t bit = 1u << (u & 31u);
                    const uint32_t prev = atomicOr(&renew[u >> 5], bit);
                    if (prev & bit) break;
                    const uint32_t pos = atomicAdd(&cnt[lv], 1u);
                    lists[((1ull << lv) - 1) + pos] = (uint32_t)u;
                    u >>= 1;
                    if (lv == 0) break;
                    --lv;
                }
            }
        }
    }
}

// Before a Traverse: the level-0 frontier (slot 0) is the root only if its
// key <= theta; the other frontier slot and the output count start at 0.
__global__ void tt_traverse_begin_kernel(const uint64_t* key, uint64_t theta, uint32_t L, uint32_t* cnt,
                                         uint32_t* out_count)
{
    cnt[L] = key[1] <= theta ? 1u : 0u;
    cnt[L + 1] = 0;
    *out_count = 0;
}

int tt_sync(sssp_tourney* t, const uint64_t* keys, cudaStream_t st)
{
    for (int64_t level = (int64_t)t->L - 1; level >= 0; --level) {
        tt_sync_level_kernel<<<grid_for(1ull << level), kTBlock, 0, st>>>((uint32_t)level, t->L, t->N, t->n, keys,
                                                                          t->d_key, t->d_renew, t->d_inq,
                                                                          t->d_lists, t->d_cnt);
        tt_reset_count_kernel<<<1, 1, 0, st>>>(t->d_cnt, (uint32_t)level);
    }
    return cudaGetLastError() == cudaSuccess ? SSSP_OK : SSSP_ERR_CUDA;
}

}  // namespace

extern "C" {

int sssp_tourney_create(uint32_t n, sssp_tourney** out)
{
    if (!out || n == 0 || n > (1u << 31)) return SSSP_ERR_INVALID_ARG;
    *out = nullptr;
    sssp_tourney* t = new (std::nothrow) sssp_tourney();
    if (!t) return SSSP_ERR_OUT_OF_MEMORY;
    t->n = n;
    t->L = 1;
    while ((1ull << t->L) < n) ++t->L;
    t->N = 1ull << t->L;
    cudaError_t e;
    if ((e = cudaMalloc(reinterpret_cast<void**>(&t->d_key), sizeof(uint64_t) * t->N)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&t->d_renew), sizeof(uint32_t) * ((t->N + 31) / 32))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&t->d_inq), sizeof(uint32_t) * ((n + 31ull) / 32))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&t->d_lists), sizeof(uint32_t) * t->N)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&t->d_cnt), sizeof(uint32_t) * (t->L + 2))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&t->d_front), sizeof(uint32_t) * 2 * t->N)) != cudaSuccess) {
        sssp_tourney_destroy(t);
        return fail(e);
    }
    // empty Q: every key +inf, nothing renewed
    if ((e = cudaMemset(t->d_key, 0xFF, sizeof(uint64_t) * t->N)) != cudaSuccess ||
        (e = cudaMemset(t->d_renew, 0, sizeof(uint32_t) * ((t->N + 31) / 32))) != cudaSuccess ||
        (e = cudaMemset(t->d_inq, 0, sizeof(uint32_t) * ((n + 31ull) / 32))) != cudaSuccess ||
        (e = cudaMemset(t->d_cnt, 0, sizeof(uint32_t) * (t->L + 2))) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        sssp_tourney_destroy(t);
        return fail(e);
    }
    *out = t;
    return SSSP_OK;
}

int sssp_tourney_destroy(sssp_tourney* t)
{
    if (!t) return SSSP_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    cudaFree(t->d_key);
    cudaFree(t->d_renew);
    cudaFree(t->d_inq);
    cudaFree(t->d_lists);
    cudaFree(t->d_cnt);
    cudaFree(t->d_front);
    delete t;
    return SSSP_OK;
}

int sssp_tourney_update(sssp_tourney* t, const uint32_t* ids, uint32_t b, void* stream)
{
    if (!t || (b > 0 && !ids)) return SSSP_ERR_INVALID_ARG;
    if (b == 0) return SSSP_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    tt_mark_kernel<<<grid_for(b), kTBlock, 0, st>>>(ids, b, 1u, t->n, t->N, t->L, t->d_inq, t->d_renew, t->d_lists,
                                                    t->d_cnt);
    return cudaGetLastError() == cudaSuccess ? SSSP_OK : SSSP_ERR_CUDA;
}

int sssp_tourney_extract(sssp_tourney* t, const uint64_t* keys, uint64_t theta, uint32_t* out, uint32_t* count_out,
                         void* stream)
{
    if (!t || !keys || !out || !count_out) return SSSP_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = tt_sync(t, keys, st);
    if (rc != SSSP_OK) return rc;
    tt_traverse_begin_kernel<<<1, 1, 0, st>>>(t->d_key, theta, t->L, t->d_cnt, count_out);
    for (uint32_t level = 0; level < t->L; ++level) {
        const uint32_t in_slot = level & 1u, out_slot = in_slot ^ 1u;
        uint32_t* fin = t->d_front + (uint64_t)in_slot * t->N;
        uint32_t* fout = t->d_front + (uint64_t)out_slot * t->N;
        tt_traverse_level_kernel<<<grid_for(2ull << level), kTBlock, 0, st>>>(
            level, t->L, t->N, t->n, theta, keys, t->d_key, t->d_inq, t->d_renew, t->d_lists, t->d_cnt,
            level == 0 ? nullptr : fin, fout, in_slot, out_slot, out, count_out);
        // the next level reads out_slot; clear in_slot for the level after it
        tt_reset_count_kernel<<<1, 1, 0, st>>>(t->d_cnt, t->L + in_slot);
    }
    return cudaGetLastError() == cudaSuccess ? SSSP_OK : SSSP_ERR_CUDA;
}

int sssp_tourney_min(sssp_tourney* t, const uint64_t* keys, uint64_t* min_out, void* stream)
{
    if (!t || !keys || !min_out) return SSSP_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = tt_sync(t, keys, st);
    if (rc != SSSP_OK) return rc;
    cudaError_t e = cudaMemcpyAsync(min_out, t->d_key + 1, sizeof(uint64_t), cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? SSSP_OK : fail(e);
}

int sssp_tourney_inq(const sssp_tourney* t, uint32_t* inq_out, void* stream)
{
    if (!t || !inq_out) return SSSP_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(inq_out, t->d_inq, sizeof(uint32_t) * ((t->n + 31ull) / 32),
                                    cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? SSSP_OK : fail(e);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The array-based LaB-PQ's Extract (Sec. 4.3) as a stand-alone operation, for
// comparing the two implementations (App. F): the queue is a list of ids; the
// ids with key <= theta are written to `ext`, the others to `keep` (both in
// list order within a warp, warps in any order).
// ---------------------------------------------------------------------------
namespace {
constexpr int kAItems = 8;  // list entries per thread per tile

__global__ void __launch_bounds__(kTBlock) array_extract_kernel(const uint32_t* __restrict__ list, uint32_t q,
                                                                const uint64_t* __restrict__ keys, uint64_t theta,
                                                                uint32_t* ext, uint32_t* ext_count, uint32_t* keep,
                                                                uint32_t* keep_count)
{
    // a tile of kTBlock * kAItems entries per block: the id and key loads of
    // the tile are in flight together; one atomic per output list per tile
    __shared__ uint32_t s_we[kTBlock / 32], s_wk[kTBlock / 32], s_base[2];
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint64_t tile = (uint64_t)kTBlock * kAItems;
    for (uint64_t t0 = (uint64_t)blockIdx.x * tile; t0 < q; t0 += (uint64_t)gridDim.x * tile) {
        uint32_t v[kAItems];
        bool x[kAItems], in[kAItems];
#pragma unroll
        for (int j = 0; j < kAItems; ++j) {
            const uint64_t i = t0 + ((uint64_t)j * kTBlock) + threadIdx.x;
            in[j] = i < q;
            v[j] = in[j] ? __ldcg(&list[i]) : 0u;
        }
#pragma unroll
        for (int j = 0; j < kAItems; ++j)
            x[j] = in[j] && __ldcg(reinterpret_cast<const unsigned long long*>(&keys[v[j]])) <= theta;
        uint32_t ne = 0, nk = 0;
#pragma unroll
        for (int j = 0; j < kAItems; ++j) {
            ne += __popc(__ballot_sync(0xFFFFFFFFu, x[j]));
            nk += __popc(__ballot_sync(0xFFFFFFFFu, in[j] && !x[j]));
        }
        if (lane == 0) { s_we[wid] = ne; s_wk[wid] = nk; }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t te = 0, tk = 0;
            for (int w = 0; w < kTBlock / 32; ++w) {
                const uint32_t a = s_we[w], b = s_wk[w];
                s_we[w] = te; s_wk[w] = tk;
                te += a; tk += b;
            }
            s_base[0] = te ? atomicAdd(ext_count, te) : 0u;
            s_base[1] = tk ? atomicAdd(keep_count, tk) : 0u;
        }
        __syncthreads();
        uint32_t pe = s_base[0] + s_we[wid], pk = s_base[1] + s_wk[wid];
#pragma unroll
        for (int j = 0; j < kAItems; ++j) {
            const uint32_t be = __ballot_sync(0xFFFFFFFFu, x[j]);
            const uint32_t bk = __ballot_sync(0xFFFFFFFFu, in[j] && !x[j]);
            if (x[j]) ext[pe + __popc(be & lt)] = v[j];
            else if (in[j]) keep[pk + __popc(bk & lt)] = v[j];
            pe += __popc(be);
            pk += __popc(bk);
        }
        __syncthreads();
    }
}
__global__ void zero2_kernel(uint32_t* a, uint32_t* b) { *a = 0; *b = 0; }
}  // namespace

extern "C" int sssp_array_extract(const uint32_t* list, uint32_t q, const uint64_t* keys, uint64_t theta,
                                  uint32_t* ext, uint32_t* ext_count, uint32_t* keep, uint32_t* keep_count,
                                  void* stream)
{
    if ((q > 0 && !list) || !keys || !ext || !ext_count || !keep || !keep_count) return SSSP_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    zero2_kernel<<<1, 1, 0, st>>>(ext_count, keep_count);
    if (q > 0) {
        uint64_t blocks = ((uint64_t)q + (uint64_t)kTBlock * kAItems - 1) / ((uint64_t)kTBlock * kAItems);
        blocks = blocks < 8192 ? blocks : 8192;
        array_extract_kernel<<<(unsigned)blocks, kTBlock, 0, st>>>(list, q, keys, theta, ext, ext_count, keep,
                                                                   keep_count);
    }
    return cudaGetLastError() == cudaSuccess ? SSSP_OK : SSSP_ERR_CUDA;
}
