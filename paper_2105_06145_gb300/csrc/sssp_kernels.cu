// sssp_kernels.cu -- device code of libsssp (sm_103a).
//
// One persistent cooperative kernel runs the whole stepping loop of
// Algorithm 1 (Sec. 3.2) over the array-based LaB-PQ of Sec. 4.3:
//
//   init      delta[.] = inf, delta[s] = 0, Q = {s}                 (Alg. 1)
//   per step  theta   = ExtDist  (Table 2; rho sampling of Sec. 6 / App. B)
//             F       = Extract(theta): queued ids with delta <= theta leave Q
//             ---- grid barrier (Extract is not concurrent with Update, Sec. 3.1)
//             for u in F, (v,w) in N(u): WriteMin(delta[v], delta[u] + w),
//                 on success Update(v) = test-and-set of v's queue bit,
//                 append v to the next queue list when the bit was clear
//             ---- grid barrier
//   until |Q| = 0
//
// State that must be coherent across blocks (delta, the queue bitmap, queue
// lists, counters) is read with L2-only loads (ld.global.cg) or atomics;
// the graph (offsets, packed edges) is read-only for the kernel's lifetime.
// Every device-wide wait is bounded by a globaltimer deadline; on expiry the
// kernel records SSSP_ERR_TIMEOUT and every block returns.

#include <cstdint>
#include <cuda_runtime.h>

#include "sssp_internal.h"

namespace sssp {

#define FULL_MASK 0xFFFFFFFFu

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t ldcg64(const uint64_t* p)
{
    return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ uint32_t ldcg32(const uint32_t* p) { return __ldcg(p); }

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void set_status(Ctrl* c, int code) { atomicCAS(&c->status, 0, code); }

// splitmix64 (Steele, Lea, Flood 2014): output k of the generator started at
// state `seed` is mix(seed + (k+1) * golden_gamma).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t sat_mul(uint64_t a, uint64_t b)
{
    return (b != 0 && a > kInf / b) ? kInf : a * b;
}

// ---------------------------------------------------------------------------
// bounded grid barrier (all blocks are co-resident: cooperative launch)
// ---------------------------------------------------------------------------
__device__ __noinline__ bool grid_sync(Ctrl* ctrl, unsigned long long& target, uint64_t timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        target += gridDim.x;
        __threadfence();
        atomicAdd(&ctrl->bar, 1ull);
        int ok = 1;
        const unsigned long long t0 = global_timer_ns();
        unsigned int spins = 0;
        while (ld_acquire_u64(&ctrl->bar) < target) {
            if ((++spins & 31u) == 0) {
                if (*reinterpret_cast<volatile int*>(&ctrl->status) != 0) { ok = 0; break; }
                if (global_timer_ns() - t0 > timeout_ns) { set_status(ctrl, SSSP_ERR_TIMEOUT); ok = 0; break; }
            }
        }
        __threadfence();
        // an error recorded before the barrier (timeout, capacity, step or time
        // guard) is visible to every block after it: all of them leave together
        if (ok && *reinterpret_cast<volatile int*>(&ctrl->status) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------------------
// block-wide scans / reductions (kBlock threads)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t warp_incl_scan64(uint64_t x, uint32_t lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(FULL_MASK, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    return x;
}

// Exclusive scan of x over the block; *total receives the block sum.
// s_tmp holds kWarps entries; callers __syncthreads() before reusing it.
__device__ __forceinline__ uint64_t block_excl_scan64(uint64_t x, uint64_t* s_tmp, uint64_t* total)
{
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t incl = warp_incl_scan64(x, lane);
    if (lane == 31) s_tmp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint64_t v = lane < (uint32_t)kWarps ? s_tmp[lane] : 0;
        v = warp_incl_scan64(v, lane);
        if (lane < (uint32_t)kWarps) s_tmp[lane] = v;
    }
    __syncthreads();
    *total = s_tmp[kWarps - 1];
    return (wid ? s_tmp[wid - 1] : 0) + incl - x;
}

__device__ __forceinline__ uint64_t block_reduce_add64(uint64_t x, uint64_t* s_tmp)
{
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL_MASK, x, o);
    __syncthreads();
    if (lane == 0) s_tmp[wid] = x;
    __syncthreads();
    uint64_t r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kWarps; ++i) r += s_tmp[i];
    return r;  // valid in thread 0
}

__device__ __forceinline__ uint64_t block_reduce_min64(uint64_t x, uint64_t* s_tmp)
{
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t y = __shfl_xor_sync(FULL_MASK, x, o);
        x = y < x ? y : x;
    }
    __syncthreads();
    if (lane == 0) s_tmp[wid] = x;
    __syncthreads();
    uint64_t r = kInf;
    if (threadIdx.x == 0)
        for (int i = 0; i < kWarps; ++i) r = s_tmp[i] < r ? s_tmp[i] : r;
    return r;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// ExtDist of rho-Stepping (Table 2; Sec. 6 "Threshold estimation"; App. B).
// Every block evaluates it redundantly from the same inputs (queue list and
// delta are stable between the previous barrier and the Extract), so no
// extra device-wide wait is needed.  Returns the same value in all threads.
// ---------------------------------------------------------------------------
__device__ uint64_t rho_extdist_block(const uint32_t* Q, uint32_t q, const uint64_t* dist, uint32_t n,
                                      uint64_t rho, uint64_t seed, uint64_t step, uint32_t dense_before,
                                      uint64_t* skeys, uint32_t cap, int* err)
{
    __shared__ uint64_t s_theta;
    uint64_t rho_eff = rho;
    if ((uint64_t)q * 20ull > (uint64_t)n && dense_before < 2) {
        rho_eff = rho / 10ull;
        if (rho_eff < 1) rho_eff = 1;
    }
    if ((uint64_t)q <= rho_eff) return kInf;  // extract every queued vertex
    const uint64_t lg = 63u - (uint32_t)__clzll((long long)((uint64_t)q + 1ull));
    uint64_t s = 10ull * (((uint64_t)q + rho_eff - 1ull) / rho_eff + 1ull + lg);
    if (s > kMaxSamples) s = kMaxSamples;
    uint32_t P = 1;
    while (P < s) P <<= 1;
    if (P > cap) {  // smem sized too small by the host: never expected
        if (threadIdx.x == 0) *err = 1;
        return kInf;
    }
    for (uint32_t j = threadIdx.x; j < P; j += blockDim.x) {
        uint64_t key = kInf;
        if (j < s) {
            const uint64_t h = splitmix64_at(seed, (step << 32) | j);
            const uint32_t pos = (uint32_t)__umul64hi(h, (uint64_t)q);
            key = ldcg64(&dist[ldcg32(&Q[pos])]);
        }
        skeys[j] = key;
    }
    __syncthreads();
    // bitonic sort of skeys[0..P), ascending
    for (uint32_t k = 2; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) {
                const uint32_t ixj = i ^ j;
                if (ixj > i) {
                    const uint64_t a = skeys[i], b = skeys[ixj];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) { skeys[i] = b; skeys[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
    uint64_t r = rho_eff * s / (uint64_t)q;
    if (r > s - 1) r = s - 1;
    if (threadIdx.x == 0) s_theta = skeys[r];
    __syncthreads();
    const uint64_t th = s_theta;
    __syncthreads();
    return th;
}

// ---------------------------------------------------------------------------
// Relaxation helpers
// ---------------------------------------------------------------------------
// WriteMin(delta[v], cand) (Sec. 2) after a plain pre-check; on success,
// Update(v): test-and-set v's queue bit; returns true when v must be
// appended to the next queue list (its bit was clear).
__device__ __forceinline__ bool relax_edge(uint64_t* dist, uint32_t* inq, uint32_t v, uint64_t cand,
                                           uint64_t dv, uint64_t& lmin, uint32_t& lupd)
{
    if (cand >= dv) return false;
    const uint64_t old = atomicMin(reinterpret_cast<unsigned long long*>(&dist[v]),
                                   (unsigned long long)cand);
    if (cand >= old) return false;
    ++lupd;
    lmin = cand < lmin ? cand : lmin;
    const uint32_t bit = 1u << (v & 31u);
    const uint32_t prev = atomicOr(&inq[v >> 5], bit);
    return (prev & bit) == 0;
}

// Warp-uniform: add the lanes' pushes to the warp's staging buffer.
__device__ __forceinline__ void stage_push(bool push, uint32_t v, uint32_t* stage, uint32_t& stc,
                                           uint32_t lane)
{
    const uint32_t b = __ballot_sync(FULL_MASK, push);
    if (push) stage[stc + __popc(b & ((1u << lane) - 1u))] = v;
    stc += __popc(b);
}

// Warp-uniform: move the staged ids to the next queue list (one atomic per flush).
__device__ __forceinline__ void stage_flush(uint32_t* stage, uint32_t& stc, uint32_t lane, Ctrl* ctrl,
                                            int nx, uint32_t* Qnext, uint32_t n)
{
    __syncwarp();
    if (stc == 0) return;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&ctrl->qsize[nx], stc);
    base = __shfl_sync(FULL_MASK, base, 0);
    if ((uint64_t)base + stc > (uint64_t)n) {
        if (lane == 0) set_status(ctrl, SSSP_ERR_INTERNAL);
    } else {
        for (uint32_t i = lane; i < stc; i += 32) Qnext[base + i] = stage[i];
    }
    __syncwarp();
    stc = 0;
}

// ---------------------------------------------------------------------------
// The persistent solve kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock, 2) solve_kernel(SolveParams p)
{
    extern __shared__ uint64_t s_dyn[];                // rho sample keys [p.sample_cap]
    __shared__ uint32_t s_stage[kWarps][kStage];       // per-warp re-queue staging
    __shared__ uint64_t s_tmp[kWarps];
    __shared__ uint32_t s_base[3];
    __shared__ int s_err;

    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
    const uint32_t n = p.n;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + tid;
    const uint32_t gwarp = blockIdx.x * kWarps + wid;
    const uint32_t nwarps = gridDim.x * kWarps;
    Ctrl* ctrl = p.ctrl;
    uint64_t* dist = p.dist;
    uint32_t* inq = p.inq;
    unsigned long long bar_target = 0;
    const uint64_t* __restrict__ off = p.off;
    const uint2* __restrict__ edges = p.edges;

    if (tid == 0) s_err = 0;
    const unsigned long long t_start = global_timer_ns();

    // ---- init: delta <- inf, delta[s] <- 0, Q.Update(s) (Algorithm 1) ----
    for (uint64_t i = gtid; i < n; i += gthreads) dist[i] = (i == p.source) ? 0ull : kInf;
    const uint32_t nwords = (n + 31u) >> 5;
    for (uint64_t i = gtid; i < nwords; i += gthreads)
        inq[i] = (i == (p.source >> 5)) ? (1u << (p.source & 31u)) : 0u;
    if (p.ext_count)
        for (uint64_t i = gtid; i < n; i += gthreads) p.ext_count[i] = 0;
    if (blockIdx.x == 0 && tid == 0) {
        p.qa[0] = p.source;
        ctrl->qsize[1] = 1;
        ctrl->qmin[0] = kInf;
        ctrl->qmin[1] = 0;
        ctrl->qmin[2] = kInf;
    }
    if (p.exit_block != 0 && blockIdx.x == p.exit_block - 1) return;  // fault-injection test
    if (!grid_sync(ctrl, bar_target, p.timeout_ns)) return;

    uint64_t delta_i = 1;          // Delta*-Stepping bucket index (Table 2)
    uint32_t dense_seen = 0;       // rho-Stepping: dense steps so far (Sec. 6)
    uint64_t prev_theta = 0;       // block 0: theta of the previous step, for the trace
    uint64_t prev_t = 0;           // block 0: start time of the previous step, for the trace
    unsigned long long t_queued = 0, t_ext = 0, t_edges = 0, t_upd = 0;

    uint64_t k = 1;
    for (;; ++k) {
        const int c = (int)(k % 3), nx = (int)((k + 1) % 3), pv = (int)((k + 2) % 3);
        const uint32_t* Qcur = (k & 1) ? p.qa : p.qb;
        uint32_t* Qnext = (k & 1) ? p.qb : p.qa;
        uint32_t q = ldcg32(&ctrl->qsize[c]);
        q = q < n ? q : n;  // a capacity fault is reported via status; never read past a list

        if (blockIdx.x == 0 && tid == 0) {
            // step k-1 is complete: fold its counters into the totals and
            // recycle its slot for Q_{k+2}.
            if (k > 1) {
                const uint32_t qq = ldcg32(&ctrl->qsize[pv]);
                const uint32_t ff = ldcg32(&ctrl->fcount[pv]);
                const uint64_t ee = ldcg64((const uint64_t*)&ctrl->fedges[pv]);
                const uint64_t uu = ldcg64((const uint64_t*)&ctrl->updates[pv]);
                t_queued += qq; t_ext += ff; t_edges += ee; t_upd += uu;
                if (p.trace && k - 2 < p.trace_cap) {
                    sssp_step_trace rec;
                    rec.theta = prev_theta; rec.queued = qq; rec.extracted = ff;
                    rec.edges = ee; rec.updates = uu; rec.t_ns = prev_t;
                    p.trace[k - 2] = rec;
                }
            }
            prev_t = global_timer_ns() - t_start;
            ctrl->qsize[pv] = 0; ctrl->fsmall[pv] = 0; ctrl->fchunk[pv] = 0; ctrl->fcount[pv] = 0;
            ctrl->fedges[pv] = 0; ctrl->updates[pv] = 0; ctrl->qmin[pv] = kInf;
        }
        if (q == 0) break;
        if (p.max_steps != 0 && k > p.max_steps) {
            if (blockIdx.x == 0 && tid == 0) set_status(ctrl, SSSP_ERR_INTERNAL);
            break;
        }
        // whole-solve time guard: block 0 records it; every block leaves at the
        // next barrier
        if (blockIdx.x == 0 && tid == 0 && global_timer_ns() - t_start > p.solve_timeout_ns)
            set_status(ctrl, SSSP_ERR_TIMEOUT);

        // ---------------- ExtDist ----------------
        uint64_t theta;
        if (p.algo == SSSP_BELLMAN_FORD) {
            theta = kInf;
        } else if (p.algo == SSSP_DELTA_STAR) {
            const uint64_t qmin = ldcg64((const uint64_t*)&ctrl->qmin[c]);
            uint64_t cur = delta_i;
            theta = sat_mul(cur, p.param);
            if (qmin > theta) {  // skip empty buckets
                cur = qmin / p.param + ((qmin % p.param) != 0);
                theta = sat_mul(cur, p.param);
            }
            delta_i = cur + 1;
        } else {
            theta = rho_extdist_block(Qcur, q, dist, n, p.param, p.seed, k, dense_seen, s_dyn,
                                      p.sample_cap, &s_err);
            if ((uint64_t)q * 20ull > (uint64_t)n) ++dense_seen;
            if (s_err) {
                if (tid == 0) set_status(ctrl, SSSP_ERR_INTERNAL);
            }
        }
        prev_theta = theta;

        // ---------------- Extract(theta) ----------------
        {
            uint64_t l_fcount = 0, l_fedges = 0, l_kmin = kInf;
            const uint64_t tile = (uint64_t)kBlock * kExtractItems;
            for (uint64_t base = (uint64_t)blockIdx.x * tile; base < q; base += (uint64_t)gridDim.x * tile) {
                uint32_t v[kExtractItems];
                uint64_t d[kExtractItems];
                uint64_t beg[kExtractItems];
                uint32_t nch[kExtractItems];
                uint8_t kind[kExtractItems];  // 0 none, 1 keep, 2 small, 3 chunked, 4 extracted w/o edges
#pragma unroll
                for (int j = 0; j < kExtractItems; ++j) {
                    const uint64_t idx = base + (uint64_t)j * kBlock + tid;
                    v[j] = idx < q ? ldcg32(&Qcur[idx]) : 0u;
                }
#pragma unroll
                for (int j = 0; j < kExtractItems; ++j) {
                    const uint64_t idx = base + (uint64_t)j * kBlock + tid;
                    d[j] = idx < q ? ldcg64(&dist[v[j]]) : kInf;
                }
                uint32_t nkeep = 0, nsmall = 0, nchunks = 0;
#pragma unroll
                for (int j = 0; j < kExtractItems; ++j) {
                    const uint64_t idx = base + (uint64_t)j * kBlock + tid;
                    kind[j] = 0; nch[j] = 0; beg[j] = 0;
                    if (idx < q) {
                        if (d[j] <= theta) {
                            atomicAnd(&inq[v[j] >> 5], ~(1u << (v[j] & 31u)));
                            const uint64_t b = __ldg(&off[v[j]]);
                            const uint64_t e = __ldg(&off[v[j] + 1]);
                            const uint64_t deg = e - b;
                            beg[j] = b;
                            l_fcount += 1;
                            l_fedges += deg;
                            if (p.ext_count) p.ext_count[v[j]] += 1u;
                            if (deg == 0) {
                                kind[j] = 4;
                            } else if (deg <= kSmallDeg) {
                                kind[j] = 2; ++nsmall;
                            } else {
                                kind[j] = 3;
                                nch[j] = (uint32_t)((e - 1) / kChunk - b / kChunk + 1);
                                nchunks += nch[j];
                            }
                        } else {
                            kind[j] = 1; ++nkeep;
                            l_kmin = d[j] < l_kmin ? d[j] : l_kmin;
                        }
                    }
                }
                // block scan of (keep, small, chunks) packed 16|16|32 bits
                const uint64_t packed = (uint64_t)nkeep | ((uint64_t)nsmall << 16) | ((uint64_t)nchunks << 32);
                uint64_t tot;
                const uint64_t ex = block_excl_scan64(packed, s_tmp, &tot);
                if (tid == 0) {
                    const uint32_t tk = (uint32_t)(tot & 0xFFFFu), ts = (uint32_t)((tot >> 16) & 0xFFFFu);
                    const uint32_t tc = (uint32_t)(tot >> 32);
                    s_base[0] = tk ? atomicAdd(&ctrl->qsize[nx], tk) : 0u;
                    s_base[1] = ts ? atomicAdd(&ctrl->fsmall[c], ts) : 0u;
                    s_base[2] = tc ? atomicAdd(&ctrl->fchunk[c], tc) : 0u;
                    if ((uint64_t)s_base[0] + tk > n || (uint64_t)s_base[1] + ts > n ||
                        (uint64_t)s_base[2] + tc > p.item_cap)
                        set_status(ctrl, SSSP_ERR_INTERNAL);
                }
                __syncthreads();
                uint32_t pk = s_base[0] + (uint32_t)(ex & 0xFFFFu);
                uint32_t ps = s_base[1] + (uint32_t)((ex >> 16) & 0xFFFFu);
                uint64_t pc = (uint64_t)s_base[2] + (ex >> 32);
#pragma unroll
                for (int j = 0; j < kExtractItems; ++j) {
                    if (kind[j] == 1) {
                        if (pk < n) Qnext[pk] = v[j];
                        ++pk;
                    } else if (kind[j] == 2) {
                        if (ps < n) p.fsmall[ps] = v[j];
                        ++ps;
                    } else if (kind[j] == 3) {
                        const uint32_t c0 = (uint32_t)(beg[j] / kChunk);
                        for (uint32_t t = 0; t < nch[j]; ++t, ++pc)
                            if (pc < p.item_cap) p.items[pc] = make_uint2(v[j], c0 + t);
                    }
                }
                __syncthreads();  // s_tmp / s_base reuse
            }
            const uint64_t bf = block_reduce_add64(l_fcount, s_tmp);
            if (tid == 0 && bf) atomicAdd(&ctrl->fcount[c], (unsigned int)bf);
            const uint64_t be = block_reduce_add64(l_fedges, s_tmp);
            if (tid == 0 && be) atomicAdd(&ctrl->fedges[c], (unsigned long long)be);
            if (p.algo == SSSP_DELTA_STAR) {
                const uint64_t bm = block_reduce_min64(l_kmin, s_tmp);
                if (tid == 0 && bm != kInf) atomicMin(&ctrl->qmin[nx], (unsigned long long)bm);
            }
        }
        if (!grid_sync(ctrl, bar_target, p.timeout_ns)) return;

        // ---------------- relax the out-edges of F ----------------
        {
            uint32_t fs = ldcg32(&ctrl->fsmall[c]);
            fs = fs < n ? fs : n;
            uint64_t fc = ldcg32(&ctrl->fchunk[c]);
            fc = fc < p.item_cap ? fc : p.item_cap;
            uint32_t* stage = s_stage[wid];
            uint32_t stc = 0;
            uint64_t lmin = kInf;
            uint32_t lupd = 0;

            // (a) low-degree vertices: 32 per warp, edges flattened across lanes
            const uint32_t ngroups = (fs + 31u) >> 5;
            for (uint32_t g = gwarp; g < ngroups; g += nwarps) {
                const uint32_t idx = g * 32u + lane;
                const bool valid = idx < fs;
                const uint32_t u = valid ? ldcg32(&p.fsmall[idx]) : 0u;
                const uint64_t b = valid ? __ldg(&off[u]) : 0ull;
                const uint32_t deg = valid ? (uint32_t)(__ldg(&off[u + 1]) - b) : 0u;
                const uint64_t du = valid ? ldcg64(&dist[u]) : 0ull;
                const uint32_t incl = (uint32_t)warp_incl_scan64(deg, lane);
                const uint32_t excl = incl - deg;
                const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
                uint32_t started = 0;
                const uint32_t lmask = lane == 31 ? FULL_MASK : ((2u << lane) - 1u);
                for (uint32_t r0 = 0; r0 < total; r0 += 128) {
                    uint64_t eidx[4], cdu[4];
                    bool ok[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const uint32_t rb = r0 + 32u * t;
                        const uint32_t contrib =
                            (deg > 0 && excl >= rb && excl < rb + 32u) ? (1u << (excl - rb)) : 0u;
                        const uint32_t starts = __reduce_or_sync(FULL_MASK, contrib);
                        const uint32_t e = rb + lane;
                        ok[t] = e < total;
                        int owner = (int)(started + __popc(starts & lmask)) - 1;
                        owner = owner < 0 ? 0 : owner;
                        started += __popc(starts);
                        const uint64_t ob = __shfl_sync(FULL_MASK, b, owner);
                        const uint32_t oe = __shfl_sync(FULL_MASK, excl, owner);
                        cdu[t] = __shfl_sync(FULL_MASK, du, owner);
                        eidx[t] = ob + (e - oe);
                    }
                    uint2 ed[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) ed[t] = ok[t] ? __ldcs(&edges[eidx[t]]) : make_uint2(0, 0);
                    uint64_t dv[4];
#pragma unroll
                    for (int t = 0; t < 4; ++t) dv[t] = ok[t] ? ldcg64(&dist[ed[t].x]) : 0ull;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        const bool push = ok[t] && relax_edge(dist, inq, ed[t].x, cdu[t] + ed[t].y, dv[t], lmin, lupd);
                        stage_push(push, ed[t].x, stage, stc, lane);
                    }
                    if (stc > (uint32_t)(kStage - 256)) stage_flush(stage, stc, lane, ctrl, nx, Qnext, n);
                }
            }

            // (b) higher-degree vertices: one warp per chunk item of <= kChunk edges,
            //     read as 16-byte pairs of packed edges
            const uint4* pairs = reinterpret_cast<const uint4*>(edges);
            for (uint64_t it = gwarp; it < fc; it += nwarps) {
                const uint2 item = __ldcg(&p.items[it]);
                const uint32_t u = item.x;
                const uint64_t b = __ldg(&off[u]);
                const uint64_t e = __ldg(&off[u + 1]);
                const uint64_t c0 = (uint64_t)item.y * kChunk;
                const uint64_t cs = b > c0 ? b : c0;
                const uint64_t ce = e < c0 + kChunk ? e : c0 + kChunk;
                const uint64_t du = ldcg64(&dist[u]);
                const uint64_t p0 = cs >> 1, p1 = (ce + 1) >> 1;
                // up to kChunk/2 = 128 pairs: two halves of 64, each with two
                // 16-byte loads per lane in flight
#pragma unroll 1
                for (uint64_t h0 = p0; h0 < p1; h0 += 64) {
                    uint4 pr[2];
                    bool oka[2], okb[2];
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const uint64_t P = h0 + 32u * t + lane;
                        const bool okp = P < p1;
                        pr[t] = okp ? __ldcs(&pairs[P]) : make_uint4(0, 0, 0, 0);
                        oka[t] = okp && (2 * P >= cs) && (2 * P < ce);
                        okb[t] = okp && (2 * P + 1 >= cs) && (2 * P + 1 < ce);
                    }
                    uint64_t dva[2], dvb[2];
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        dva[t] = oka[t] ? ldcg64(&dist[pr[t].x]) : 0ull;
                        dvb[t] = okb[t] ? ldcg64(&dist[pr[t].z]) : 0ull;
                    }
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const bool pa = oka[t] && relax_edge(dist, inq, pr[t].x, du + pr[t].y, dva[t], lmin, lupd);
                        stage_push(pa, pr[t].x, stage, stc, lane);
                        const bool pb = okb[t] && relax_edge(dist, inq, pr[t].z, du + pr[t].w, dvb[t], lmin, lupd);
                        stage_push(pb, pr[t].z, stage, stc, lane);
                    }
                }
                if (stc > (uint32_t)(kStage - 256)) stage_flush(stage, stc, lane, ctrl, nx, Qnext, n);
            }
            stage_flush(stage, stc, lane, ctrl, nx, Qnext, n);

            const uint64_t bu = block_reduce_add64(lupd, s_tmp);
            if (tid == 0 && bu) atomicAdd(&ctrl->updates[c], (unsigned long long)bu);
            if (p.algo == SSSP_DELTA_STAR) {
                const uint64_t bm = block_reduce_min64(lmin, s_tmp);
                if (tid == 0 && bm != kInf) atomicMin(&ctrl->qmin[nx], (unsigned long long)bm);
            }
        }
        if (!grid_sync(ctrl, bar_target, p.timeout_ns)) return;
    }

    if (blockIdx.x == 0 && tid == 0) {
        ctrl->steps = k - 1;
        ctrl->queued = t_queued;
        ctrl->extracted = t_ext;
        ctrl->edges = t_edges;
        ctrl->updates_total = t_upd;
        if (p.stats_out) {
            sssp_stats so;
            so.steps = k - 1; so.queued = t_queued; so.extracted = t_ext; so.edges = t_edges;
            so.updates = t_upd; so.status = *reinterpret_cast<volatile int*>(&ctrl->status); so.grid = 0;
            *p.stats_out = so;
        }
    }
}

const void* solve_kernel_ptr() { return reinterpret_cast<const void*>(&solve_kernel); }

// ---------------------------------------------------------------------------
// Graph upload: pack (target, weight) pairs into 8-byte edge records.
// ---------------------------------------------------------------------------
__global__ void pack_edges_kernel(const uint32_t* __restrict__ tgt, const uint32_t* __restrict__ w,
                                  uint2* __restrict__ edges, uint64_t m, uint64_t m_pad)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_pad; i += stride)
        edges[i] = i < m ? make_uint2(tgt[i], w[i]) : make_uint2(0u, 0u);
}

cudaError_t launch_pack_edges(const uint32_t* tgt, const uint32_t* w, uint2* edges, uint64_t m,
                              uint64_t m_pad, cudaStream_t st)
{
    uint64_t blocks = (m_pad + 255) / 256;
    if (blocks > 65535ull * 16) blocks = 65535ull * 16;
    if (blocks == 0) blocks = 1;
    pack_edges_kernel<<<(unsigned)blocks, 256, 0, st>>>(tgt, w, edges, m, m_pad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ExtDist alone (one block), for testing the threshold rule in isolation.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) rho_threshold_kernel(const uint32_t* queue, uint32_t q,
                                                               const uint64_t* dist, uint32_t n,
                                                               uint64_t rho, uint64_t seed, uint64_t step,
                                                               uint32_t dense_before, uint64_t* theta_out,
                                                               uint32_t* err_out, uint32_t cap)
{
    extern __shared__ uint64_t s_keys[];
    __shared__ int s_e;
    if (threadIdx.x == 0) s_e = 0;
    __syncthreads();
    const uint64_t th = rho_extdist_block(queue, q, dist, n, rho, seed, step, dense_before, s_keys, cap, &s_e);
    __syncthreads();
    if (threadIdx.x == 0) {
        *theta_out = th;
        *err_out = (uint32_t)s_e;
    }
}

uint32_t rho_sample_bound(uint32_t n, uint64_t rho)
{
    uint64_t r = rho / 10ull;
    if (r < 1) r = 1;
    uint64_t lg = 0;
    for (uint64_t x = (uint64_t)n + 1ull; x > 1; x >>= 1) ++lg;
    uint64_t s = 10ull * (((uint64_t)n + r - 1ull) / r + 1ull + lg);
    if (s > kMaxSamples) s = kMaxSamples;
    uint32_t P = 1;
    while (P < s) P <<= 1;
    return P;
}

cudaError_t launch_rho_threshold(const uint32_t* queue, uint32_t q, const uint64_t* dist, uint32_t n,
                                 uint64_t rho, uint64_t seed, uint64_t step, uint32_t dense_before,
                                 uint64_t* theta_out, uint32_t* err_out, cudaStream_t st)
{
    const uint32_t cap = kMaxSamples;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(rho_threshold_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)(cap * sizeof(uint64_t)));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    rho_threshold_kernel<<<1, kBlock, cap * sizeof(uint64_t), st>>>(queue, q, dist, n, rho, seed, step,
                                                                    dense_before, theta_out, err_out, cap);
    return cudaGetLastError();
}

}  // namespace sssp
