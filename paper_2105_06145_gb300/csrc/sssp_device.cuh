// sssp_device.cuh -- device helpers shared by the solve kernels of libsssp
// (single solve: sssp_kernels.cu; batched solves: sssp_batch.cu).
#pragma once

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

// Load of delta[v] for the relaxation pre-check.  kL1: through the SM's L1
// (ld.global.ca), for kernels that initialise delta once per launch: within
// such a launch delta only decreases after the init barrier (and L1 holds no
// line from before the launch), so a value served from a non-coherent L1 line
// can only be too high -- the pre-check then lets an extra atomicMin through,
// never skips a needed one.  Kernels that re-initialise distance arrays
// during the launch (the server's slots) must use the L2 load.
template <bool kL1>
__device__ __forceinline__ uint64_t ld_precheck(const uint64_t* p)
{
    if (kL1) return __ldca(reinterpret_cast<const unsigned long long*>(p));
    return __ldcg(reinterpret_cast<const unsigned long long*>(p));
}

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

__device__ __forceinline__ void set_status(int* status, int code) { atomicCAS(status, 0, code); }

// System-scope acquire / release accesses to host-mapped memory (the
// servers' command and completion records).
__device__ __forceinline__ unsigned int ld_acquire_sys_u32(const unsigned int* p)
{
    unsigned int v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_sys_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_sys_u32(unsigned int* p, unsigned int v)
{
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

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
static __device__ __noinline__ bool grid_sync(unsigned long long* bar, int* status, unsigned long long* target,
                                      uint64_t timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long tgt = *target + gridDim.x;
        *target = tgt;
        __threadfence();
        atomicAdd(bar, 1ull);
        int ok = 1;
        const unsigned long long t0 = global_timer_ns();
        unsigned int spins = 0;
        while (ld_acquire_u64(bar) < tgt) {
            if ((++spins & 31u) == 0) {
                if (*reinterpret_cast<volatile int*>(status) != 0) { ok = 0; break; }
                if (global_timer_ns() - t0 > timeout_ns) { set_status(status, SSSP_ERR_TIMEOUT); ok = 0; break; }
            }
        }
        __threadfence();
        // an error recorded before the barrier (timeout, capacity, step or time
        // guard) is visible to every block after it: all of them leave together
        if (ok && *reinterpret_cast<volatile int*>(status) != 0) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Variant for kernels whose every error path also raises kBarErr in the
// barrier word (raise_error): the error reaches waiting blocks through the
// word they spin on, so the wait needs no separate status load, and blocks
// waiting for a block that failed are released at once.
constexpr unsigned long long kBarErr = 1ull << 62;

__device__ __forceinline__ void raise_error(unsigned long long* bar, int* status, int code)
{
    atomicCAS(status, 0, code);
    atomicOr(bar, kBarErr);
}

static __device__ __noinline__ bool grid_sync_err(unsigned long long* bar, int* status, unsigned long long* target,
                                                  uint64_t timeout_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long tgt = *target + gridDim.x;
        *target = tgt;
        __threadfence();
        atomicAdd(bar, 1ull);
        int ok = 1;
        const unsigned long long t0 = global_timer_ns();
        unsigned int spins = 0;
        unsigned long long v;
        while ((v = ld_acquire_u64(bar)) < tgt) {
            if ((++spins & 31u) == 0 && global_timer_ns() - t0 > timeout_ns) {
                raise_error(bar, status, SSSP_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        if (v & kBarErr) ok = 0;
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
//
// Sample count s, rank r and the effective rho' of a step with q queued ids:
// rho' = max(1, rho/10) in the first `reduced` dense steps (20 q > n; the
// paper uses the first two), else rho; s = min(max_samples, 10 (ceil(q/rho')
// + 1 + floor(log2(q+1)))) with max_samples 4096 (1024 in warm-up steps);
// r = min(s-1, floor(rho' s / q)); theta is the r-th smallest (0-based) of the
// s sampled keys.  Returns false when q <= rho' (theta = +inf: extract every
// queued id).
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool rho_sample_plan(uint32_t q, uint32_t n, uint64_t rho, uint32_t dense_before,
                                                uint32_t reduced, uint32_t* s_out, uint32_t* r_out,
                                                uint32_t max_samples = kMaxSamples)
{
    uint64_t rho_eff = rho;
    if ((uint64_t)q * 20ull > (uint64_t)n && dense_before < reduced) {
        rho_eff = rho / 10ull;
        if (rho_eff < 1) rho_eff = 1;
    }
    if ((uint64_t)q <= rho_eff) return false;
    const uint64_t lg = 63u - (uint32_t)__clzll((long long)((uint64_t)q + 1ull));
    uint64_t s = 10ull * (((uint64_t)q + rho_eff - 1ull) / rho_eff + 1ull + lg);
    if (s > max_samples) s = max_samples;
    uint64_t r = rho_eff * s / (uint64_t)q;
    if (r > s - 1) r = s - 1;
    *s_out = (uint32_t)s;
    *r_out = (uint32_t)r;
    return true;
}

// Queue position of sample j of step `step`: splitmix64 output step*2^32 + j
// from state `seed`, reduced to [0, q) by multiply-high.
__device__ __forceinline__ uint32_t rho_sample_pos(uint64_t seed, uint64_t step, uint32_t j, uint32_t q)
{
    const uint64_t h = splitmix64_at(seed, (step << 32) | j);
    return (uint32_t)__umul64hi(h, (uint64_t)q);
}

// Block-wide: the r-th smallest (0-based) of the s keys, all threads get it.
// s <= blockDim: thread i holds key i in `x` (threads i >= s pass anything)
// and a bitonic network sorts the P = pow2(s) keys in registers -- shuffles
// for partner distances < 32, shared memory `xbuf` (blockDim keys) beyond.
// Larger s: the keys are in skeys[0..s) and are sorted there (P <= cap).
__device__ __forceinline__ uint64_t block_select(uint64_t x, uint32_t s, uint32_t r, uint64_t* skeys, uint32_t cap,
                                                 int* err)
{
    __shared__ uint64_t s_sel;
    const uint32_t i = threadIdx.x;
    uint32_t P = 1;
    while (P < s) P <<= 1;
    if (P <= blockDim.x) {
        x = i < s ? x : kInf;
        for (uint32_t k = 2; k <= P; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                uint64_t y;
                if (j >= 32) {
                    __syncthreads();
                    skeys[i] = x;
                    __syncthreads();
                    y = skeys[i ^ j];
                } else {
                    y = __shfl_xor_sync(FULL_MASK, x, j);
                }
                const bool up = (i & k) == 0, lower = (i & j) == 0;
                x = (lower == up) ? (y < x ? y : x) : (y < x ? x : y);
            }
        }
        if (i == r) s_sel = x;
    } else {
        if (P > cap) {  // shared memory sized too small by the host: never expected
            if (i == 0) { *err = 1; s_sel = kInf; }
        } else {
            for (uint32_t j = s + i; j < P; j += blockDim.x) skeys[j] = kInf;
            __syncthreads();
            for (uint32_t k = 2; k <= P; k <<= 1) {
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    for (uint32_t t = i; t < P; t += blockDim.x) {
                        const uint32_t tj = t ^ j;
                        if (tj > t) {
                            const uint64_t a = skeys[t], b = skeys[tj];
                            const bool up = (t & k) == 0;
                            if ((a > b) == up) { skeys[t] = b; skeys[tj] = a; }
                        }
                    }
                    __syncthreads();
                }
            }
            if (i == 0) s_sel = skeys[r];
        }
    }
    __syncthreads();
    const uint64_t th = s_sel;
    __syncthreads();
    return th;
}

// The whole ExtDist of rho-Stepping in one block (used by the threshold entry
// point; the solve kernel runs the same steps with its Extract loads in flight).
static __device__ __noinline__ uint64_t rho_extdist_block(const uint32_t* Q, uint32_t q, const uint64_t* dist, uint32_t n,
                                      uint64_t rho, uint64_t seed, uint64_t step, uint32_t dense_before,
                                      uint32_t reduced, uint64_t* skeys, uint32_t cap, int* err,
                                      uint32_t max_samples = kMaxSamples)
{
    uint32_t s, r;
    if (!rho_sample_plan(q, n, rho, dense_before, reduced, &s, &r, max_samples)) return kInf;  // extract every queued vertex
    uint64_t x = kInf;
    if (s <= blockDim.x) {
        if (threadIdx.x < s) x = ldcg64(&dist[ldcg32(&Q[rho_sample_pos(seed, step, threadIdx.x, q)])]);
    } else {
        for (uint32_t j = threadIdx.x; j < s; j += blockDim.x)
            skeys[j] = ldcg64(&dist[ldcg32(&Q[rho_sample_pos(seed, step, j, q)])]);
        __syncthreads();
    }
    return block_select(x, s, r, skeys, cap, err);
}

// ---------------------------------------------------------------------------
// Relaxation helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 make_rec(uint64_t start, uint64_t len, uint64_t du)
{
    const uint64_t a = start | (len << 40);
    return make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)du, (uint32_t)(du >> 32));
}
__device__ __forceinline__ uint64_t rec_start(uint4 r) { return ((uint64_t)r.x | ((uint64_t)(r.y & 0xFFu) << 32)); }
__device__ __forceinline__ uint32_t rec_len(uint4 r) { return r.y >> 8; }
__device__ __forceinline__ uint64_t rec_du(uint4 r) { return (uint64_t)r.z | ((uint64_t)r.w << 32); }

// Warp-uniform: add the lanes' pushes to the warp's staging buffer.
__device__ __forceinline__ void stage_push(bool push, uint32_t v, uint32_t* stage, uint32_t& stc,
                                           uint32_t lane)
{
    const uint32_t b = __ballot_sync(FULL_MASK, push);
    if (push) stage[stc + __popc(b & ((1u << lane) - 1u))] = v;
    stc += __popc(b);
}

// Warp-uniform: the re-check after a fused step (SSSP_SOLVE_FUSED).  Lane
// entry j is a vertex u[j] the block extracted in that step and the distance
// du[j] it was relaxed with (kInf: no entry).  Where delta[u] has dropped below
// du since, u is queued again (Update: test-and-set of its queue bit, staged
// when the bit was clear).
template <int P>
__device__ __forceinline__ void requeue_dropped(const uint32_t (&u)[P], const uint64_t (&du)[P], const uint64_t* dist,
                                                uint32_t* inq, uint32_t* stage, uint32_t& stc, uint32_t lane,
                                                uint64_t& lmin)
{
    uint64_t dv[P];
#pragma unroll
    for (int j = 0; j < P; ++j) dv[j] = du[j] != kInf ? ldcg64(&dist[u[j]]) : kInf;
#pragma unroll
    for (int j = 0; j < P; ++j) {
        bool push = false;
        if (dv[j] < du[j]) {
            lmin = dv[j] < lmin ? dv[j] : lmin;
            const uint32_t prev = atomicOr(&inq[u[j] >> 5], 1u << (u[j] & 31u));
            push = (prev & (1u << (u[j] & 31u))) == 0;
        }
        stage_push(push, u[j], stage, stc, lane);
    }
}

// Warp-uniform: the second half of a batch of (up to) 4 relaxations per lane,
// given the pre-check values dv[t] = delta[v[t]]:
//   for every candidate with cand < delta[v]: WriteMin(delta[v], cand)
//   (Sec. 2) as a fire-and-forget atomic minimum, then Update(v): the
//   test-and-set of v's queue bit (all test-and-sets of the batch in flight);
//   the ids whose bit was clear are staged for the next queue list.
// A candidate that passes the pre-check but loses the race to a smaller one
// still marks v: the winner lowered delta[v] in this same phase and queues v
// too, so the queued set is exactly the set whose distance dropped, and the
// bit keeps each vertex at most once in the queue.
__device__ __forceinline__ void relax_apply4(uint64_t* dist, uint32_t* inq, const uint32_t (&v)[4],
                                             const uint64_t (&cand)[4], const uint64_t (&dv)[4],
                                             const bool (&ok)[4], uint32_t* stage, uint32_t& stc,
                                             uint32_t lane, uint64_t& lmin, uint32_t& lupd)
{
    uint32_t prev[4];
    uint32_t pass = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        prev[t] = ~0u;
        if (ok[t] && cand[t] < dv[t]) {
            atomicMin(reinterpret_cast<unsigned long long*>(&dist[v[t]]), (unsigned long long)cand[t]);
            ++lupd;
            lmin = cand[t] < lmin ? cand[t] : lmin;
            prev[t] = atomicOr(&inq[v[t] >> 5], 1u << (v[t] & 31u));
            pass |= 1u << t;
        }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const bool push = ((pass >> t) & 1u) && (prev[t] & (1u << (v[t] & 31u))) == 0;
        stage_push(push, v[t], stage, stc, lane);
    }
}

// Warp-uniform: one batch of (up to) 4 relaxations per lane (4 gathers of
// delta[v] in flight, then relax_apply4).
template <bool kL1 = false>
__device__ __forceinline__ void relax_batch4(uint64_t* dist, uint32_t* inq, const uint32_t (&v)[4],
                                             const uint64_t (&cand)[4], const bool (&ok)[4],
                                             uint32_t* stage, uint32_t& stc, uint32_t lane,
                                             uint64_t& lmin, uint32_t& lupd)
{
    uint64_t dv[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) dv[t] = ok[t] ? ld_precheck<kL1>(&dist[v[t]]) : 0ull;
    relax_apply4(dist, inq, v, cand, dv, ok, stage, stc, lane, lmin, lupd);
}

// Warp-uniform: move the staged ids to the next queue list (one atomic per flush).
__device__ __forceinline__ void stage_flush(uint32_t* stage, uint32_t& stc, uint32_t lane, unsigned int* qsize,
                                            int* status, uint32_t* Qnext, uint32_t cap)
{
    __syncwarp();
    if (stc == 0) return;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(qsize, stc);
    base = __shfl_sync(FULL_MASK, base, 0);
    if ((uint64_t)base + stc > (uint64_t)cap) {
        if (lane == 0) set_status(status, SSSP_ERR_INTERNAL);
    } else {
        for (uint32_t i = lane; i < stc; i += 32) Qnext[base + i] = stage[i];
    }
    __syncwarp();
    stc = 0;
}

// Warp-uniform: relax the edges of one chunk record (at most 2^kChunkLog2Max
// edges of vertex u, within one aligned block of the edge array whose length
// is even), read as 16-byte pairs of packed edges.  With kPull (bidirectional relaxation for undirected
// graphs, Sec. 6): the delta[v] values gathered for the pre-check first relax
// u itself -- WriteMin(delta[u], min over the chunk of delta[v] + w), with the
// usual Update(u) -- and the improved delta[u] is then pushed to the chunk's
// neighbours.
// Each 64-pair round stages at most 129 ids (128 targets and u itself), so the
// warp's staging buffer is flushed to the next queue list (qsize, Qnext of
// capacity qcap) before a round that might not fit.
template <bool kPull, bool kL1 = false>
__device__ __forceinline__ void relax_chunk(uint4 rec, uint64_t du, const uint4* __restrict__ pairs,
                                            uint64_t* dist, uint32_t* inq, uint32_t* stage, uint32_t& stc,
                                            uint32_t lane, uint64_t& lmin, uint32_t& lupd, unsigned int* qsize,
                                            int* status, uint32_t* Qnext, uint32_t qcap)
{
    const uint64_t cs = rec_start(rec), ce = cs + rec_len(rec);
    const uint64_t p0 = cs >> 1, p1 = (ce + 1) >> 1;
#pragma unroll 1
    for (uint32_t h = 0; p0 + h < p1; h += 64) {  // warp-uniform
        if (stc > (uint32_t)kStage - 129u) stage_flush(stage, stc, lane, qsize, status, Qnext, qcap);
        uint32_t vv[4], ww[4];
        bool ok[4];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const uint64_t P = p0 + h + 32u * t + lane;
            const bool okp = P < p1;
            const uint4 pr = okp ? __ldcs(&pairs[P]) : make_uint4(0, 0, 0, 0);
            vv[2 * t] = pr.x; ww[2 * t] = pr.y; ok[2 * t] = okp && 2 * P >= cs;       // 2P < ce when P < p1
            vv[2 * t + 1] = pr.z; ww[2 * t + 1] = pr.w; ok[2 * t + 1] = okp && 2 * P + 1 < ce;  // 2P+1 >= cs when P >= p0
        }
        uint64_t dv[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) dv[t] = ok[t] ? ld_precheck<kL1>(&dist[vv[t]]) : 0ull;
        if (kPull) {
            uint64_t pull = kInf;
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (ok[t] && dv[t] != kInf && dv[t] + ww[t] < pull) pull = dv[t] + ww[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const uint64_t y = __shfl_xor_sync(FULL_MASK, pull, o);
                pull = y < pull ? y : pull;
            }
            bool push_u = false;
            if (pull < du) {  // warp-uniform
                du = pull;
                if (lane == 0) {
                    const uint32_t u = rec.z;
                    atomicMin(reinterpret_cast<unsigned long long*>(&dist[u]), (unsigned long long)pull);
                    ++lupd;
                    lmin = pull < lmin ? pull : lmin;
                    const uint32_t prev = atomicOr(&inq[u >> 5], 1u << (u & 31u));
                    push_u = (prev & (1u << (u & 31u))) == 0;
                }
            }
            stage_push(push_u, rec.z, stage, stc, lane);
        }
        uint64_t cand[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) cand[t] = du + ww[t];
        relax_apply4(dist, inq, vv, cand, dv, ok, stage, stc, lane, lmin, lupd);
    }
}

// Warp-uniform: relax the out-edges of up to 32 vertices at once, one per lane
// (lane j: first edge b_j, degree deg_j -- 0 for none -- and distance du_j),
// with the edges of all of them spread over the lanes 32 at a time.  The
// lanes with deg > 0 are first packed to the front so that the k-th edge run
// belongs to lane k.  When allow_flush, staged ids are flushed whenever fewer
// than 256 staging slots are left; otherwise the caller guarantees room for
// every push (at most the total degree).
template <bool kL1 = false>
__device__ __forceinline__ void relax_flat(uint64_t b, uint32_t deg, uint64_t du, const uint2* __restrict__ edges,
                                           uint64_t* dist, uint32_t* inq, uint32_t* stage, uint32_t& stc,
                                           uint32_t lane, uint64_t& lmin, uint32_t& lupd, bool allow_flush,
                                           unsigned int* qsize, int* status, uint32_t* Qnext, uint32_t qcap)
{
    const uint32_t active = __ballot_sync(FULL_MASK, deg > 0);
    if (active == 0) return;
    if ((active & (active + 1u)) != 0) {  // the active lanes are not a prefix: pack them to the front
        const uint32_t cnt = __popc(active);
        uint32_t rest = active;  // position of the lane-th set bit of active
        for (uint32_t i = 0; i < lane && i < cnt; ++i) rest &= rest - 1u;
        const int src = lane < cnt ? __ffs(rest) - 1 : (int)lane;
        const uint64_t b2 = __shfl_sync(FULL_MASK, b, src);
        const uint32_t d2 = __shfl_sync(FULL_MASK, deg, src);
        const uint64_t u2 = __shfl_sync(FULL_MASK, du, src);
        b = lane < cnt ? b2 : 0ull;
        deg = lane < cnt ? d2 : 0u;
        du = lane < cnt ? u2 : 0ull;
    }
    const uint32_t lmask = lane == 31 ? FULL_MASK : ((2u << lane) - 1u);
    const uint32_t incl = (uint32_t)warp_incl_scan64(deg, lane);
    const uint32_t excl = incl - deg;
    const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
    uint32_t started = 0;
    for (uint32_t r0 = 0; r0 < total; r0 += 32 * kSmallRounds) {
        uint64_t eidx[kSmallRounds], cdu[kSmallRounds];
        bool ok[kSmallRounds];
#pragma unroll
        for (int t = 0; t < kSmallRounds; ++t) {
            const uint32_t rb = r0 + 32u * t;
            const uint32_t contrib = (deg > 0 && excl >= rb && excl < rb + 32u) ? (1u << (excl - rb)) : 0u;
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
        uint32_t vv[kSmallRounds];
        uint64_t cand[kSmallRounds];
#pragma unroll
        for (int t = 0; t < kSmallRounds; ++t) {
            const uint2 ed = ok[t] ? __ldcs(&edges[eidx[t]]) : make_uint2(0, 0);
            vv[t] = ed.x;
            cand[t] = cdu[t] + ed.y;
        }
        relax_batch4<kL1>(dist, inq, vv, cand, ok, stage, stc, lane, lmin, lupd);
        if (allow_flush && stc > (uint32_t)(kStage - 256)) stage_flush(stage, stc, lane, qsize, status, Qnext, qcap);
    }
}

// Warp-uniform: move the first `done` staged ids to the next queue list and
// shift the rest of the staging buffer down.
__device__ __forceinline__ void stage_flush_prefix(uint32_t* stage, uint32_t& stc, uint32_t done, uint32_t lane,
                                                   unsigned int* qsize, int* status, uint32_t* Qnext, uint32_t cap)
{
    __syncwarp();
    if (done == 0) return;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(qsize, done);
    base = __shfl_sync(FULL_MASK, base, 0);
    if ((uint64_t)base + done > (uint64_t)cap) {
        if (lane == 0) set_status(status, SSSP_ERR_INTERNAL);
    } else {
        for (uint32_t i = lane; i < done; i += 32) Qnext[base + i] = stage[i];
    }
    __syncwarp();
    for (uint32_t i0 = 0; i0 + done < stc; i0 += 32) {
        const uint32_t i = i0 + lane;
        const uint32_t x = (i + done < stc) ? stage[i + done] : 0u;
        __syncwarp();
        if (i + done < stc) stage[i] = x;
        __syncwarp();
    }
    stc -= done;
}

// Block-wide reduction of two sums and a minimum; results valid in thread 0.
__device__ __forceinline__ void block_reduce_2add_min(uint64_t& a, uint64_t& b, uint64_t& mn, uint64_t* s_tmp)
{
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(FULL_MASK, a, o);
        b += __shfl_xor_sync(FULL_MASK, b, o);
        const uint64_t y = __shfl_xor_sync(FULL_MASK, mn, o);
        mn = y < mn ? y : mn;
    }
    __syncthreads();
    if (lane == 0) { s_tmp[wid] = a; s_tmp[kWarps + wid] = b; s_tmp[2 * kWarps + wid] = mn; }
    __syncthreads();
    if (wid == 0) {
        a = lane < (uint32_t)kWarps ? s_tmp[lane] : 0;
        b = lane < (uint32_t)kWarps ? s_tmp[kWarps + lane] : 0;
        mn = lane < (uint32_t)kWarps ? s_tmp[2 * kWarps + lane] : kInf;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(FULL_MASK, a, o);
            b += __shfl_xor_sync(FULL_MASK, b, o);
            const uint64_t y = __shfl_xor_sync(FULL_MASK, mn, o);
            mn = y < mn ? y : mn;
        }
    }
}

// Warp-wide reduction of four sums and two minima (every lane gets the results).
__device__ __forceinline__ void warp_reduce_4add_2min(uint64_t (&a)[4], uint64_t (&mn)[2])
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int t = 0; t < 4; ++t) a[t] += __shfl_xor_sync(FULL_MASK, a[t], o);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const uint64_t y = __shfl_xor_sync(FULL_MASK, mn[t], o);
            mn[t] = y < mn[t] ? y : mn[t];
        }
    }
}

// ---------------------------------------------------------------------------
// Local relaxation of super-sparse steps (Sec. 6, local BFS).
//
// The warp's staging buffer is its local frontier: entries [0, lq) have been
// looked at, [lq, stc) wait.  Up to 32 waiting vertices at a time, a vertex
// whose distance is still <= theta and whose out-degree is 1..kSmallDeg has its
// out-edges relaxed at once (WriteMin and Update as in the main relaxation);
// the ids that queues are appended behind and are looked at in turn.  Every id
// stays staged and so reaches Q_next: a vertex relaxed here is extracted again
// in a later step (a vertex this step would have extracted next).  With lrel
// (one entry per vertex), the distance a vertex was relaxed with here is
// recorded, so that its later extraction can skip the edges when the distance
// has not changed since (relaxing them again with the same value cannot lower
// any target).  Stops after `budget` relaxed vertices, or when the frontier is
// exhausted.  Returns the edges relaxed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t local_relax(uint64_t theta, uint32_t budget, const uint64_t* __restrict__ off,
                                                const uint2* __restrict__ edges, uint64_t* dist, uint32_t* inq,
                                                uint32_t* stage, uint32_t& stc, uint32_t lane, uint64_t& lmin,
                                                uint32_t& lupd, unsigned int* qsize, int* status, uint32_t* Qnext,
                                                uint32_t n, uint64_t* lrel = nullptr)
{
    uint32_t lq = 0, done = 0;
    uint64_t scanned = 0;
    while (lq < stc && done < budget) {  // warp-uniform
        if (stc + 256u > (uint32_t)kStage) {
            // make room: the looked-at prefix goes to the next queue list
            stage_flush_prefix(stage, stc, lq, lane, qsize, status, Qnext, n);
            lq = 0;
            if (stc + (uint32_t)kSmallDeg > (uint32_t)kStage) break;
        }
        __syncwarp();
        uint32_t cnt = stc - lq;
        cnt = cnt < 32u ? cnt : 32u;
        uint64_t b = 0, du = 0;
        uint32_t deg = 0, x = 0;
        if (lane < cnt) {
            // the distance and the edge range are loaded together (the graph
            // is read-only), so a round waits for one load, not two in a row
            x = stage[lq + lane];
            du = ldcg64(&dist[x]);
            const uint64_t bx = __ldg(&off[x]), ex = __ldg(&off[x + 1]);
            if (du <= theta) {
                b = bx;
                const uint64_t d = ex - bx;
                deg = d <= (uint64_t)kSmallDeg ? (uint32_t)d : 0u;
            }
        }
        // take the lanes whose edges fit in the staging room left (a prefix,
        // never empty: the room is >= kSmallDeg)
        const uint32_t room = (uint32_t)kStage - stc;
        const uint32_t incl = (uint32_t)warp_incl_scan64(deg, lane);
        const uint32_t take = __popc(__ballot_sync(FULL_MASK, lane < cnt && incl <= room));
        if (lane >= take) deg = 0;
        if (lrel && deg > 0) lrel[x] = du;
        done += __popc(__ballot_sync(FULL_MASK, deg > 0));
        scanned += __shfl_sync(FULL_MASK, incl, take - 1);
        lq += take;
        relax_flat(b, deg, du, edges, dist, inq, stage, stc, lane, lmin, lupd, false, qsize, status, Qnext, n);
    }
    return lane == 0 ? scanned : 0;
}


}  // namespace sssp
