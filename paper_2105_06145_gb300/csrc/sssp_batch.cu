// sssp_batch.cu -- batched solves: k independent stepping-SSSP instances
// (Algorithm 1 with the ExtDist of Table 2, one LaB-PQ each) in one
// persistent cooperative launch.
//
// Each instance has its own graph pointers (one shared graph for
// sssp_solve_sources, one graph per instance for sssp_solve_multi), source,
// parameter, distance array, queue bitmap and lists, and its own threshold.
// All instances advance through the steps together; per step:
//   phase T  per-instance bookkeeping and theta_i (instances spread over blocks)
//   ---- grid barrier
//   phase E  Extract(theta_i) for every instance, work spread over all blocks
//            in tiles that each lie within one instance
//   ---- grid barrier (Extract is not concurrent with Update, Sec. 3.1)
//   phase R  relaxation of every instance's extracted vertices, work spread
//            over all warps
//   ---- grid barrier
// An instance whose queue is empty simply has no work.  The fixed per-step
// costs (barriers, phase latencies) are paid once for all instances.

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>
#include <new>

#include <cuda_runtime.h>

#include "sssp_internal.h"
#include "sssp_device.cuh"

namespace sssp {

// Per-instance step state (device; zeroed by the host before each launch).
// Ring slots as in the single solve: slot k%3 holds |Q_k| / min_Q delta and
// the Extract output of step k.
struct InstCtrl {
    unsigned int qsize[3], fsmall[3], fchunk[3], fcount[3];
    unsigned long long qmin[3], fedges[3], updates[3];
    unsigned long long umin[3];    // smallest distance written by a step's relaxation (slot of its next queue)
    unsigned long long theta;      // theta of the current step
    unsigned long long delta_i;    // Delta*-Stepping bucket index
    unsigned int dense_seen;       // rho-Stepping: dense steps so far
    unsigned int last_step;        // steps the instance took (set when its queue empties)
    unsigned long long queued, extracted, edges, updates_total;
    unsigned long long admit_step; // global step at which the instance's first queue is read
    unsigned int running;          // the instance takes part in the steps
    unsigned int seq;              // serving: sequence number of the admitted query
    unsigned long long t_admit_ns; // serving: device time of admission
    unsigned long long ticket;     // serving: ticket of the admitted query
};

// Per-instance pointers and sizes (device, read-only during the launch).
struct InstDesc {
    const uint64_t* off;
    const uint2* edges;
    uint64_t* dist;
    uint32_t* inq;
    uint32_t* qa;
    uint32_t* qb;
    uint4* fsmall;
    uint4* items;
    uint64_t fsmall_cap;
    uint64_t item_cap;
    uint32_t n;
    uint32_t source;
    uint64_t param;
    uint64_t seed;
    uint32_t bidir;          // bidirectional relaxation of chunk records (symmetric graph)
    uint32_t local_budget;   // local relaxation of super-sparse steps (0 = off)
    uint32_t rho_reduced;    // rho-Stepping: dense steps that use rho/10 (Sec. 6)
    uint32_t pad;
};

struct BatchCtrl {
    unsigned long long bar;
    int status;
    unsigned int pad;
    unsigned long long steps;
};

struct BatchParams {
    InstDesc* inst;
    InstCtrl* ictrl;
    BatchCtrl* ctrl;
    uint32_t k;
    int algo;
    uint64_t timeout_ns;
    uint64_t solve_timeout_ns;
    uint32_t sample_cap;
};

// Exclusive prefix sums of s_arr[0..k) in place (k <= kMaxBatch); returns the
// total in every thread.  Uses s_tmp[0..kWarps).
__device__ __forceinline__ uint64_t block_prefix_inplace(uint32_t* s_arr, uint32_t k, uint64_t* s_tmp)
{
    uint64_t carry = 0;
    for (uint32_t base = 0; base < k; base += kBlock) {
        const uint32_t i = base + threadIdx.x;
        const uint64_t x = i < k ? s_arr[i] : 0u;
        uint64_t tot;
        const uint64_t ex = block_excl_scan64(x, s_tmp, &tot);
        if (i < k) s_arr[i] = (uint32_t)(carry + ex);
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) s_arr[k] = (uint32_t)carry;
    __syncthreads();
    return carry;
}

// Largest i with s_pre[i] <= x (s_pre non-decreasing, s_pre[0] = 0).
__device__ __forceinline__ uint32_t find_segment(const uint32_t* s_pre, uint32_t k, uint64_t x)
{
    uint32_t lo = 0, hi = k;  // answer in [lo, hi)
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)s_pre[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Shared memory of the batched kernels.
struct BatchSmem {
    uint32_t pre0[kMaxBatch + 1];
    uint32_t pre1[kMaxBatch + 1];
    uint64_t tmp[3 * kWarps];
    uint32_t base[3];
    unsigned long long bar_target;
    unsigned long long t_start;
    int err;
    int flag;
};

// Init of instance i's state for a solve whose first queue is read at global
// step k0: delta <- inf, delta[s] <- 0, Q = {s} (Algorithm 1).  The distance
// fill is grid-strided; the rest is done by one thread.
__device__ __forceinline__ void init_instance_fill(const InstDesc& d, uint64_t gtid, uint64_t gthreads)
{
    for (uint64_t v = gtid; v < d.n; v += gthreads) d.dist[v] = (v == d.source) ? 0ull : kInf;
    const uint32_t nwords = (d.n + 31u) >> 5;
    for (uint64_t w = gtid; w < nwords; w += gthreads)
        d.inq[w] = (w == (d.source >> 5)) ? (1u << (d.source & 31u)) : 0u;
}
__device__ __forceinline__ void init_instance_ctrl(const InstDesc& d, InstCtrl* C, uint64_t k0)
{
    ((k0 & 1) ? d.qa : d.qb)[0] = d.source;
    for (int r = 0; r < 3; ++r) {
        C->qsize[r] = 0; C->fsmall[r] = 0; C->fchunk[r] = 0; C->fcount[r] = 0;
        C->qmin[r] = kInf; C->fedges[r] = 0; C->updates[r] = 0; C->umin[r] = kInf;
    }
    C->qsize[k0 % 3] = 1;
    C->qmin[k0 % 3] = 0;
    C->delta_i = 1;
    C->dense_seen = 0;
    C->last_step = 0;
    C->queued = 0; C->extracted = 0; C->edges = 0; C->updates_total = 0;
    C->admit_step = k0;
    C->running = 1;
}

// Phase T: bookkeeping and theta_i for the running instances (instances spread
// over blocks).
__device__ void phase_T(const BatchParams& p, uint64_t k, BatchSmem& S, uint64_t* s_keys)
{
    const uint32_t tid = threadIdx.x;
    const int c = (int)(k % 3), pv = (int)((k + 2) % 3);
    for (uint32_t i = blockIdx.x; i < p.k; i += gridDim.x) {
        InstCtrl* C = &p.ictrl[i];
        const InstDesc& D = p.inst[i];
        if (!ldcg32(&C->running)) continue;  // block-uniform
        uint32_t q = ldcg32(&C->qsize[c]);
        q = q < D.n ? q : D.n;
        if (tid == 0) {
            if (k > ldcg64((const uint64_t*)&C->admit_step)) {
                C->queued += ldcg32(&C->qsize[pv]);
                C->extracted += ldcg32(&C->fcount[pv]);
                C->edges += ldcg64((const uint64_t*)&C->fedges[pv]);
                C->updates_total += ldcg64((const uint64_t*)&C->updates[pv]);
            }
            if (q == 0 && C->last_step == 0) C->last_step = (unsigned)(k - C->admit_step);
            C->qsize[pv] = 0; C->fsmall[pv] = 0; C->fchunk[pv] = 0; C->fcount[pv] = 0;
            C->fedges[pv] = 0; C->updates[pv] = 0; C->qmin[pv] = kInf; C->umin[pv] = kInf;
        }
        if (q == 0) { __syncthreads(); continue; }  // block-uniform
        uint64_t theta;
        if (p.algo == SSSP_BELLMAN_FORD) {
            theta = kInf;
        } else if (p.algo == SSSP_DELTA_STAR || p.algo == SSSP_DELTA) {
            const uint64_t qmin = ldcg64((const uint64_t*)&C->qmin[c]);
            uint64_t cur = ldcg64((const uint64_t*)&C->delta_i);
            if (p.algo == SSSP_DELTA && k > ldcg64((const uint64_t*)&C->admit_step)) {
                // FinishCheck: advance unless the previous step wrote below its threshold
                const uint64_t umin = ldcg64((const uint64_t*)&C->umin[c]);
                if (!(umin < ldcg64((const uint64_t*)&C->theta))) cur += 1;
            }
            theta = sat_mul(cur, D.param);
            if (qmin > theta) {
                cur = qmin / D.param + ((qmin % D.param) != 0);
                theta = sat_mul(cur, D.param);
            }
            __syncthreads();
            if (tid == 0) C->delta_i = p.algo == SSSP_DELTA_STAR ? cur + 1 : cur;
        } else if (p.algo == SSSP_DIJKSTRA) {
            theta = ldcg64((const uint64_t*)&C->qmin[c]);
        } else {
            const uint32_t* Qcur = (k & 1) ? D.qa : D.qb;
            const uint32_t dense_seen = ldcg32(&C->dense_seen);
            const uint64_t lstep = k - ldcg64((const uint64_t*)&C->admit_step) + 1;  // the instance's own step
            theta = rho_extdist_block(Qcur, q, D.dist, D.n, D.param, D.seed, lstep, dense_seen, D.rho_reduced,
                                      s_keys, p.sample_cap, &S.err);
            if (tid == 0 && (uint64_t)q * 20ull > (uint64_t)D.n) C->dense_seen = dense_seen + 1;
        }
        if (tid == 0) C->theta = theta;
        __syncthreads();
    }
}

// Phase E: Extract(theta_i) of every running instance, in tiles that each lie
// within one instance.  Returns false (in every block) when no instance has
// queued vertices.
__device__ bool phase_E(const BatchParams& p, uint64_t k, BatchSmem& S)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const int c = (int)(k % 3), nx = (int)((k + 1) % 3);
    const uint32_t K = p.k;
    int* status = &p.ctrl->status;
    const uint32_t tileq = (uint32_t)kBlock * kExtractItems;
    for (uint32_t i = tid; i < K; i += kBlock) {
        uint32_t q = ldcg32(&p.ictrl[i].running) ? ldcg32(&p.ictrl[i].qsize[c]) : 0u;
        const uint32_t n_i = p.inst[i].n;
        q = q < n_i ? q : n_i;
        S.pre0[i] = (q + tileq - 1) / tileq;  // tiles of instance i
    }
    __syncthreads();
    const uint64_t ntiles = block_prefix_inplace(S.pre0, K, S.tmp);
    if (ntiles == 0) return false;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint32_t i = find_segment(S.pre0, K, t);
        const InstDesc& D = p.inst[i];
        InstCtrl* C = &p.ictrl[i];
        const uint32_t n = D.n;
        uint32_t q = ldcg32(&C->qsize[c]);
        q = q < n ? q : n;
        const uint64_t theta = ldcg64((const uint64_t*)&C->theta);
        const uint32_t* Qcur = (k & 1) ? D.qa : D.qb;
        uint32_t* Qnext = (k & 1) ? D.qb : D.qa;
        const uint64_t base = (t - S.pre0[i]) * (uint64_t)tileq;
        uint32_t v[kExtractItems];
        uint64_t d[kExtractItems];
        uint32_t kind[kExtractItems];  // 0 none, 1 keep, 2 small, 3 chunked, 4 extracted w/o edges
#pragma unroll
        for (int j = 0; j < kExtractItems; ++j) {
            const uint64_t idx = base + (uint64_t)j * kBlock + tid;
            v[j] = idx < q ? ldcg32(&Qcur[idx]) : 0u;
        }
#pragma unroll
        for (int j = 0; j < kExtractItems; ++j) {
            const uint64_t idx = base + (uint64_t)j * kBlock + tid;
            d[j] = idx < q ? ldcg64(&D.dist[v[j]]) : kInf;
        }
        uint32_t nkeep = 0, nsmall = 0, nchunks = 0;
        uint64_t l_fcount = 0, l_fedges = 0, l_kmin = kInf;
#pragma unroll
        for (int j = 0; j < kExtractItems; ++j) {
            const uint64_t idx = base + (uint64_t)j * kBlock + tid;
            kind[j] = 0;
            if (idx < q) {
                if (d[j] <= theta) {
                    atomicAnd(&D.inq[v[j] >> 5], ~(1u << (v[j] & 31u)));
                    const uint64_t b = __ldg(&D.off[v[j]]);
                    const uint64_t e = __ldg(&D.off[v[j] + 1]);
                    const uint64_t deg = e - b;
                    l_fcount += 1;
                    l_fedges += deg;
                    if (deg == 0) {
                        kind[j] = 4;
                    } else if (deg <= kSmallDeg) {
                        kind[j] = 2; ++nsmall;
                    } else {
                        kind[j] = 3;
                        nchunks += (uint32_t)((e - 1) / kChunk - b / kChunk + 1);
                    }
                } else {
                    kind[j] = 1; ++nkeep;
                    l_kmin = d[j] < l_kmin ? d[j] : l_kmin;
                }
            }
        }
        const uint64_t packed = (uint64_t)nkeep | ((uint64_t)nsmall << 16) | ((uint64_t)nchunks << 32);
        uint64_t tot;
        const uint64_t ex = block_excl_scan64(packed, S.tmp, &tot);
        if (tid == 0) {
            const uint32_t tk = (uint32_t)(tot & 0xFFFFu), ts = (uint32_t)((tot >> 16) & 0xFFFFu);
            const uint32_t tc = (uint32_t)(tot >> 32);
            S.base[0] = tk ? atomicAdd(&C->qsize[nx], tk) : 0u;
            S.base[1] = ts ? atomicAdd(&C->fsmall[c], ts) : 0u;
            S.base[2] = tc ? atomicAdd(&C->fchunk[c], tc) : 0u;
            if ((uint64_t)S.base[0] + tk > n || (uint64_t)S.base[1] + ts > D.fsmall_cap ||
                (uint64_t)S.base[2] + tc > D.item_cap)
                set_status(status, SSSP_ERR_INTERNAL);
        }
        __syncthreads();
        uint32_t pk = S.base[0] + (uint32_t)(ex & 0xFFFFu);
        uint64_t ps = (uint64_t)S.base[1] + ((ex >> 16) & 0xFFFFu);
        uint64_t pc = (uint64_t)S.base[2] + (ex >> 32);
#pragma unroll
        for (int j = 0; j < kExtractItems; ++j) {
            uint64_t bj = 0, ej = 0;
            if (kind[j] >= 2) { bj = __ldg(&D.off[v[j]]); ej = __ldg(&D.off[v[j] + 1]); }
            const uint64_t nch = kind[j] == 3 ? (ej - 1) / kChunk - bj / kChunk + 1 : 0;
            if (kind[j] == 1) {
                if (pk < n) Qnext[pk] = v[j];
                ++pk;
            } else if (kind[j] == 2) {
                if (ps < D.fsmall_cap) D.fsmall[ps] = make_rec(bj, ej - bj, d[j]);
                ++ps;
            } else if (kind[j] == 3 && nch <= 4) {
                for (uint64_t c0 = bj / kChunk * kChunk; c0 < ej; c0 += kChunk, ++pc) {
                    const uint64_t cs = bj > c0 ? bj : c0;
                    const uint64_t ce = ej < c0 + kChunk ? ej : c0 + kChunk;
                    if (pc < D.item_cap) D.items[pc] = make_rec(cs, ce - cs, v[j]);
                }
            }
            uint32_t many = __ballot_sync(FULL_MASK, kind[j] == 3 && nch > 4);
            while (many) {
                const int src = __ffs(many) - 1;
                many &= many - 1;
                const uint64_t sb = __shfl_sync(FULL_MASK, bj, src);
                const uint64_t se = __shfl_sync(FULL_MASK, ej, src);
                const uint32_t sv = __shfl_sync(FULL_MASK, v[j], src);
                const uint64_t sp = __shfl_sync(FULL_MASK, pc, src);
                const uint64_t sn = (se - 1) / kChunk - sb / kChunk + 1;
                for (uint64_t tt = lane; tt < sn; tt += 32) {
                    const uint64_t c0 = (sb / kChunk + tt) * kChunk;
                    const uint64_t cs = sb > c0 ? sb : c0;
                    const uint64_t ce = se < c0 + kChunk ? se : c0 + kChunk;
                    if (sp + tt < D.item_cap) D.items[sp + tt] = make_rec(cs, ce - cs, sv);
                }
            }
            if (kind[j] == 3 && nch > 4) pc += nch;
        }
        uint64_t bf = l_fcount, be = l_fedges, bm = l_kmin;
        block_reduce_2add_min(bf, be, bm, S.tmp);
        if (tid == 0) {
            if (bf) atomicAdd(&C->fcount[c], (unsigned int)bf);
            if (be) atomicAdd(&C->fedges[c], (unsigned long long)be);
            if (algo_tracks_qmin(p.algo) && bm != kInf) atomicMin(&C->qmin[nx], (unsigned long long)bm);
        }
        __syncthreads();
    }
    return true;
}

// Warp-uniform: local relaxation of a super-sparse step of one instance (Sec. 6;
// the rule of the single solve: the step's queue is at most n/20 and its
// extracted vertices have mean degree < 20), from the ids the warp has staged
// for that instance; the edges it relaxes are added to the step's edge count.
__device__ __noinline__ void local_step(const BatchParams& p, const InstDesc* D, InstCtrl* C, uint64_t k,
                                        uint32_t* stage, uint32_t& stc, uint32_t lane, uint64_t& lmin,
                                        uint32_t& lupd)
{
    const int c = (int)(k % 3), nx = (int)((k + 1) % 3);
    const uint64_t q = ldcg32(&C->qsize[c]);
    const uint64_t fcnt = ldcg32(&C->fcount[c]);
    const uint64_t fed = ldcg64((const uint64_t*)&C->fedges[c]);
    const uint64_t theta = ldcg64((const uint64_t*)&C->theta);
    if (q * 20ull > (uint64_t)D->n || fed >= 20ull * fcnt) return;
    uint32_t* Qn = (k & 1) ? D->qb : D->qa;
    const uint64_t le = local_relax(theta, D->local_budget, D->off, D->edges, D->dist, D->inq, stage, stc, lane,
                                    lmin, lupd, &C->qsize[nx], &p.ctrl->status, Qn, D->n);
    if (lane == 0 && le) atomicAdd(&C->fedges[c], (unsigned long long)le);
}

// Phase R: relaxation of every running instance's extracted vertices, work
// spread over all warps.
__device__ void phase_R(const BatchParams& p, uint64_t k, BatchSmem& S, uint32_t* stage)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
    const uint32_t gwarp = blockIdx.x * kWarps + wid;
    const uint32_t nwarps = gridDim.x * kWarps;
    const int c = (int)(k % 3), nx = (int)((k + 1) % 3);
    const uint32_t K = p.k;
    int* status = &p.ctrl->status;
    for (uint32_t i = tid; i < K; i += kBlock) {
        const InstCtrl* C = &p.ictrl[i];
        const bool run = ldcg32(&C->running) != 0;
        uint64_t fs = run ? ldcg32(&C->fsmall[c]) : 0;
        const uint64_t cap = p.inst[i].fsmall_cap;
        fs = fs < cap ? fs : cap;
        uint64_t fc = run ? ldcg32(&C->fchunk[c]) : 0;
        const uint64_t icap = p.inst[i].item_cap;
        fc = fc < icap ? fc : icap;
        S.pre0[i] = (uint32_t)((fs + 31u) >> 5);  // low-degree groups
        S.pre1[i] = (uint32_t)fc;                 // chunk records
    }
    __syncthreads();
    const uint64_t ngroups = block_prefix_inplace(S.pre0, K, S.tmp);
    const uint64_t nchunks_all = block_prefix_inplace(S.pre1, K, S.tmp);
        {
            uint32_t cur = 0xFFFFFFFFu;  // instance whose ids are staged / whose counters accumulate
            uint32_t stc = 0;
            uint64_t lmin = kInf;
            uint32_t lupd = 0;
            const uint32_t lmask = lane == 31 ? FULL_MASK : ((2u << lane) - 1u);
            // switch the warp's staging and counters to instance i
#define SWITCH_INSTANCE(i_)                                                                      \
    do {                                                                                         \
        if ((i_) != cur) {                                                                       \
            if (cur != 0xFFFFFFFFu) {                                                            \
                InstCtrl* Cc = &p.ictrl[cur];                                                    \
                const InstDesc* Dc = &p.inst[cur];                                               \
                uint32_t* Qn = (k & 1) ? Dc->qb : Dc->qa;                                        \
                if (Dc->local_budget) local_step(p, Dc, Cc, k, stage, stc, lane, lmin, lupd);    \
                stage_flush(stage, stc, lane, &Cc->qsize[nx], status, Qn, Dc->n);                \
                uint32_t u_ = lupd;                                                              \
                for (int o = 16; o > 0; o >>= 1) u_ += __shfl_xor_sync(FULL_MASK, u_, o);        \
                uint64_t m_ = lmin;                                                              \
                for (int o = 16; o > 0; o >>= 1) {                                               \
                    const uint64_t y_ = __shfl_xor_sync(FULL_MASK, m_, o);                       \
                    m_ = y_ < m_ ? y_ : m_;                                                      \
                }                                                                                \
                if (lane == 0 && u_) atomicAdd(&Cc->updates[c], (unsigned long long)u_);         \
                if (lane == 0 && algo_tracks_qmin(p.algo) && m_ != kInf) {                       \
                    atomicMin(&Cc->qmin[nx], (unsigned long long)m_);                            \
                    atomicMin(&Cc->umin[nx], (unsigned long long)m_);                            \
                }                                                                                \
                lupd = 0;                                                                        \
                lmin = kInf;                                                                     \
            }                                                                                    \
            cur = (i_);                                                                          \
        }                                                                                        \
    } while (0)

            // (a) low-degree vertices: 32 records per warp, edges flattened across lanes
            for (uint64_t g = gwarp; g < ngroups; g += nwarps) {
                const uint32_t i = find_segment(S.pre0, K, g);
                SWITCH_INSTANCE(i);
                const InstDesc* Dp = &p.inst[i];
                uint64_t* const idist = Dp->dist;
                uint32_t* const iinq = Dp->inq;
                const uint2* const iedges = Dp->edges;
                const uint64_t fcap = Dp->fsmall_cap;
                uint64_t fs = ldcg32(&p.ictrl[i].fsmall[c]);
                fs = fs < fcap ? fs : fcap;
                const uint64_t lg = g - S.pre0[i];
                const uint4 rec = (lg * 32u + lane < fs) ? __ldcg(&Dp->fsmall[lg * 32u + lane]) : make_uint4(0, 0, 0, 0);
                const uint64_t b = rec_start(rec);
                const uint32_t deg = rec_len(rec);
                const uint64_t du = rec_du(rec);
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
                    uint32_t vv[kSmallRounds];
                    uint64_t cand[kSmallRounds];
#pragma unroll
                    for (int t = 0; t < kSmallRounds; ++t) {
                        const uint2 ed = ok[t] ? __ldcs(&iedges[eidx[t]]) : make_uint2(0, 0);
                        vv[t] = ed.x;
                        cand[t] = cdu[t] + ed.y;
                    }
                    relax_batch4(idist, iinq, vv, cand, ok, stage, stc, lane, lmin, lupd);
                    if (stc > (uint32_t)(kStage - 256)) {
                        uint32_t* Qn = (k & 1) ? Dp->qb : Dp->qa;
                        stage_flush(stage, stc, lane, &p.ictrl[i].qsize[nx], status, Qn, Dp->n);
                    }
                }
            }
            // (b) higher-degree vertices: one warp per chunk record
            for (uint64_t it = gwarp; it < nchunks_all; it += nwarps) {
                const uint32_t i = find_segment(S.pre1, K, it);
                SWITCH_INSTANCE(i);
                const InstDesc* Dp = &p.inst[i];
                uint64_t* const idist = Dp->dist;
                const uint4 rc = __ldcg(&Dp->items[it - S.pre1[i]]);
                const uint64_t du = ldcg64(&idist[rc.z]);
                uint32_t* const Qn_i = (k & 1) ? Dp->qb : Dp->qa;
                if (Dp->bidir)
                    relax_chunk<true>(rc, du, reinterpret_cast<const uint4*>(Dp->edges), idist, Dp->inq, stage,
                                      stc, lane, lmin, lupd, &p.ictrl[i].qsize[nx], status, Qn_i, Dp->n);
                else
                    relax_chunk<false>(rc, du, reinterpret_cast<const uint4*>(Dp->edges), idist, Dp->inq, stage,
                                       stc, lane, lmin, lupd, &p.ictrl[i].qsize[nx], status, Qn_i, Dp->n);
                if (stc > (uint32_t)(kStage - 256)) {
                    uint32_t* Qn = (k & 1) ? Dp->qb : Dp->qa;
                    stage_flush(stage, stc, lane, &p.ictrl[i].qsize[nx], status, Qn, Dp->n);
                }
            }
            SWITCH_INSTANCE(0xFFFFFFFEu);  // flush what is left
#undef SWITCH_INSTANCE
        }
}

__global__ void __launch_bounds__(kBlock, 1) batch_kernel(BatchParams p)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint32_t* s_stage = reinterpret_cast<uint32_t*>(s_dyn);  // [kWarps][kStage]
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_dyn);   // rho samples (aliases the empty staging)
    __shared__ BatchSmem S;
    const uint32_t tid = threadIdx.x, wid = tid >> 5;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + tid;
    BatchCtrl* bctrl = p.ctrl;
    int* status = &bctrl->status;
    uint32_t* stage = s_stage + wid * kStage;
    if (tid == 0) {
        S.bar_target = 0;
        S.t_start = global_timer_ns();
        S.err = 0;
    }
    for (uint32_t i = 0; i < p.k; ++i) init_instance_fill(p.inst[i], gtid, gthreads);
    for (uint64_t i = gtid; i < p.k; i += gthreads) init_instance_ctrl(p.inst[i], &p.ictrl[i], 1);
    if (!grid_sync(&bctrl->bar, status, &S.bar_target, p.timeout_ns)) return;

    uint64_t k = 1;
    for (;; ++k) {
        phase_T(p, k, S, s_keys);
        if (tid == 0) {
            if (S.err) set_status(status, SSSP_ERR_INTERNAL);
            if (blockIdx.x == 0 && global_timer_ns() - S.t_start > p.solve_timeout_ns)
                set_status(status, SSSP_ERR_TIMEOUT);
        }
        if (!grid_sync(&bctrl->bar, status, &S.bar_target, p.timeout_ns)) return;
        if (!phase_E(p, k, S)) break;  // every queue is empty: all blocks agree
        if (!grid_sync(&bctrl->bar, status, &S.bar_target, p.timeout_ns)) return;
        phase_R(p, k, S, stage);
        if (!grid_sync(&bctrl->bar, status, &S.bar_target, p.timeout_ns)) return;
    }
    for (uint64_t i = gtid; i < p.k; i += gthreads) {
        InstCtrl* C = &p.ictrl[i];
        if (C->last_step == 0) C->last_step = (unsigned)(k - 1);
    }
    if (gtid == 0) bctrl->steps = k - 1;
}

// ---------------------------------------------------------------------------
// Serving: a long-lived persistent loop over S query slots.  At every step
// boundary block 0 retires finished queries (completion records in host-mapped
// memory) and admits newly submitted ones (commands in host-mapped memory);
// admitted queries join the running ones at the next step, so their work
// overlaps on the device (continuous batching).  With no query left the loop
// waits a bounded idle time for new commands, then the kernel exits.
// ---------------------------------------------------------------------------
struct ServeState {               // device memory, kept across launches
    unsigned long long seen_submitted;
    unsigned long long step;      // last global step run
    unsigned int nadmit;
    unsigned int exit_flag;
    unsigned int admit[kMaxBatch];
};
struct ServeParams {
    BatchParams b;
    SlotCmd* cmd;
    SlotDone* done;
    ServeShared* shared;
    ServeState* state;
    uint64_t idle_ns;
    uint64_t param;
};


// Block 0 only: retire finished slots, admit new commands; returns (in every
// thread of block 0) false when the loop should exit.
__device__ bool serve_admission(const ServeParams& sp, uint64_t k, BatchSmem& S)
{
    const BatchParams& p = sp.b;
    const uint32_t tid = threadIdx.x;
    const int c = (int)(k % 3), pv = (int)((k + 2) % 3);
    ServeState* st = sp.state;
    for (;;) {
        // retire: running slots whose queue for step k is empty finished at step k-1
        for (uint32_t i = tid; i < p.k; i += kBlock) {
            InstCtrl* C = &p.ictrl[i];
            if (!C->running || ldcg32(&C->qsize[c]) != 0) continue;
            if (k > C->admit_step) {
                C->queued += ldcg32(&C->qsize[pv]);
                C->extracted += ldcg32(&C->fcount[pv]);
                C->edges += ldcg64((const uint64_t*)&C->fedges[pv]);
                C->updates_total += ldcg64((const uint64_t*)&C->updates[pv]);
            }
            SlotDone* D = &sp.done[i];
            D->ticket = C->ticket;
            D->t_admit_ns = C->t_admit_ns;
            D->t_done_ns = global_timer_ns();
            D->edges = C->edges;
            D->extracted = C->extracted;
            D->steps = (unsigned int)(k - C->admit_step);
            D->status = *reinterpret_cast<volatile int*>(&p.ctrl->status);
            __threadfence_system();
            st_release_sys_u32(&D->seq, C->seq);
            C->running = 0;
            for (int r = 0; r < 3; ++r) {
                C->qsize[r] = 0; C->fsmall[r] = 0; C->fchunk[r] = 0; C->fcount[r] = 0;
                C->fedges[r] = 0; C->updates[r] = 0; C->qmin[r] = kInf;
            }
        }
        __syncthreads();
        // admit: free slots whose command carries a new sequence number
        if (tid == 0) {
            const unsigned long long sub = ld_acquire_sys_u64(&sp.shared->submitted);
            S.flag = sub != st->seen_submitted;
            st->seen_submitted = sub;
        }
        __syncthreads();
        if (S.flag) {
            for (uint32_t i = tid; i < p.k; i += kBlock) {
                InstCtrl* C = &p.ictrl[i];
                if (C->running) continue;
                const unsigned int cs = ld_acquire_sys_u32(&sp.cmd[i].seq);
                if (cs == C->seq) continue;
                const volatile SlotCmd* cm = &sp.cmd[i];
                InstDesc* d = &p.inst[i];
                d->dist = reinterpret_cast<uint64_t*>(cm->dist_ptr);
                d->source = cm->source < d->n ? cm->source : 0u;
                d->seed = 0x2105061450000000ull ^ (uint64_t)d->source;
                d->param = sp.param;
                init_instance_ctrl(*d, C, k);
                C->seq = cs;
                C->ticket = cm->ticket;
                C->t_admit_ns = global_timer_ns();
                st->admit[atomicAdd(&st->nadmit, 1u)] = i;
            }
        }
        __syncthreads();
        // anything running?
        uint32_t nrun = 0;
        for (uint32_t i = tid; i < p.k; i += kBlock) nrun += p.ictrl[i].running ? 1u : 0u;
        nrun = __syncthreads_count(nrun != 0);
        if (tid == 0) {
            S.flag = 0;
            if (ld_acquire_sys_u32(&sp.shared->stop)) {
                S.flag = 2;  // leave now
            } else if (nrun == 0) {
                // idle: wait (bounded) for a new command
                const unsigned long long t0 = global_timer_ns();
                S.flag = 2;
                while (global_timer_ns() - t0 < sp.idle_ns) {
                    if (ld_acquire_sys_u64(&sp.shared->submitted) != st->seen_submitted) { S.flag = 1; break; }
                    if (ld_acquire_sys_u32(&sp.shared->stop)) break;
                    __nanosleep(2000);
                }
            }
        }
        __syncthreads();
        if (S.flag == 0) return true;   // work to do
        if (S.flag == 2) return false;  // idle or stopped: exit
        // S.flag == 1: a command arrived while idle; admit it
    }
}

__global__ void __launch_bounds__(kBlock, 1) serve_kernel(ServeParams sp)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint32_t* s_stage = reinterpret_cast<uint32_t*>(s_dyn);
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_dyn);
    __shared__ BatchSmem S;
    const BatchParams& p = sp.b;
    const uint32_t tid = threadIdx.x, wid = tid >> 5;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + tid;
    BatchCtrl* bctrl = p.ctrl;
    int* status = &bctrl->status;
    uint32_t* stage = s_stage + wid * kStage;
    ServeState* st = sp.state;
    if (tid == 0) {
        S.bar_target = 0;
        S.err = 0;
    }
    __syncthreads();
    uint64_t k = ldcg64((const uint64_t*)&st->step) + 1;
    for (;; ++k) {
        // ---- phase A: retire and admit (block 0) ----
        if (blockIdx.x == 0) {
            const bool go = serve_admission(sp, k, S);
            if (tid == 0) st->exit_flag = go ? 0u : 1u;
        }
        if (!grid_sync(&bctrl->bar, status, &S.bar_target, p.timeout_ns)) return;
        if (ldcg32(&st->exit_flag)) break;
        // ---- phase I + T: initialise admitted slots, thresholds ----
        const uint32_t na = ldcg32(&st->nadmit);
        for (uint32_t a = 0; a < na; ++a) {
            const uint32_t i = ldcg32(&st->admit[a]);
            InstDesc d;
            d.dist = p.inst[i].dist; d.inq = p.inst[i].inq; d.n = p.inst[i].n; d.source = p.inst[i].source;
            init_instance_fill(d, gtid, gthreads);
        }
        phase_T(p, k, S, s_keys);
        if (tid == 0 && S.err) set_status(status, SSSP_ERR_INTERNAL);
        if (!grid_sync(&bctrl->bar, status, &S.bar_target, p.timeout_ns)) return;
        if (blockIdx.x == 0 && tid == 0) st->nadmit = 0;
        // ---- phase E, R ----
        if (phase_E(p, k, S)) {
            if (!grid_sync(&bctrl->bar, status, &S.bar_target, p.timeout_ns)) return;
            phase_R(p, k, S, stage);
        }
        if (blockIdx.x == 0 && tid == 0) st->step = k;
        if (!grid_sync(&bctrl->bar, status, &S.bar_target, p.timeout_ns)) return;
    }
    if (gtid == 0) st->step = k;
}

const void* serve_kernel_ptr() { return reinterpret_cast<const void*>(&serve_kernel); }

const void* batch_kernel_ptr() { return reinterpret_cast<const void*>(&batch_kernel); }

// ---------------------------------------------------------------------------
// Host side: a per-device workspace grown to the largest batch seen.
// ---------------------------------------------------------------------------
namespace {

struct Workspace {
    int device = -1;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    InstDesc* d_desc = nullptr;
    InstCtrl* d_ictrl = nullptr;
    BatchCtrl* d_ctrl = nullptr;
    uint32_t cap_k = 0;
    InstDesc* h_desc = nullptr;     // pinned staging of the descriptors
    InstCtrl* h_ictrl = nullptr;    // pinned readback
    BatchCtrl* h_ctrl = nullptr;
    cudaEvent_t desc_copied = nullptr;
    uint32_t last_k = 0;
    uint32_t grid = 0;
};

std::mutex g_ws_mu;
Workspace g_ws[64];

int fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? SSSP_ERR_OUT_OF_MEMORY : SSSP_ERR_CUDA; }

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t instance_scratch_bytes(uint32_t n, uint64_t fsmall_cap, uint64_t item_cap)
{
    return align256(4ull * ((n + 31ull) / 32)) + 2 * align256(4ull * n) + align256(16ull * fsmall_cap) +
           align256(16ull * item_cap);
}

int ensure_workspace(Workspace& w, int dev, uint32_t k, size_t scratch_bytes)
{
    cudaError_t e;
    if (w.device < 0) {
        w.device = dev;
        if ((e = cudaEventCreateWithFlags(&w.desc_copied, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
        if ((e = cudaMalloc(reinterpret_cast<void**>(&w.d_ctrl), sizeof(BatchCtrl))) != cudaSuccess) return fail(e);
        if ((e = cudaMallocHost(reinterpret_cast<void**>(&w.h_ctrl), sizeof(BatchCtrl))) != cudaSuccess) return fail(e);
    }
    if (k > w.cap_k) {
        cudaEventSynchronize(w.desc_copied);
        cudaDeviceSynchronize();
        cudaFree(w.d_desc);
        cudaFree(w.d_ictrl);
        cudaFreeHost(w.h_desc);
        cudaFreeHost(w.h_ictrl);
        w.d_desc = nullptr; w.d_ictrl = nullptr; w.h_desc = nullptr; w.h_ictrl = nullptr; w.cap_k = 0;
        if ((e = cudaMalloc(reinterpret_cast<void**>(&w.d_desc), sizeof(InstDesc) * k)) != cudaSuccess ||
            (e = cudaMalloc(reinterpret_cast<void**>(&w.d_ictrl), sizeof(InstCtrl) * k)) != cudaSuccess ||
            (e = cudaMallocHost(reinterpret_cast<void**>(&w.h_desc), sizeof(InstDesc) * k)) != cudaSuccess ||
            (e = cudaMallocHost(reinterpret_cast<void**>(&w.h_ictrl), sizeof(InstCtrl) * k)) != cudaSuccess)
            return fail(e);
        w.cap_k = k;
    }
    if (scratch_bytes > w.scratch_bytes) {
        cudaDeviceSynchronize();
        cudaFree(w.scratch);
        w.scratch = nullptr;
        w.scratch_bytes = 0;
        if ((e = cudaMalloc(&w.scratch, scratch_bytes)) != cudaSuccess) return fail(e);
        w.scratch_bytes = scratch_bytes;
    }
    return SSSP_OK;
}

int batch_blocks(int dev, uint32_t* grid)
{
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    const void* fn = batch_kernel_ptr();
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchDynSmem);
    if (e != cudaSuccess) return fail(e);
    int bps = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlock, kBatchDynSmem)) != cudaSuccess) return fail(e);
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return fail(e);
    if (bps < 1) return SSSP_ERR_CUDA;
    *grid = (uint32_t)(bps * sms);
    return SSSP_OK;
}

// Bidirectional relaxation and local relaxation of an instance: those of the
// graph's tuning (sssp_graph_get_tuning) when it is for the batch's rule.
// Local relaxation only on graphs of at least kBatchLocalMinN vertices: on
// large high-diameter graphs it shortens every instance's long chain of small
// steps (measured: 64 sources on a 4096^2 road-like grid, 3.4x -> 11.2x the
// plain loop), while a batch of many small graphs already fills the device
// with their small steps and loses to the per-instance local passes
// (512 graphs of 2^10..2^18 vertices: 16.5x -> 9.0x).
constexpr uint32_t kBatchLocalMinN = 1u << 20;
void batch_extras(const sssp_graph* g, sssp_algo algo, InstDesc* d)
{
    sssp_tuning t;
    d->bidir = 0;
    d->local_budget = 0;
    d->rho_reduced = kRhoReducedDefault;
    if (sssp_lookup_batch_tuning(g, &t) && t.algo == algo) {
        d->rho_reduced = t.rho_reduced == 0 ? kRhoReducedDefault
                         : t.rho_reduced == SSSP_RHO_REDUCED_NONE ? 0u : t.rho_reduced;
        d->bidir = ((t.flags & SSSP_SOLVE_BIDIRECTIONAL) && (g->flags & SSSP_GRAPH_SYMMETRIC)) ? 1u : 0u;
        if ((algo == SSSP_RHO || algo == SSSP_DELTA_STAR) && g->n >= kBatchLocalMinN) d->local_budget = t.local_budget;
    }
}

// Common path: instance i uses graph gs[i] (n_i, caps), output outs[i].
int solve_batch(const sssp_graph* const* gs, const uint32_t* sources, uint32_t k, sssp_algo algo,
                const uint64_t* params, uint64_t* const* outs, void* stream)
{
    if (k == 0 || k > kMaxBatch || !gs || !sources || !outs) return SSSP_ERR_INVALID_ARG;
    if (!algo_valid(algo)) return SSSP_ERR_INVALID_ARG;
    int dev = -1;
    size_t scratch = 0;
    uint32_t min_n = 0xFFFFFFFFu;
    for (uint32_t i = 0; i < k; ++i) {
        const sssp_graph* g = gs[i];
        if (!g || !outs[i] || sources[i] >= g->n) return SSSP_ERR_INVALID_ARG;
        if (dev < 0) dev = g->device; else if (g->device != dev) return SSSP_ERR_INVALID_ARG;
        const uint64_t prm = params ? params[i] : sssp_graph_batch_param(g, algo);
        if (algo_needs_param(algo) && prm == 0) return SSSP_ERR_INVALID_ARG;
        scratch += instance_scratch_bytes(g->n, g->fsmall_cap, g->item_cap);
        min_n = g->n < min_n ? g->n : min_n;
    }
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (dev < 0 || dev >= 64) return SSSP_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return fail(e);
    Workspace& w = g_ws[dev];
    int rc = ensure_workspace(w, dev, k, scratch);
    if (rc != SSSP_OK) return rc;
    if (w.grid == 0 && (rc = batch_blocks(dev, &w.grid)) != SSSP_OK) return rc;

    // the pinned descriptor staging is reused: wait until the previous copy left it
    if ((e = cudaEventSynchronize(w.desc_copied)) != cudaSuccess) return fail(e);
    uint32_t sample_cap = 1;
    unsigned char* base = static_cast<unsigned char*>(w.scratch);
    for (uint32_t i = 0; i < k; ++i) {
        const sssp_graph* g = gs[i];
        InstDesc& d = w.h_desc[i];
        d.off = g->d_off;
        d.edges = g->d_edges;
        d.dist = outs[i];
        d.n = g->n;
        d.source = sources[i];
        d.param = params ? params[i] : sssp_graph_batch_param(g, algo);
        d.seed = 0x2105061450000000ull ^ (uint64_t)sources[i];
        batch_extras(g, algo, &d);
        d.fsmall_cap = g->fsmall_cap;
        d.item_cap = g->item_cap;
        d.inq = reinterpret_cast<uint32_t*>(base); base += align256(4ull * ((g->n + 31ull) / 32));
        d.qa = reinterpret_cast<uint32_t*>(base); base += align256(4ull * g->n);
        d.qb = reinterpret_cast<uint32_t*>(base); base += align256(4ull * g->n);
        d.fsmall = reinterpret_cast<uint4*>(base); base += align256(16ull * g->fsmall_cap);
        d.items = reinterpret_cast<uint4*>(base); base += align256(16ull * g->item_cap);
        if (algo == SSSP_RHO) {
            const uint32_t sc = rho_sample_bound(g->n, d.param);
            sample_cap = sc > sample_cap ? sc : sample_cap;
        }
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((e = cudaMemcpyAsync(w.d_desc, w.h_desc, sizeof(InstDesc) * k, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return fail(e);
    if ((e = cudaEventRecord(w.desc_copied, st)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(w.d_ictrl, 0, sizeof(InstCtrl) * k, st)) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(w.d_ctrl, 0, sizeof(BatchCtrl), st)) != cudaSuccess) return fail(e);
    BatchParams p;
    memset(&p, 0, sizeof p);
    p.inst = w.d_desc;
    p.ictrl = w.d_ictrl;
    p.ctrl = w.d_ctrl;
    p.k = k;
    p.algo = (int)algo;
    p.timeout_ns = 2000000000ull;
    p.solve_timeout_ns = 120000000000ull;
    p.sample_cap = sample_cap;
    void* args[] = {&p};
    e = cudaLaunchCooperativeKernel(batch_kernel_ptr(), dim3(w.grid), dim3(kBlock), args, kBatchDynSmem, st);
    if (e != cudaSuccess) return fail(e);
    w.last_k = k;
    (void)min_n;
    return SSSP_OK;
}

// Which kind of batched launch ran last on a device (sssp_batch_last_stats
// reports that one).
enum { kLastSeparate = 0, kLastShared = 1 };
std::atomic<int> g_last_kind[64];
void set_last_kind(int dev, int kind)
{
    if (dev >= 0 && dev < 64) g_last_kind[dev].store(kind);
}
int last_kind(int dev) { return dev >= 0 && dev < 64 ? g_last_kind[dev].load() : kLastSeparate; }

}  // namespace
}  // namespace sssp

// ---------------------------------------------------------------------------
// Host side of the server.
// ---------------------------------------------------------------------------
struct sssp_server {
    const sssp_graph* g = nullptr;
    int device = 0;
    uint32_t S = 0;
    sssp_algo algo = SSSP_RHO;
    uint64_t param = 0;
    uint64_t idle_ns = 2000000;
    uint32_t grid = 0;
    uint32_t sample_cap = 1;
    void* scratch = nullptr;
    sssp::InstDesc* d_desc = nullptr;
    sssp::InstCtrl* d_ictrl = nullptr;
    sssp::BatchCtrl* d_ctrl = nullptr;
    sssp::ServeState* d_state = nullptr;
    sssp::SlotCmd* h_cmd = nullptr;       // mapped
    sssp::SlotDone* h_done = nullptr;     // mapped
    sssp::ServeShared* h_shared = nullptr;  // mapped
    sssp::SlotCmd* d_cmd = nullptr;
    sssp::SlotDone* d_done = nullptr;
    sssp::ServeShared* d_shared = nullptr;
    cudaStream_t stream = nullptr;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv;
    bool stopping = false;
    struct Pending { uint64_t ticket; uint32_t source; uint64_t dist; uint64_t t_submit; };
    std::deque<Pending> pending;
    struct Slot { bool busy = false; uint32_t seq = 0; uint64_t ticket = 0; uint64_t t_submit = 0; };
    std::vector<Slot> slots;
    struct Result { bool done = false; sssp_query_info info{}; uint64_t t_submit = 0; };
    std::unordered_map<uint64_t, Result> results;
    std::deque<uint64_t> completed;   // tickets completed and not yet drained
    uint64_t next_ticket = 1;
    bool kernel_running = false;
    uint64_t launches = 0;
    int fatal = SSSP_OK;
    sssp::MsServer* ms = nullptr;         // shared-scan slots (SSSP_BATCH_SHARED), else separate instances
};

namespace sssp {
namespace {

uint64_t host_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

void server_loop(sssp_server* s)
{
    cudaSetDevice(s->device);
    ServeParams sp;
    memset(&sp, 0, sizeof sp);
    sp.b.inst = s->d_desc;
    sp.b.ictrl = s->d_ictrl;
    sp.b.ctrl = s->d_ctrl;
    sp.b.k = s->S;
    sp.b.algo = (int)s->algo;
    sp.b.timeout_ns = 2000000000ull;
    sp.b.solve_timeout_ns = ~0ull;
    sp.b.sample_cap = s->sample_cap;
    sp.cmd = s->d_cmd;
    sp.done = s->d_done;
    sp.shared = s->d_shared;
    sp.state = s->d_state;
    sp.idle_ns = s->idle_ns;
    sp.param = s->param;
    unsigned long long submitted = 0;
    for (;;) {
        bool progress = false;
        bool any_busy = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stopping) break;
            bool assigned = false;
            for (uint32_t i = 0; i < s->S && !s->pending.empty(); ++i) {
                sssp_server::Slot& sl = s->slots[i];
                if (sl.busy) continue;
                const sssp_server::Pending pd = s->pending.front();
                s->pending.pop_front();
                sl.busy = true;
                sl.seq += 1;
                sl.ticket = pd.ticket;
                sl.t_submit = pd.t_submit;
                SlotCmd* cm = &s->h_cmd[i];
                __atomic_store_n(&cm->ticket, pd.ticket, __ATOMIC_RELAXED);
                __atomic_store_n(&cm->dist_ptr, pd.dist, __ATOMIC_RELAXED);
                __atomic_store_n(&cm->source, pd.source, __ATOMIC_RELAXED);
                __atomic_store_n(&cm->seq, sl.seq, __ATOMIC_RELEASE);
                assigned = true;
            }
            if (assigned) {
                ++submitted;
                __atomic_store_n(&s->h_shared->submitted, submitted, __ATOMIC_RELEASE);
                progress = true;
            }
            // completions
            for (uint32_t i = 0; i < s->S; ++i) {
                sssp_server::Slot& sl = s->slots[i];
                if (!sl.busy) continue;
                any_busy = true;
                const SlotDone* dn = &s->h_done[i];
                if (__atomic_load_n(&dn->seq, __ATOMIC_ACQUIRE) != sl.seq) continue;
                sssp_server::Result& r = s->results[sl.ticket];
                r.done = true;
                r.info.status = __atomic_load_n(&dn->status, __ATOMIC_RELAXED);
                r.info.steps = __atomic_load_n(&dn->steps, __ATOMIC_RELAXED);
                r.info.edges = __atomic_load_n(&dn->edges, __ATOMIC_RELAXED);
                const uint64_t ta = __atomic_load_n(&dn->t_admit_ns, __ATOMIC_RELAXED);
                const uint64_t td = __atomic_load_n(&dn->t_done_ns, __ATOMIC_RELAXED);
                r.info.device_ns = td - ta;
                r.info.device_admit_ns = ta;
                r.info.device_done_ns = td;
                r.info.latency_ns = host_ns() - sl.t_submit;
                s->completed.push_back(sl.ticket);
                sl.busy = false;
                progress = true;
            }
            if (progress) s->cv.notify_all();
        }
        // keep the device loop alive while there is work
        if (s->kernel_running && cudaStreamQuery(s->stream) == cudaSuccess) {
            s->kernel_running = false;
            int status = SSSP_OK;
            if (s->ms) {
                status = ms_server_status(s->ms);
            } else {
                BatchCtrl hc;
                if (cudaMemcpy(&hc, s->d_ctrl, sizeof hc, cudaMemcpyDeviceToHost) == cudaSuccess) status = hc.status;
            }
            if (status != SSSP_OK) {
                std::lock_guard<std::mutex> lk(s->mu);
                s->fatal = status;
                s->cv.notify_all();
                break;
            }
        }
        if (!s->kernel_running) {
            bool need;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                need = false;
                for (uint32_t i = 0; i < s->S; ++i) need |= s->slots[i].busy;
                need |= !s->pending.empty();
            }
            if (need) {
                void* args[] = {&sp};
                cudaError_t e = cudaSuccess;
                if (s->ms) {
                    e = ms_server_launch(s->ms, s->stream) == SSSP_OK ? cudaSuccess : cudaErrorLaunchFailure;
                } else {
                    e = cudaMemsetAsync(s->d_ctrl, 0, sizeof(BatchCtrl), s->stream);
                    if (e == cudaSuccess)
                        e = cudaLaunchCooperativeKernel(serve_kernel_ptr(), dim3(s->grid), dim3(kBlock), args,
                                                        kBatchDynSmem, s->stream);
                }
                if (e != cudaSuccess) {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->fatal = SSSP_ERR_CUDA;
                    s->cv.notify_all();
                    break;
                }
                s->kernel_running = true;
                ++s->launches;
                progress = true;
            }
        }
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(any_busy ? 5 : 50));
    }
    // shutting down: make the device loop leave and wait for it
    __atomic_store_n(&s->h_shared->stop, 1u, __ATOMIC_RELEASE);
    cudaStreamSynchronize(s->stream);
}

}  // namespace
}  // namespace sssp

using namespace sssp;

extern "C" {

int sssp_solve_sources_ex(const sssp_graph* g, const uint32_t* sources, uint32_t k, sssp_algo algo,
                          const uint64_t* params, uint32_t mode, uint64_t* dist_out, void* stream)
{
    if (!g || !dist_out || !sources || k == 0 || k > kMaxBatch || mode > SSSP_BATCH_SEPARATE)
        return SSSP_ERR_INVALID_ARG;
    if (!algo_valid(algo)) return SSSP_ERR_INVALID_ARG;
    sssp_tuning t;
    const bool tuned = sssp_lookup_batch_tuning(g, &t) && t.algo == algo;
    if (mode == SSSP_BATCH_AUTO) {
        mode = tuned && t.batch_mode ? t.batch_mode : SSSP_BATCH_SHARED;
        if (mode == SSSP_BATCH_SHARED && !ms_batch_supported(algo, k)) mode = SSSP_BATCH_SEPARATE;
    }
    std::vector<uint64_t*> outs(k);
    for (uint32_t i = 0; i < k; ++i) outs[i] = dist_out + (size_t)i * g->n;
    if (mode == SSSP_BATCH_SHARED) {
        if (!ms_batch_supported(algo, k)) return SSSP_ERR_INVALID_ARG;
        uint32_t red = kRhoReducedDefault;
        if (tuned && t.rho_reduced) red = t.rho_reduced == SSSP_RHO_REDUCED_NONE ? 0u : t.rho_reduced;
        const bool bidir = tuned && (t.flags & SSSP_SOLVE_BIDIRECTIONAL) && (g->flags & SSSP_GRAPH_SYMMETRIC);
        const uint32_t ws = tuned ? t.rho_warmup_steps : 0u;
        const uint64_t wr = tuned ? t.rho_warmup : 0u;
        const int rc = ms_solve_sources(g, sources, k, algo, params, outs.data(), red, ws, wr, bidir, stream);
        if (rc == SSSP_OK) set_last_kind(g->device, kLastShared);
        return rc;
    }
    std::vector<const sssp_graph*> gs(k, g);
    const int rc = solve_batch(gs.data(), sources, k, algo, params, outs.data(), stream);
    if (rc == SSSP_OK) set_last_kind(g->device, kLastSeparate);
    return rc;
}

int sssp_solve_sources(const sssp_graph* g, const uint32_t* sources, uint32_t k, sssp_algo algo,
                       const uint64_t* params, uint64_t* dist_out, void* stream)
{
    return sssp_solve_sources_ex(g, sources, k, algo, params, SSSP_BATCH_AUTO, dist_out, stream);
}

int sssp_solve_multi(const sssp_graph* const* gs, const uint32_t* sources, uint32_t k, sssp_algo algo,
                     const uint64_t* params, uint64_t* const* dist_outs, void* stream)
{
    const int rc = solve_batch(gs, sources, k, algo, params, dist_outs, stream);
    if (rc == SSSP_OK) set_last_kind(gs[0]->device, kLastSeparate);
    return rc;
}

int sssp_batch_last_stats(sssp_stats* out, uint32_t k, void* stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SSSP_ERR_CUDA;
    if (last_kind(dev) == kLastShared) return ms_last_stats(dev, out, k, reinterpret_cast<cudaStream_t>(stream));
    std::lock_guard<std::mutex> lk(g_ws_mu);
    Workspace& w = g_ws[dev];
    if (w.device < 0 || k > w.last_k || (k > 0 && !out)) return SSSP_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(w.h_ctrl, w.d_ctrl, sizeof(BatchCtrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && k)
        e = cudaMemcpyAsync(w.h_ictrl, w.d_ictrl, sizeof(InstCtrl) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(e);
    for (uint32_t i = 0; i < k; ++i) {
        const InstCtrl& c = w.h_ictrl[i];
        out[i].steps = c.last_step;
        out[i].queued = c.queued;
        out[i].extracted = c.extracted;
        out[i].edges = c.edges;
        out[i].updates = c.updates_total;
        out[i].status = w.h_ctrl->status;
        out[i].grid = w.grid;
    }
    return w.h_ctrl->status;
}

int sssp_server_create(const sssp_graph* g, const sssp_server_config* cfg, sssp_server** out)
{
    if (!g || !out) return SSSP_ERR_INVALID_ARG;
    *out = nullptr;
    sssp_server_config c;
    memset(&c, 0, sizeof c);
    if (cfg) c = *cfg;
    if (!algo_valid(c.algo)) return SSSP_ERR_INVALID_ARG;
    if (c.idle_ns > 1000000000ull || c.gang_wait_ns > 1000000000ull) return SSSP_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(g->device);
    if (e != cudaSuccess) return fail(e);
    sssp_server* s = new (std::nothrow) sssp_server();
    if (!s) return SSSP_ERR_OUT_OF_MEMORY;
    s->g = g;
    s->device = g->device;
    s->algo = c.algo;
    s->param = c.param ? c.param : sssp_graph_batch_param(g, c.algo);
    if (algo_needs_param(s->algo) && s->param == 0) { delete s; return SSSP_ERR_INVALID_ARG; }
    s->idle_ns = c.idle_ns ? c.idle_ns : 2000000ull;
    // the slots' kernel: one shared edge scan (SSSP_BATCH_SHARED) or separate instances
    if (c.batch_mode > SSSP_BATCH_SEPARATE) { delete s; return SSSP_ERR_INVALID_ARG; }
    sssp_tuning bt;
    const bool btuned = sssp_lookup_batch_tuning(g, &bt) && bt.algo == c.algo;
    uint32_t mode = c.batch_mode;
    if (mode == SSSP_BATCH_AUTO) {
        mode = btuned && bt.batch_mode ? bt.batch_mode : SSSP_BATCH_SHARED;
        if (mode == SSSP_BATCH_SHARED && !ms_batch_supported(c.algo, 1)) mode = SSSP_BATCH_SEPARATE;
    } else if (mode == SSSP_BATCH_SHARED && !ms_batch_supported(c.algo, 1)) {
        delete s;
        return SSSP_ERR_INVALID_ARG;
    }
    // admission by free HBM: the slots' working memory out of a fraction of what is free
    size_t free_b = 0, total_b = 0;
    if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) { delete s; return fail(e); }
    const double frac = (c.hbm_fraction > 0.0 && c.hbm_fraction <= 1.0) ? c.hbm_fraction : 0.5;
    const uint64_t budget = (uint64_t)((double)free_b * frac);
    const uint64_t cap = mode == SSSP_BATCH_SHARED ? 64u : kMaxBatch;
    uint64_t want = c.slots ? c.slots : cap;
    if (!c.slots && g->batch_tuned && btuned && bt.slots) want = bt.slots;
    if (want > cap) want = cap;
    const size_t per_slot = instance_scratch_bytes(g->n, g->fsmall_cap, g->item_cap);
    if (mode == SSSP_BATCH_SHARED) {
        while (want > 0 && ms_server_bytes(g, (uint32_t)want) > budget) --want;
    } else {
        const uint64_t fit = budget / (per_slot ? per_slot : 1);
        if (fit < want) want = fit;
    }
    if (want == 0) { delete s; return SSSP_ERR_OUT_OF_MEMORY; }
    s->S = (uint32_t)want;
    s->slots.resize(s->S);
    const size_t S = s->S;
    if ((e = cudaHostAlloc(reinterpret_cast<void**>(&s->h_cmd), sizeof(SlotCmd) * S, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostAlloc(reinterpret_cast<void**>(&s->h_done), sizeof(SlotDone) * S, cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostAlloc(reinterpret_cast<void**>(&s->h_shared), sizeof(ServeShared), cudaHostAllocMapped)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_cmd), s->h_cmd, 0)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_done), s->h_done, 0)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&s->d_shared), s->h_shared, 0)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess) {
        sssp_server_destroy(s);
        return fail(e);
    }
    memset(s->h_cmd, 0, sizeof(SlotCmd) * S);
    memset(s->h_done, 0, sizeof(SlotDone) * S);
    memset(s->h_shared, 0, sizeof(ServeShared));
    if (mode == SSSP_BATCH_SHARED) {
        uint32_t red = kRhoReducedDefault;
        if (btuned && bt.rho_reduced) red = bt.rho_reduced == SSSP_RHO_REDUCED_NONE ? 0u : bt.rho_reduced;
        const bool bidir = btuned && (bt.flags & SSSP_SOLVE_BIDIRECTIONAL);
        // (no warm-up steps in the server: under a stream of queries the
        // warm-up cohorts served RMAT-22 at 325 queries/s against 507 without)
        const int rc = ms_server_create(g, s->S, s->algo, s->param, red, 0u, 0u, bidir, s->d_cmd, s->d_done,
                                        s->d_shared, s->idle_ns, c.gang, c.gang_wait_ns, &s->ms);
        if (rc != SSSP_OK) { sssp_server_destroy(s); return rc; }
        s->worker = std::thread(server_loop, s);
        *out = s;
        return SSSP_OK;
    }
    int rc = batch_blocks(g->device, &s->grid);
    if (rc != SSSP_OK) { sssp_server_destroy(s); return rc; }
    {
        const void* fn = serve_kernel_ptr();
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchDynSmem);
        int bps = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlock, kBatchDynSmem);
        if (e != cudaSuccess || bps < 1) { sssp_server_destroy(s); return e != cudaSuccess ? fail(e) : SSSP_ERR_CUDA; }
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
        s->grid = (uint32_t)(bps * sms);
    }
    s->sample_cap = s->algo == SSSP_RHO ? rho_sample_bound(g->n, s->param) : 1;
    if ((e = cudaMalloc(&s->scratch, per_slot * S)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&s->d_desc), sizeof(InstDesc) * S)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&s->d_ictrl), sizeof(InstCtrl) * S)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&s->d_ctrl), sizeof(BatchCtrl))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&s->d_state), sizeof(ServeState))) != cudaSuccess) {
        sssp_server_destroy(s);
        return fail(e);
    }
    std::vector<InstDesc> desc(S);
    unsigned char* base = static_cast<unsigned char*>(s->scratch);
    for (size_t i = 0; i < S; ++i) {
        InstDesc& d = desc[i];
        memset(&d, 0, sizeof d);
        d.off = g->d_off;
        d.edges = g->d_edges;
        d.n = g->n;
        d.param = s->param;
        batch_extras(g, s->algo, &d);
        d.fsmall_cap = g->fsmall_cap;
        d.item_cap = g->item_cap;
        d.inq = reinterpret_cast<uint32_t*>(base); base += align256(4ull * ((g->n + 31ull) / 32));
        d.qa = reinterpret_cast<uint32_t*>(base); base += align256(4ull * g->n);
        d.qb = reinterpret_cast<uint32_t*>(base); base += align256(4ull * g->n);
        d.fsmall = reinterpret_cast<uint4*>(base); base += align256(16ull * g->fsmall_cap);
        d.items = reinterpret_cast<uint4*>(base); base += align256(16ull * g->item_cap);
    }
    if ((e = cudaMemcpy(s->d_desc, desc.data(), sizeof(InstDesc) * S, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(s->d_ictrl, 0, sizeof(InstCtrl) * S)) != cudaSuccess ||
        (e = cudaMemset(s->d_state, 0, sizeof(ServeState))) != cudaSuccess) {
        sssp_server_destroy(s);
        return fail(e);
    }
    s->worker = std::thread(server_loop, s);
    *out = s;
    return SSSP_OK;
}

int sssp_server_slots(const sssp_server* s, uint32_t* slots)
{
    if (!s || !slots) return SSSP_ERR_INVALID_ARG;
    *slots = s->S;
    return SSSP_OK;
}

int sssp_server_mode(const sssp_server* s, uint32_t* mode)
{
    if (!s || !mode) return SSSP_ERR_INVALID_ARG;
    *mode = s->ms ? SSSP_BATCH_SHARED : SSSP_BATCH_SEPARATE;
    return SSSP_OK;
}

int sssp_server_submit(sssp_server* s, uint32_t source, uint64_t* dist_out, uint64_t* ticket)
{
    if (!s || !dist_out || !ticket || source >= s->g->n) return SSSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal != SSSP_OK) return s->fatal;
    if (s->stopping) return SSSP_ERR_INVALID_ARG;
    const uint64_t t = s->next_ticket++;
    sssp_server::Pending pd;
    pd.ticket = t;
    pd.source = source;
    pd.dist = reinterpret_cast<uint64_t>(dist_out);
    pd.t_submit = host_ns();
    s->pending.push_back(pd);
    s->results[t].t_submit = pd.t_submit;
    *ticket = t;
    return SSSP_OK;
}

int sssp_server_poll(sssp_server* s, uint64_t ticket, sssp_query_info* info)
{
    if (!s) return SSSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return SSSP_ERR_INVALID_ARG;
    if (!it->second.done) return s->fatal != SSSP_OK ? s->fatal : 0;
    if (info) *info = it->second.info;
    s->results.erase(it);
    return 1;
}

int sssp_server_wait(sssp_server* s, uint64_t ticket, uint64_t timeout_ns, sssp_query_info* info)
{
    if (!s) return SSSP_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->results.find(ticket);
    if (it == s->results.end()) return SSSP_ERR_INVALID_ARG;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns ? timeout_ns : 60000000000ull);
    while (!s->results[ticket].done && s->fatal == SSSP_OK) {
        if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) return SSSP_ERR_TIMEOUT;
    }
    auto& r = s->results[ticket];
    if (!r.done) return s->fatal;
    if (info) *info = r.info;
    s->results.erase(ticket);
    return 1;
}

int sssp_server_drain(sssp_server* s, uint64_t* tickets, sssp_query_info* infos, uint32_t max)
{
    if (!s || (max > 0 && (!tickets || !infos))) return SSSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    uint32_t got = 0;
    while (got < max && !s->completed.empty()) {
        const uint64_t t = s->completed.front();
        s->completed.pop_front();
        auto it = s->results.find(t);
        if (it == s->results.end()) continue;  // already collected by poll / wait
        tickets[got] = t;
        infos[got] = it->second.info;
        s->results.erase(it);
        ++got;
    }
    if (got == 0 && s->fatal != SSSP_OK) return s->fatal;
    return (int)got;
}

int sssp_server_stats(const sssp_server* s, uint64_t* launches, uint32_t* busy_slots, uint64_t* pending)
{
    if (!s) return SSSP_ERR_INVALID_ARG;
    sssp_server* m = const_cast<sssp_server*>(s);
    std::lock_guard<std::mutex> lk(m->mu);
    uint32_t b = 0;
    for (const auto& sl : m->slots) b += sl.busy ? 1u : 0u;
    if (launches) *launches = m->launches;
    if (busy_slots) *busy_slots = b;
    if (pending) *pending = m->pending.size();
    return SSSP_OK;
}

int sssp_server_destroy(sssp_server* s)
{
    if (!s) return SSSP_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->stream) { cudaStreamSynchronize(s->stream); cudaStreamDestroy(s->stream); }
    ms_server_destroy(s->ms);
    cudaFree(s->scratch);
    cudaFree(s->d_desc);
    cudaFree(s->d_ictrl);
    cudaFree(s->d_ctrl);
    cudaFree(s->d_state);
    if (s->h_cmd) cudaFreeHost(s->h_cmd);
    if (s->h_done) cudaFreeHost(s->h_done);
    if (s->h_shared) cudaFreeHost(s->h_shared);
    delete s;
    return SSSP_OK;
}

}  // extern "C"
