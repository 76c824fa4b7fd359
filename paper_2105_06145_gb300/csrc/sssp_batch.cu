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

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

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
    unsigned long long theta;      // theta of the current step
    unsigned long long delta_i;    // Delta*-Stepping bucket index
    unsigned int dense_seen;       // rho-Stepping: dense steps so far
    unsigned int last_step;        // steps the instance took (set when its queue empties)
    unsigned long long queued, extracted, edges, updates_total;
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
};

struct BatchCtrl {
    unsigned long long bar;
    int status;
    unsigned int pad;
    unsigned long long steps;
};

struct BatchParams {
    const InstDesc* inst;
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

__global__ void __launch_bounds__(kBlock, 1) batch_kernel(BatchParams p)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint32_t* s_stage = reinterpret_cast<uint32_t*>(s_dyn);  // [kWarps][kStage]
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_dyn);   // rho samples (aliases the empty staging)
    __shared__ uint32_t s_pre0[kMaxBatch + 1];
    __shared__ uint32_t s_pre1[kMaxBatch + 1];
    __shared__ uint64_t s_tmp[3 * kWarps];
    __shared__ uint32_t s_base[3];
    __shared__ unsigned long long s_bar_target, s_t_start;
    __shared__ int s_err;

    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + tid;
    const uint32_t gwarp = blockIdx.x * kWarps + wid;
    const uint32_t nwarps = gridDim.x * kWarps;
    const uint32_t K = p.k;
    BatchCtrl* bctrl = p.ctrl;
    int* status = &bctrl->status;
    uint32_t* stage = s_stage + wid * kStage;

    if (tid == 0) {
        s_bar_target = 0;
        s_t_start = global_timer_ns();
        s_err = 0;
    }

    // ---- init of every instance: delta <- inf, delta[s] <- 0, Q = {s} ----
    for (uint32_t i = 0; i < K; ++i) {
        const InstDesc d = p.inst[i];
        for (uint64_t v = gtid; v < d.n; v += gthreads) d.dist[v] = (v == d.source) ? 0ull : kInf;
        const uint32_t nwords = (d.n + 31u) >> 5;
        for (uint64_t w = gtid; w < nwords; w += gthreads)
            d.inq[w] = (w == (d.source >> 5)) ? (1u << (d.source & 31u)) : 0u;
    }
    for (uint64_t i = gtid; i < K; i += gthreads) {
        InstCtrl* C = &p.ictrl[i];
        p.inst[i].qa[0] = p.inst[i].source;
        C->qsize[1] = 1;
        C->qmin[0] = kInf;
        C->qmin[1] = 0;
        C->qmin[2] = kInf;
        C->delta_i = 1;
    }
    if (!grid_sync(&bctrl->bar, status, &s_bar_target, p.timeout_ns)) return;

    uint64_t k = 1;
    for (;; ++k) {
        const int c = (int)(k % 3), nx = (int)((k + 1) % 3), pv = (int)((k + 2) % 3);

        // ---------------- phase T: bookkeeping and theta_i ----------------
        for (uint32_t i = blockIdx.x; i < K; i += gridDim.x) {
            InstCtrl* C = &p.ictrl[i];
            const InstDesc& D = p.inst[i];
            uint32_t q = ldcg32(&C->qsize[c]);
            q = q < D.n ? q : D.n;
            if (tid == 0) {
                if (k > 1) {
                    C->queued += ldcg32(&C->qsize[pv]);
                    C->extracted += ldcg32(&C->fcount[pv]);
                    C->edges += ldcg64((const uint64_t*)&C->fedges[pv]);
                    C->updates_total += ldcg64((const uint64_t*)&C->updates[pv]);
                }
                if (q == 0 && C->last_step == 0) C->last_step = (unsigned)(k - 1);
                C->qsize[pv] = 0; C->fsmall[pv] = 0; C->fchunk[pv] = 0; C->fcount[pv] = 0;
                C->fedges[pv] = 0; C->updates[pv] = 0; C->qmin[pv] = kInf;
            }
            if (q == 0) { __syncthreads(); continue; }  // block-uniform
            uint64_t theta;
            if (p.algo == SSSP_BELLMAN_FORD) {
                theta = kInf;
            } else if (p.algo == SSSP_DELTA_STAR) {
                const uint64_t qmin = ldcg64((const uint64_t*)&C->qmin[c]);
                uint64_t cur = ldcg64((const uint64_t*)&C->delta_i);
                theta = sat_mul(cur, D.param);
                if (qmin > theta) {
                    cur = qmin / D.param + ((qmin % D.param) != 0);
                    theta = sat_mul(cur, D.param);
                }
                __syncthreads();
                if (tid == 0) C->delta_i = cur + 1;
            } else {
                const uint32_t* Qcur = (k & 1) ? D.qa : D.qb;
                const uint32_t dense_seen = ldcg32(&C->dense_seen);
                theta = rho_extdist_block(Qcur, q, D.dist, D.n, D.param, D.seed, k, dense_seen, s_keys,
                                          p.sample_cap, &s_err);
                if (tid == 0 && (uint64_t)q * 20ull > (uint64_t)D.n) C->dense_seen = dense_seen + 1;
            }
            if (tid == 0) C->theta = theta;
            __syncthreads();
        }
        if (tid == 0) {
            if (s_err) set_status(status, SSSP_ERR_INTERNAL);
            if (blockIdx.x == 0 && global_timer_ns() - s_t_start > p.solve_timeout_ns)
                set_status(status, SSSP_ERR_TIMEOUT);
        }
        if (!grid_sync(&bctrl->bar, status, &s_bar_target, p.timeout_ns)) return;

        // ---------------- phase E: Extract(theta_i) ----------------
        const uint32_t tileq = (uint32_t)kBlock * kExtractItems;
        for (uint32_t i = tid; i < K; i += kBlock) {
            uint32_t q = ldcg32(&p.ictrl[i].qsize[c]);
            const uint32_t n_i = p.inst[i].n;
            q = q < n_i ? q : n_i;
            s_pre0[i] = (q + tileq - 1) / tileq;  // tiles of instance i
        }
        __syncthreads();
        const uint64_t ntiles = block_prefix_inplace(s_pre0, K, s_tmp);
        if (ntiles == 0) break;  // every queue is empty: all blocks agree
        for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const uint32_t i = find_segment(s_pre0, K, t);
            const InstDesc& D = p.inst[i];
            InstCtrl* C = &p.ictrl[i];
            const uint32_t n = D.n;
            uint32_t q = ldcg32(&C->qsize[c]);
            q = q < n ? q : n;
            const uint64_t theta = ldcg64((const uint64_t*)&C->theta);
            const uint32_t* Qcur = (k & 1) ? D.qa : D.qb;
            uint32_t* Qnext = (k & 1) ? D.qb : D.qa;
            const uint64_t base = (t - s_pre0[i]) * (uint64_t)tileq;
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
            const uint64_t ex = block_excl_scan64(packed, s_tmp, &tot);
            if (tid == 0) {
                const uint32_t tk = (uint32_t)(tot & 0xFFFFu), ts = (uint32_t)((tot >> 16) & 0xFFFFu);
                const uint32_t tc = (uint32_t)(tot >> 32);
                s_base[0] = tk ? atomicAdd(&C->qsize[nx], tk) : 0u;
                s_base[1] = ts ? atomicAdd(&C->fsmall[c], ts) : 0u;
                s_base[2] = tc ? atomicAdd(&C->fchunk[c], tc) : 0u;
                if ((uint64_t)s_base[0] + tk > n || (uint64_t)s_base[1] + ts > D.fsmall_cap ||
                    (uint64_t)s_base[2] + tc > D.item_cap)
                    set_status(status, SSSP_ERR_INTERNAL);
            }
            __syncthreads();
            uint32_t pk = s_base[0] + (uint32_t)(ex & 0xFFFFu);
            uint64_t ps = (uint64_t)s_base[1] + ((ex >> 16) & 0xFFFFu);
            uint64_t pc = (uint64_t)s_base[2] + (ex >> 32);
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
            block_reduce_2add_min(bf, be, bm, s_tmp);
            if (tid == 0) {
                if (bf) atomicAdd(&C->fcount[c], (unsigned int)bf);
                if (be) atomicAdd(&C->fedges[c], (unsigned long long)be);
                if (p.algo == SSSP_DELTA_STAR && bm != kInf) atomicMin(&C->qmin[nx], (unsigned long long)bm);
            }
            __syncthreads();
        }
        if (!grid_sync(&bctrl->bar, status, &s_bar_target, p.timeout_ns)) return;

        // ---------------- phase R: relax every instance's extracted vertices ----------------
        for (uint32_t i = tid; i < K; i += kBlock) {
            const InstCtrl* C = &p.ictrl[i];
            uint64_t fs = ldcg32(&C->fsmall[c]);
            const uint64_t cap = p.inst[i].fsmall_cap;
            fs = fs < cap ? fs : cap;
            uint64_t fc = ldcg32(&C->fchunk[c]);
            const uint64_t icap = p.inst[i].item_cap;
            fc = fc < icap ? fc : icap;
            s_pre0[i] = (uint32_t)((fs + 31u) >> 5);  // low-degree groups
            s_pre1[i] = (uint32_t)fc;                 // chunk records
        }
        __syncthreads();
        const uint64_t ngroups = block_prefix_inplace(s_pre0, K, s_tmp);
        const uint64_t nchunks_all = block_prefix_inplace(s_pre1, K, s_tmp);
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
                uint32_t* Qn = (k & 1) ? p.inst[cur].qb : p.inst[cur].qa;                        \
                stage_flush(stage, stc, lane, &Cc->qsize[nx], status, Qn, p.inst[cur].n);        \
                uint32_t u_ = lupd;                                                              \
                for (int o = 16; o > 0; o >>= 1) u_ += __shfl_xor_sync(FULL_MASK, u_, o);        \
                uint64_t m_ = lmin;                                                              \
                for (int o = 16; o > 0; o >>= 1) {                                               \
                    const uint64_t y_ = __shfl_xor_sync(FULL_MASK, m_, o);                       \
                    m_ = y_ < m_ ? y_ : m_;                                                      \
                }                                                                                \
                if (lane == 0 && u_) atomicAdd(&Cc->updates[c], (unsigned long long)u_);         \
                if (lane == 0 && p.algo == SSSP_DELTA_STAR && m_ != kInf)                        \
                    atomicMin(&Cc->qmin[nx], (unsigned long long)m_);                            \
                lupd = 0;                                                                        \
                lmin = kInf;                                                                     \
            }                                                                                    \
            cur = (i_);                                                                          \
        }                                                                                        \
    } while (0)

            // (a) low-degree vertices: 32 records per warp, edges flattened across lanes
            for (uint64_t g = gwarp; g < ngroups; g += nwarps) {
                const uint32_t i = find_segment(s_pre0, K, g);
                SWITCH_INSTANCE(i);
                const InstDesc* Dp = &p.inst[i];
                uint64_t* const idist = Dp->dist;
                uint32_t* const iinq = Dp->inq;
                const uint2* const iedges = Dp->edges;
                const uint64_t fcap = Dp->fsmall_cap;
                uint64_t fs = ldcg32(&p.ictrl[i].fsmall[c]);
                fs = fs < fcap ? fs : fcap;
                const uint64_t lg = g - s_pre0[i];
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
                const uint32_t i = find_segment(s_pre1, K, it);
                SWITCH_INSTANCE(i);
                const InstDesc* Dp = &p.inst[i];
                uint64_t* const idist = Dp->dist;
                const uint4 rc = __ldcg(&Dp->items[it - s_pre1[i]]);
                const uint64_t du = ldcg64(&idist[rc.z]);
                relax_chunk(rc, du, reinterpret_cast<const uint4*>(Dp->edges), idist, Dp->inq, stage, stc, lane,
                            lmin, lupd);
                if (stc > (uint32_t)(kStage - 256)) {
                    uint32_t* Qn = (k & 1) ? Dp->qb : Dp->qa;
                    stage_flush(stage, stc, lane, &p.ictrl[i].qsize[nx], status, Qn, Dp->n);
                }
            }
            SWITCH_INSTANCE(0xFFFFFFFEu);  // flush what is left
#undef SWITCH_INSTANCE
        }
        if (!grid_sync(&bctrl->bar, status, &s_bar_target, p.timeout_ns)) return;
    }

    // every queue is empty: record the step counts
    for (uint64_t i = gtid; i < K; i += gthreads) {
        InstCtrl* C = &p.ictrl[i];
        if (C->last_step == 0) C->last_step = (unsigned)(k - 1);
    }
    if (gtid == 0) bctrl->steps = k - 1;
}

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
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveDynSmem);
    if (e != cudaSuccess) return fail(e);
    int bps = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kBlock, kSolveDynSmem)) != cudaSuccess) return fail(e);
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return fail(e);
    if (bps < 1) return SSSP_ERR_CUDA;
    *grid = (uint32_t)(bps * sms);
    return SSSP_OK;
}

// Common path: instance i uses graph gs[i] (n_i, caps), output outs[i].
int solve_batch(const sssp_graph* const* gs, const uint32_t* sources, uint32_t k, sssp_algo algo,
                const uint64_t* params, uint64_t* const* outs, void* stream)
{
    if (k == 0 || k > kMaxBatch || !gs || !sources || !outs) return SSSP_ERR_INVALID_ARG;
    if (algo != SSSP_RHO && algo != SSSP_DELTA_STAR && algo != SSSP_BELLMAN_FORD) return SSSP_ERR_INVALID_ARG;
    int dev = -1;
    size_t scratch = 0;
    uint32_t min_n = 0xFFFFFFFFu;
    for (uint32_t i = 0; i < k; ++i) {
        const sssp_graph* g = gs[i];
        if (!g || !outs[i] || sources[i] >= g->n) return SSSP_ERR_INVALID_ARG;
        if (dev < 0) dev = g->device; else if (g->device != dev) return SSSP_ERR_INVALID_ARG;
        const uint64_t prm = params ? params[i] : sssp_default_param(g->n, g->m, algo, g->mean_w);
        if (algo != SSSP_BELLMAN_FORD && prm == 0) return SSSP_ERR_INVALID_ARG;
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
        d.param = params ? params[i] : sssp_default_param(g->n, g->m, algo, g->mean_w);
        d.seed = 0x2105061450000000ull ^ (uint64_t)sources[i];
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
    e = cudaLaunchCooperativeKernel(batch_kernel_ptr(), dim3(w.grid), dim3(kBlock), args, kSolveDynSmem, st);
    if (e != cudaSuccess) return fail(e);
    w.last_k = k;
    (void)min_n;
    return SSSP_OK;
}

}  // namespace
}  // namespace sssp

using namespace sssp;

extern "C" {

int sssp_solve_sources(const sssp_graph* g, const uint32_t* sources, uint32_t k, sssp_algo algo,
                       const uint64_t* params, uint64_t* dist_out, void* stream)
{
    if (!g || !dist_out || k == 0 || k > kMaxBatch) return SSSP_ERR_INVALID_ARG;
    std::vector<const sssp_graph*> gs(k, g);
    std::vector<uint64_t*> outs(k);
    for (uint32_t i = 0; i < k; ++i) outs[i] = dist_out + (size_t)i * g->n;
    return solve_batch(gs.data(), sources, k, algo, params, outs.data(), stream);
}

int sssp_solve_multi(const sssp_graph* const* gs, const uint32_t* sources, uint32_t k, sssp_algo algo,
                     const uint64_t* params, uint64_t* const* dist_outs, void* stream)
{
    return solve_batch(gs, sources, k, algo, params, dist_outs, stream);
}

int sssp_batch_last_stats(sssp_stats* out, uint32_t k, void* stream)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SSSP_ERR_CUDA;
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

}  // extern "C"
