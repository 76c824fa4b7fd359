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
// lists, counters) is read with L2-only loads (ld.global.cg) or atomics --
// except the relaxation's pre-check of delta[v], which reads through L1 and
// may see a value that is too high, never one too low (ld_precheck); the
// graph (offsets, packed edges) is read-only for the kernel's lifetime.
// Every device-wide wait is bounded by a globaltimer deadline; on expiry the
// kernel records SSSP_ERR_TIMEOUT and every block returns.

#include <cstdint>
#include <cuda_runtime.h>

#include "sssp_internal.h"
#include "sssp_device.cuh"

namespace sssp {

// Fused super-sparse steps (SSSP_SOLVE_FUSED) are compiled into the narrow
// shape only: in the wide one (64 registers a thread) the extra live state
// spills.  The wide shape runs every step unfused.
constexpr bool kFusedSteps = kBlock <= 512;

// ---------------------------------------------------------------------------
// Block 0, one thread: add the counters of step `step` (ring slot `slot`) to
// the solve's totals and to its trace record, then reset the slot for reuse.
// Called during step step+1 (the slot is complete by then and is not written
// again before step step+2), and once more when the loop ends.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void fold_step(const SolveParams& p, Ctrl* ctrl, int slot, uint64_t step)
{
    if (step >= 1) {
        const uint32_t qq = ldcg32(&ctrl->qsize[slot]);
        const uint32_t ff = ldcg32(&ctrl->fcount[slot]);
        const uint64_t ee = ldcg64((const uint64_t*)&ctrl->fedges[slot]);
        const uint64_t uu = ldcg64((const uint64_t*)&ctrl->updates[slot]);
        const uint64_t le = ldcg64((const uint64_t*)&ctrl->ledges[slot]);
        ctrl->queued += qq; ctrl->extracted += ff; ctrl->edges += ee + le; ctrl->updates_total += uu;
        if (p.trace && step - 1 < p.trace_cap) {
            sssp_step_trace* rec = &p.trace[step - 1];  // theta and times are written during the step
            rec->queued = qq; rec->extracted = ff; rec->edges = ee + le; rec->updates = uu;
        }
    }
    ctrl->qsize[slot] = 0; ctrl->fsmall[slot] = 0; ctrl->fchunk[slot] = 0; ctrl->fcount[slot] = 0;
    ctrl->fedges[slot] = 0; ctrl->updates[slot] = 0; ctrl->qmin[slot] = kInf; ctrl->umin[slot] = kInf;
    ctrl->ledges[slot] = 0;
}

// ---------------------------------------------------------------------------
// The persistent solve kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock, kMinBlocks) solve_kernel(SolveParams p)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint32_t* s_stage = reinterpret_cast<uint32_t*>(s_dyn);  // [kWarps][kStage]
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_dyn);   // rho samples (aliases the empty staging)
    __shared__ uint64_t s_tmp[6 * kWarps];
    __shared__ uint32_t s_base[3];
    __shared__ uint32_t s_wcnt[kWarps];
    __shared__ int s_err;

    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
    const uint32_t n = p.n;
    const uint64_t gthreads = (uint64_t)gridDim.x * kBlock;
    const uint64_t gtid = (uint64_t)blockIdx.x * kBlock + tid;
    Ctrl* ctrl = p.ctrl;
    uint64_t* dist = p.dist;
    uint32_t* inq = p.inq;
    __shared__ unsigned long long s_bar_target;   // thread 0: barrier arrivals expected so far
    __shared__ unsigned long long s_t_start;      // solve start (globaltimer)
    const uint64_t* __restrict__ off = p.off;
    const uint2* __restrict__ edges = p.edges;
    const uint4* __restrict__ pairs = reinterpret_cast<const uint4*>(p.edges);
    uint32_t* stage = s_stage + wid * kStage;

    if (tid == 0) {
        s_err = 0;
        s_bar_target = 0;
        s_t_start = global_timer_ns();
    }

    // ---- init: delta <- inf, delta[s] <- 0, Q.Update(s) (Algorithm 1) ----
    for (uint64_t i = gtid; i < n; i += gthreads) dist[i] = (i == p.source) ? 0ull : kInf;
    const uint32_t nwords = (n + 31u) >> 5;
    for (uint64_t i = gtid; i < nwords; i += gthreads)
        inq[i] = (i == (p.source >> 5)) ? (1u << (p.source & 31u)) : 0u;
    if (p.ext_count)
        for (uint64_t i = gtid; i < n; i += gthreads) p.ext_count[i] = 0;
    if (p.lrel)
        for (uint64_t i = gtid; i < n; i += gthreads) p.lrel[i] = kInf;
    if (p.trace)
        for (uint64_t i = gtid; i < p.trace_cap; i += gthreads) {
            p.trace[i].t_extract_end_max = 0;
            p.trace[i].t_relax_end_min = kInf;
            p.trace[i].t_relax_end_max = 0;
        }
    if (blockIdx.x == 0 && tid == 0) {
        ctrl->t0 = s_t_start;
        p.qa[0] = p.source;
        ctrl->qsize[1] = 1;
        ctrl->qmin[0] = kInf;
        ctrl->qmin[1] = 0;
        ctrl->qmin[2] = kInf;
        ctrl->umin[0] = kInf;
        ctrl->umin[1] = kInf;
        ctrl->umin[2] = kInf;
    }
    if (p.exit_block != 0 && blockIdx.x == p.exit_block - 1) return;  // fault-injection test
    const bool started = grid_sync_err(&ctrl->bar, &ctrl->status, &s_bar_target, p.timeout_ns);
    if (tid == 0) s_t_start = ldcg64((const uint64_t*)&ctrl->t0);  // one time origin for every block
    __syncthreads();

    uint64_t delta_i = 1;          // Delta*- / Delta-Stepping bucket index (Table 2)
    uint64_t prev_theta = 0;       // theta of the previous step (Delta-Stepping FinishCheck)
    uint32_t dense_seen = 0;       // rho-Stepping: dense steps so far (Sec. 6)
    bool prev_fused = false;       // the previous step was fused (SSSP_SOLVE_FUSED; grid-uniform)
    uint32_t fre_L = 0;            // ... and this block's slice of its queue had fre_L entries

    uint64_t k = 1;
    for (; started; ++k) {
        const int c = (int)(k % 3), nx = (int)((k + 1) % 3), pv = (int)((k + 2) % 3);
        const uint32_t* Qcur = (k & 1) ? p.qa : p.qb;
        uint32_t* Qnext = (k & 1) ? p.qb : p.qa;
        // the step's inputs, loaded together: |Q_k|, min_Q delta, and the
        // smallest distance the previous step wrote
        uint32_t q = ldcg32(&ctrl->qsize[c]);
        const uint64_t qmin_c = algo_tracks_qmin(p.algo) ? ldcg64((const uint64_t*)&ctrl->qmin[c]) : kInf;
        const uint64_t umin_c = p.algo == SSSP_DELTA ? ldcg64((const uint64_t*)&ctrl->umin[c]) : kInf;
        q = q < n ? q : n;  // a capacity fault is reported via status; never read past a list

        // an empty queue ends the solve, unless the previous step was fused:
        // then this step only re-checks that step's extractions (below)
        if (q == 0 && !(kFusedSteps && prev_fused)) {
            if (blockIdx.x == 0 && tid == 0) fold_step(p, ctrl, pv, k - 1);
            break;
        }
        if (p.max_steps != 0 && k > p.max_steps) {
            if (blockIdx.x == 0 && tid == 0) {
                fold_step(p, ctrl, pv, k - 1);
                raise_error(&ctrl->bar, &ctrl->status, SSSP_ERR_INTERNAL);
            }
            break;
        }
        // global warp rank for the relaxation's round-robin over records,
        // numbered across the blocks first: consecutive records (a hub's
        // chunks; the few records of a small step) land on different SMs
        const uint32_t gwarp = wid * gridDim.x + blockIdx.x;
        const uint32_t nwarps = gridDim.x * kWarps;
        if (blockIdx.x == 0 && tid == 0) {
            const unsigned long long now = global_timer_ns() - s_t_start;
            if (p.trace && k - 1 < p.trace_cap) p.trace[k - 1].t_ns = now;
            // whole-solve time guard: block 0 records it; every block leaves at
            // the next barrier
            if (now > p.solve_timeout_ns) raise_error(&ctrl->bar, &ctrl->status, SSSP_ERR_TIMEOUT);
        }

        // ---------------- ExtDist ----------------
        uint64_t theta;
        bool rho_sample = false;  // rho-Stepping with q > rho': theta from samples
        uint32_t s_cnt = 0, r_idx = 0;
        if (q == 0) {
            theta = 0;  // re-check step: nothing to extract
        } else if (p.algo == SSSP_BELLMAN_FORD) {
            theta = kInf;
        } else if (p.algo == SSSP_DELTA_STAR || p.algo == SSSP_DELTA) {
            const uint64_t qmin = qmin_c;
            if (p.algo == SSSP_DELTA && k > 1) {
                // FinishCheck: advance the bucket unless the previous step
                // wrote a distance below its threshold
                const uint64_t umin = umin_c;
                if (!(umin < prev_theta)) delta_i += 1;
            }
            uint64_t cur = delta_i;
            theta = sat_mul(cur, p.param);
            if (qmin > theta) {  // skip empty buckets
                cur = qmin / p.param + ((qmin % p.param) != 0);
                theta = sat_mul(cur, p.param);
            }
            delta_i = p.algo == SSSP_DELTA_STAR ? cur + 1 : cur;
            prev_theta = theta;
        } else if (p.algo == SSSP_DIJKSTRA) {
            theta = qmin_c;  // min over Q (Table 2)
        } else {
            // rho-Stepping: theta is selected from s sampled keys in the first
            // Extract round below, with that round's loads in flight
            theta = kInf;
            // (warm-up steps: rho = warm_rho, at most 1024 samples, no
            // dense-step reduction, not counted as dense steps)
            const bool warm = k <= p.warm_steps;
            rho_sample = rho_sample_plan(q, n, warm ? p.warm_rho : p.param, warm ? 0xFFFFFFFFu : dense_seen,
                                         p.rho_reduced, &s_cnt, &r_idx, warm ? kWarmSamples : kMaxSamples);
            if ((uint64_t)q * 20ull > (uint64_t)n && !warm) ++dense_seen;
        }

        // SSSP_SOLVE_FUSED: a super-sparse step whose theta every block has
        // already (not one that samples it) and whose queue fits one Extract
        // round per block runs Extract and the relaxation block by block
        const uint64_t per_block_q = ((uint64_t)q + gridDim.x - 1) / gridDim.x;
        const bool fused = kFusedSteps && p.fre != nullptr && q != 0 && !rho_sample && (uint64_t)q * 20ull <= (uint64_t)n &&
                           per_block_q <= (uint64_t)kExtractCap;
        const uint4* fre_prev = p.fre + ((uint64_t)blockIdx.x * 2u + ((k + 1) & 1u)) * kExtractCap;
        uint32_t stc = 0;          // the warp's staged ids (next queue list)
        uint64_t lmin = kInf;      // smallest distance this thread wrote or re-queued
        uint32_t lupd = 0;         // successful WriteMin of this thread
        uint64_t f_cnt = 0, f_edg = 0, f_kmin = kInf;  // fused step: extracted, their edges, min kept key
        uint32_t fre_next = 0;

        if (fused) {
            // ---------------- Extract(theta) and relaxation, fused ----------------
            // The block's slice of Q_k (entry i held by thread i mod kBlock) is
            // extracted and relaxed by the block itself, with no device-wide
            // wait in between.  Other blocks' WriteMin may lower the distance
            // of an entry while it is examined.  A kept entry keeps its queue
            // bit and is examined again in the next step.  An extracted one is
            // recorded with the distance it is relaxed with; in the next step
            // (when every WriteMin of this step is visible) the block re-queues
            // those whose distance has dropped since: a WriteMin that found the
            // bit still set before this block cleared it queued nothing.
            const uint64_t r0 = (uint64_t)blockIdx.x * per_block_q;
            const uint32_t L = (uint32_t)(r0 >= q ? 0 : ((uint64_t)q - r0 < per_block_q ? (uint64_t)q - r0 : per_block_q));
            uint4* fre_cur = p.fre + ((uint64_t)blockIdx.x * 2u + (k & 1u)) * kExtractCap;
            const uint32_t small_deg = p.small_deg, cl = p.chunk_log2;
            uint32_t v[kExtractPer], ru[kExtractPer];
            uint64_t d[kExtractPer], rdu[kExtractPer];
            // ids, the previous step's records, then keys and current distances (all in flight)
#pragma unroll
            for (int j = 0; j < kExtractPer; ++j) {
                const uint32_t i = tid + (uint32_t)j * kBlock;
                v[j] = i < L ? ldcg32(&Qcur[r0 + i]) : 0u;
                const uint4 r = i < fre_L ? __ldcg(&fre_prev[i]) : make_uint4(0u, 0u, ~0u, ~0u);
                ru[j] = r.x;
                rdu[j] = (uint64_t)r.z | ((uint64_t)r.w << 32);
            }
            uint64_t sb0 = 0, se0 = 0;
#pragma unroll
            for (int j = 0; j < kExtractPer; ++j) {
                const uint32_t i = tid + (uint32_t)j * kBlock;
                d[j] = i < L ? ldcg64(&dist[v[j]]) : kInf;
            }
            if (tid < L) {
                sb0 = __ldg(&off[v[0]]);
                se0 = __ldg(&off[v[0] + 1]);
            }
            requeue_dropped(ru, rdu, dist, inq, stage, stc, lane, lmin);
            // (1) keep / extract; kept ids are staged for the next queue list
            uint32_t extm = 0;
#pragma unroll
            for (int j = 0; j < kExtractPer; ++j) {
                const uint32_t i = tid + (uint32_t)j * kBlock;
                if (i >= L) continue;
                if (d[j] <= theta) {
                    atomicAnd(&inq[v[j] >> 5], ~(1u << (v[j] & 31u)));
                    extm |= 1u << j;
                } else {
                    f_kmin = d[j] < f_kmin ? d[j] : f_kmin;
                }
            }
#pragma unroll
            for (int j = 0; j < kExtractPer; ++j) {
                const uint32_t i = tid + (uint32_t)j * kBlock;
                stage_push(i < L && !((extm >> j) & 1u), v[j], stage, stc, lane);
            }
            if (p.trace && k - 1 < p.trace_cap) {
                if (blockIdx.x == 0 && tid == 0) {
                    p.trace[k - 1].theta = theta;
                    p.trace[k - 1].t_relax_ns = global_timer_ns() - s_t_start;
                }
                if (tid == 0)
                    atomicMax((unsigned long long*)&p.trace[k - 1].t_extract_end_max, global_timer_ns() - s_t_start);
            }
            // (2) edge ranges (the first entry's was loaded with its key); the
            //     record for the next step's re-check
            uint64_t b[kExtractPer], e[kExtractPer];
#pragma unroll
            for (int j = 0; j < kExtractPer; ++j) {
                const uint32_t i = tid + (uint32_t)j * kBlock;
                b[j] = 0; e[j] = 0;
                if ((extm >> j) & 1u) {
                    b[j] = j == 0 ? sb0 : __ldg(&off[v[j]]);
                    e[j] = j == 0 ? se0 : __ldg(&off[v[j] + 1]);
                    // locally relaxed with this same distance: its edges are done
                    if (p.lrel && ldcg64(&p.lrel[v[j]]) == d[j]) e[j] = b[j];
                    f_cnt += 1;
                    f_edg += e[j] - b[j];
                    if (p.ext_count) p.ext_count[p.iperm ? p.iperm[v[j]] : v[j]] += 1u;
                }
                if (i < L) {
                    const uint64_t du = ((extm >> j) & 1u) ? d[j] : kInf;
                    fre_cur[i] = make_uint4(v[j], 0u, (uint32_t)du, (uint32_t)(du >> 32));
                }
            }
            // (3) out-degree <= small_deg: flattened over the warp's lanes
#pragma unroll
            for (int j = 0; j < kExtractPer; ++j) {
                const uint64_t deg = e[j] - b[j];
                const uint32_t sd = (((extm >> j) & 1u) && deg <= small_deg) ? (uint32_t)deg : 0u;
                if (stc > (uint32_t)(kStage - 256)) stage_flush(stage, stc, lane, &ctrl->qsize[nx], &ctrl->status, Qnext, n);
                relax_flat<true>(b[j], sd, d[j], edges, dist, inq, stage, stc, lane, lmin, lupd, true,
                                 &ctrl->qsize[nx], &ctrl->status, Qnext, n);
            }
            // (4) larger: the whole warp, one 2^chunk_log2-aligned piece at a time
#pragma unroll
            for (int j = 0; j < kExtractPer; ++j) {
                uint32_t many = __ballot_sync(FULL_MASK, ((extm >> j) & 1u) && e[j] - b[j] > small_deg);
                while (many) {
                    const int src = __ffs(many) - 1;
                    many &= many - 1;
                    const uint64_t sb = __shfl_sync(FULL_MASK, b[j], src);
                    const uint64_t se = __shfl_sync(FULL_MASK, e[j], src);
                    const uint64_t sdu = __shfl_sync(FULL_MASK, d[j], src);
                    const uint32_t su = __shfl_sync(FULL_MASK, v[j], src);
                    for (uint64_t cs = sb; cs < se;) {
                        const uint64_t nb = ((cs >> cl) + 1) << cl;
                        const uint64_t ce = se < nb ? se : nb;
                        const uint4 rec = make_rec(cs, ce - cs, su);
                        if (p.bidir)
                            relax_chunk<true, true>(rec, sdu, pairs, dist, inq, stage, stc, lane, lmin, lupd,
                                                    &ctrl->qsize[nx], &ctrl->status, Qnext, n);
                        else
                            relax_chunk<false, true>(rec, sdu, pairs, dist, inq, stage, stc, lane, lmin, lupd,
                                                     &ctrl->qsize[nx], &ctrl->status, Qnext, n);
                        cs = ce;
                    }
                }
            }
            fre_next = L;
        } else if (q != 0) {
        // ---------------- Extract(theta) ----------------
        // Q_k is cut into R x gridDim.x runs of equal length (at most
        // kExtractCap entries each); in round r, block b takes run r*gridDim.x+b.
        // Interleaving the runs gives every block a sample of the whole list:
        // the entries queued last (at the end of the list) are extracted far
        // more often than the ones kept from earlier steps, so contiguous
        // slices would leave the last blocks with most of the extractions.
        // Each round is staged in shared memory: (1) ids and
        // keys are loaded with every load of the round in flight; (2) the
        // extracted ids leave Q (queue bit cleared) and their edge ranges are
        // read; (3) one block scan and one atomic per output list reserve the
        // block's output ranges; (4) the staged records are written out.
        // Kept ids -> next queue list; extracted ids -> relaxation records
        // (degree <= small_deg: one record in fsmall; larger: one record per
        // 2^chunk_log2-aligned run of its edges in items).
        {
            const uint32_t small_deg = p.small_deg, cl = p.chunk_log2;
            const uint64_t chunk = 1ull << cl;
            uint4* s_rec = reinterpret_cast<uint4*>(s_dyn);                      // [kExtractCap]
            uint8_t* s_kind = s_dyn + (size_t)kExtractCap * sizeof(uint4);      // [kExtractCap]
            enum : uint8_t { kNone = 0, kKeep = 1, kSmall = 2, kChunked = 3, kNoEdges = 4 };
            uint64_t l_fcount = 0, l_fedges = 0, l_kmin = kInf;
            const uint64_t per_block = ((uint64_t)q + gridDim.x - 1) / gridDim.x;
            const uint32_t rounds = (uint32_t)((per_block + kExtractCap - 1) / kExtractCap);  // >= 1 (q >= 1)
            const uint64_t run = (per_block + rounds - 1) / rounds;                           // <= kExtractCap
            // every block runs the first round (possibly empty) so that every
            // block knows theta
            for (uint32_t rr = 0; rr < rounds; ++rr) {
                const uint64_t r0 = ((uint64_t)rr * gridDim.x + blockIdx.x) * run;
                const uint32_t L = (uint32_t)(r0 >= q ? 0 : ((uint64_t)q - r0) < run ? ((uint64_t)q - r0) : run);
                const bool select_now = rho_sample && rr == 0;
                const bool sel_in_regs = select_now && s_cnt <= (uint32_t)kBlock;
                // (1) ids, keys, and the keep / extract decision; in a sparse
                //     step (20 q <= n: few entries per thread, most of them
                //     extracted) the edge range of the first entry is loaded
                //     with its key instead of after the decision
                uint32_t extm = 0;  // bit j: entry j of this thread is extracted
                const bool spec_range = (uint64_t)q * 20ull <= (uint64_t)n;
                uint64_t sb0 = 0, se0 = 0;
                {
                    uint32_t v[kExtractPer];
                    uint64_t d[kExtractPer];
                    uint32_t sid = 0;
                    if (sel_in_regs && tid < s_cnt) sid = ldcg32(&Qcur[rho_sample_pos(p.seed, k, tid, q)]);
#pragma unroll
                    for (int j = 0; j < kExtractPer; ++j) {
                        const uint32_t i = tid + (uint32_t)j * kBlock;
                        v[j] = i < L ? ldcg32(&Qcur[r0 + i]) : 0u;
                    }
                    uint64_t skey = kInf;
                    if (sel_in_regs && tid < s_cnt) skey = ldcg64(&dist[sid]);
#pragma unroll
                    for (int j = 0; j < kExtractPer; ++j) {
                        const uint32_t i = tid + (uint32_t)j * kBlock;
                        d[j] = i < L ? ldcg64(&dist[v[j]]) : kInf;
                    }
                    if (spec_range && tid < L) {
                        sb0 = __ldg(&off[v[0]]);
                        se0 = __ldg(&off[v[0] + 1]);
                    }
                    if (select_now) {
                        // ExtDist of rho-Stepping (Table 2; Sec. 6; App. B)
                        if (!sel_in_regs) {
                            for (uint32_t j = tid; j < s_cnt; j += kBlock)
                                s_keys[j] = ldcg64(&dist[ldcg32(&Qcur[rho_sample_pos(p.seed, k, j, q)])]);
                            __syncthreads();
                        }
                        theta = block_select(skey, s_cnt, r_idx, s_keys, p.sample_cap, &s_err);
                        if (s_err && tid == 0) raise_error(&ctrl->bar, &ctrl->status, SSSP_ERR_INTERNAL);
                    }
#pragma unroll
                    for (int j = 0; j < kExtractPer; ++j) {
                        const uint32_t i = tid + (uint32_t)j * kBlock;
                        if (i >= L) continue;
                        if (d[j] <= theta) {
                            atomicAnd(&inq[v[j] >> 5], ~(1u << (v[j] & 31u)));
                            extm |= 1u << j;
                            s_rec[i] = make_uint4(v[j], (uint32_t)d[j], (uint32_t)(d[j] >> 32), 0u);
                        } else {
                            s_rec[i].x = v[j];
                            l_kmin = d[j] < l_kmin ? d[j] : l_kmin;
                        }
                    }
                }
                // (2) edge ranges of the extracted ids
                uint32_t nkeep = 0, nsmall = 0, nchunks = 0;
                {
                    uint64_t b[kExtractPer], e[kExtractPer];
#pragma unroll
                    for (int j = 0; j < kExtractPer; ++j) {
                        const uint32_t i = tid + (uint32_t)j * kBlock;
                        b[j] = 0; e[j] = 0;
                        if ((extm >> j) & 1u) {
                            const uint32_t u = s_rec[i].x;
                            if (j == 0 && spec_range) {
                                b[j] = sb0;
                                e[j] = se0;
                            } else {
                                b[j] = __ldg(&off[u]);
                                e[j] = __ldg(&off[u + 1]);
                            }
                            // locally relaxed with this same distance: its edges are done
                            if (p.lrel) {
                                const uint4 r = s_rec[i];
                                if (ldcg64(&p.lrel[u]) == ((uint64_t)r.y | ((uint64_t)r.z << 32))) e[j] = b[j];
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < kExtractPer; ++j) {
                        const uint32_t i = tid + (uint32_t)j * kBlock;
                        if (i >= L) continue;
                        if (!((extm >> j) & 1u)) { ++nkeep; continue; }
                        const uint4 r = s_rec[i];
                        const uint64_t deg = e[j] - b[j];
                        l_fcount += 1;
                        l_fedges += deg;
                        if (p.ext_count) p.ext_count[p.iperm ? p.iperm[r.x] : r.x] += 1u;
                        if (deg == 0) {
                            s_kind[i] = kNoEdges;
                        } else if (deg <= small_deg) {
                            s_kind[i] = kSmall;
                            s_rec[i] = make_rec(b[j], deg, (uint64_t)r.y | ((uint64_t)r.z << 32));
                            ++nsmall;
                        } else {
                            s_kind[i] = kChunked;
                            s_rec[i] = make_uint4(r.x, (uint32_t)b[j], (uint32_t)(b[j] >> 32),
                                                  deg < 0xFFFFFFFFull ? (uint32_t)deg : 0xFFFFFFFFu);
                            nchunks += (uint32_t)(((e[j] - 1) >> cl) - (b[j] >> cl) + 1);
                        }
                    }
                }
                // (3) block scan of the (keep, small, chunks) counts, packed
                //     16|16|32 bits; one atomic per output list
                const uint64_t packed = (uint64_t)nkeep | ((uint64_t)nsmall << 16) | ((uint64_t)nchunks << 32);
                uint64_t tot;
                const uint64_t ex = block_excl_scan64(packed, s_tmp, &tot);
                if (tid == 0) {
                    const uint32_t tk = (uint32_t)(tot & 0xFFFFu), ts = (uint32_t)((tot >> 16) & 0xFFFFu);
                    const uint32_t tc = (uint32_t)(tot >> 32);
                    s_base[0] = tk ? atomicAdd(&ctrl->qsize[nx], tk) : 0u;
                    s_base[1] = ts ? atomicAdd(&ctrl->fsmall[c], ts) : 0u;
                    s_base[2] = tc ? atomicAdd(&ctrl->fchunk[c], tc) : 0u;
                    if ((uint64_t)s_base[0] + tk > n || (uint64_t)s_base[1] + ts > p.fsmall_cap ||
                        (uint64_t)s_base[2] + tc > p.item_cap)
                        raise_error(&ctrl->bar, &ctrl->status, SSSP_ERR_INTERNAL);
                }
                __syncthreads();
                uint32_t pk = s_base[0] + (uint32_t)(ex & 0xFFFFu);
                uint64_t ps = (uint64_t)s_base[1] + ((ex >> 16) & 0xFFFFu);
                uint64_t pc = (uint64_t)s_base[2] + (ex >> 32);
                // (4) write the staged entries
#pragma unroll
                for (int j = 0; j < kExtractPer; ++j) {
                    const uint32_t i = tid + (uint32_t)j * kBlock;
                    const uint8_t kd = i < L ? (((extm >> j) & 1u) ? s_kind[i] : (uint8_t)kKeep) : (uint8_t)kNone;
                    const uint4 r = (kd == kKeep || kd == kSmall || kd == kChunked) ? s_rec[i] : make_uint4(0, 0, 0, 0);
                    uint64_t bj = 0, ej = 0;
                    if (kd == kChunked) {
                        bj = (uint64_t)r.y | ((uint64_t)r.z << 32);
                        ej = r.w != 0xFFFFFFFFu ? bj + r.w : __ldg(&off[r.x + 1]);
                    }
                    const uint64_t nch = kd == kChunked ? ((ej - 1) >> cl) - (bj >> cl) + 1 : 0;
                    if (kd == kKeep) {
                        if (pk < n) Qnext[pk] = r.x;
                        ++pk;
                    } else if (kd == kSmall) {
                        if (ps < p.fsmall_cap) p.fsmall[ps] = r;
                        ++ps;
                    } else if (kd == kChunked && nch <= 4) {
                        for (uint64_t c0 = (bj >> cl) << cl; c0 < ej; c0 += chunk, ++pc) {
                            const uint64_t cs = bj > c0 ? bj : c0;
                            const uint64_t ce = ej < c0 + chunk ? ej : c0 + chunk;
                            if (pc < p.item_cap) p.items[pc] = make_rec(cs, ce - cs, r.x);
                        }
                    }
                    // vertices with many chunks: the whole warp writes their records
                    uint32_t many = __ballot_sync(FULL_MASK, kd == kChunked && nch > 4);
                    while (many) {
                        const int src = __ffs(many) - 1;
                        many &= many - 1;
                        const uint64_t sb = __shfl_sync(FULL_MASK, bj, src);
                        const uint64_t se = __shfl_sync(FULL_MASK, ej, src);
                        const uint32_t sv = __shfl_sync(FULL_MASK, r.x, src);
                        const uint64_t sp = __shfl_sync(FULL_MASK, pc, src);
                        const uint64_t sn = ((se - 1) >> cl) - (sb >> cl) + 1;
                        for (uint64_t t = lane; t < sn; t += 32) {
                            const uint64_t c0 = ((sb >> cl) + t) << cl;
                            const uint64_t cs = sb > c0 ? sb : c0;
                            const uint64_t ce = se < c0 + chunk ? se : c0 + chunk;
                            if (sp + t < p.item_cap) p.items[sp + t] = make_rec(cs, ce - cs, sv);
                        }
                    }
                    if (kd == kChunked && nch > 4) pc += nch;
                }
                __syncthreads();  // s_tmp / s_base / staging reuse
            }
            if (blockIdx.x == 0 && tid == 0 && p.trace && k - 1 < p.trace_cap) p.trace[k - 1].theta = theta;
            uint64_t bf = l_fcount, be = l_fedges, bm = l_kmin;
            block_reduce_2add_min(bf, be, bm, s_tmp);
            if (tid == 0) {
                if (bf) atomicAdd(&ctrl->fcount[c], (unsigned int)bf);
                if (be) atomicAdd(&ctrl->fedges[c], (unsigned long long)be);
                if (algo_tracks_qmin(p.algo) && bm != kInf) atomicMin(&ctrl->qmin[nx], (unsigned long long)bm);
            }
        }
        if (p.trace && tid == 0 && k - 1 < p.trace_cap)
            atomicMax((unsigned long long*)&p.trace[k - 1].t_extract_end_max, global_timer_ns() - s_t_start);
        if (!grid_sync_err(&ctrl->bar, &ctrl->status, &s_bar_target, p.timeout_ns)) break;
        }

        // ---------------- relax the out-edges of F ----------------
        if (!fused && blockIdx.x == 0 && tid == 0 && p.trace && k - 1 < p.trace_cap)
            p.trace[k - 1].t_relax_ns = global_timer_ns() - s_t_start;
        if (kFusedSteps && !fused && fre_L != 0) {
            // the previous step was fused: re-queue its extractions whose
            // distance dropped since (see the fused step)
            uint32_t ru[kExtractPer];
            uint64_t rdu[kExtractPer];
#pragma unroll
            for (int j = 0; j < kExtractPer; ++j) {
                const uint32_t i = tid + (uint32_t)j * kBlock;
                const uint4 r = i < fre_L ? __ldcg(&fre_prev[i]) : make_uint4(0u, 0u, ~0u, ~0u);
                ru[j] = r.x;
                rdu[j] = (uint64_t)r.z | ((uint64_t)r.w << 32);
            }
            requeue_dropped(ru, rdu, dist, inq, stage, stc, lane, lmin);
        }
        if (!fused) {
            // the warp's first records are loaded together with the record
            // counts (within the arrays' capacity; used only if below the count)
            const uint64_t i_first = (uint64_t)gwarp * 32u + lane;
            const uint4 spec_small = i_first < p.fsmall_cap ? __ldcg(&p.fsmall[i_first]) : make_uint4(0, 0, 0, 0);
            const uint4 spec_chunk = gwarp < p.item_cap ? __ldcg(&p.items[gwarp]) : make_uint4(0, 0, 0, 0);
            uint64_t fs = ldcg32(&ctrl->fsmall[c]);
            fs = fs < p.fsmall_cap ? fs : p.fsmall_cap;
            uint64_t fc = ldcg32(&ctrl->fchunk[c]);
            fc = fc < p.item_cap ? fc : p.item_cap;

            // (a) low-degree vertices: 32 records per warp, edges flattened across lanes
            const uint64_t ngroups = (fs + 31u) >> 5;
            uint64_t g = gwarp;
            uint4 rnext = (g < ngroups && i_first < fs) ? spec_small : make_uint4(0, 0, 0, 0);
            for (; g < ngroups; g += nwarps) {
                const uint4 rec = rnext;
                const uint64_t gn = g + nwarps;  // prefetch the next group's records
                rnext = (gn < ngroups && gn * 32u + lane < fs) ? __ldcg(&p.fsmall[gn * 32u + lane])
                                                              : make_uint4(0, 0, 0, 0);
                relax_flat<true>(rec_start(rec), rec_len(rec), rec_du(rec), edges, dist, inq, stage, stc, lane,
                                 lmin, lupd, true, &ctrl->qsize[nx], &ctrl->status, Qnext, n);
            }

            // (b) higher-degree vertices: one warp per chunk record; the next
            //     record is prefetched while the current chunk is relaxed, and
            //     delta[u] is read when the chunk starts (Algorithm 1 reads it at
            //     relaxation time; the freshest value wastes the fewest relaxations)
            {
                uint64_t it = gwarp;
                uint4 rn = it < fc ? spec_chunk : make_uint4(0, 0, 0, 0);
                for (; it < fc; it += nwarps) {
                    const uint4 rc = rn;
                    const uint64_t nit = it + nwarps;
                    rn = nit < fc ? __ldcg(&p.items[nit]) : make_uint4(0, 0, 0, 0);
                    const uint64_t du = ldcg64(&dist[rc.z]);
                    if (p.bidir)
                        relax_chunk<true, true>(rc, du, pairs, dist, inq, stage, stc, lane, lmin, lupd,
                                                &ctrl->qsize[nx], &ctrl->status, Qnext, n);
                    else
                        relax_chunk<false, true>(rc, du, pairs, dist, inq, stage, stc, lane, lmin, lupd,
                                                 &ctrl->qsize[nx], &ctrl->status, Qnext, n);
                    if (stc > (uint32_t)(kStage - 256)) stage_flush(stage, stc, lane, &ctrl->qsize[nx], &ctrl->status, Qnext, n);
                }
            }
        }
        {
            // (d) super-sparse steps (Sec. 6, local BFS): keep relaxing from the
            //     vertices this warp has just queued while they are within theta
            //     (after a fused step without the device-wide degree check)
            uint64_t ledg = 0;
            if (p.local_budget != 0 && q != 0 && (uint64_t)q * 20ull <= (uint64_t)n) {
                bool go = fused;
                if (!fused) {
                    const uint64_t fcnt = ldcg32(&ctrl->fcount[c]);
                    const uint64_t fed = ldcg64((const uint64_t*)&ctrl->fedges[c]);
                    go = fed < 20ull * fcnt;
                }
                if (go)
                    ledg = local_relax(theta, p.local_budget, off, edges, dist, inq, stage, stc, lane, lmin, lupd,
                                       &ctrl->qsize[nx], &ctrl->status, Qnext, n, p.lrel);
            }

            // (c) block-aggregated flush of what is left in the warps' staging,
            //     together with the step's counters (a fused step's Extract
            //     counters too): warp sums by shuffles, then one block phase
            //     (warp 0) for the flush reservation and the counters
            uint64_t sums[4] = {lupd, ledg, f_cnt, f_edg}, mins[2] = {lmin, f_kmin};
            warp_reduce_4add_2min(sums, mins);
            if (lane == 0) {
                s_wcnt[wid] = stc;
#pragma unroll
                for (int t = 0; t < 4; ++t) s_tmp[t * kWarps + wid] = sums[t];
#pragma unroll
                for (int t = 0; t < 2; ++t) s_tmp[(4 + t) * kWarps + wid] = mins[t];
            }
            __syncthreads();
            if (wid == 0) {
                const uint32_t cnt = lane < (uint32_t)kWarps ? s_wcnt[lane] : 0u;
                const uint32_t incl = (uint32_t)warp_incl_scan64(cnt, lane);
                uint32_t tot = __shfl_sync(FULL_MASK, incl, 31);
                if (lane < (uint32_t)kWarps) s_wcnt[lane] = incl - cnt;
#pragma unroll
                for (int t = 0; t < 4; ++t) sums[t] = lane < (uint32_t)kWarps ? s_tmp[t * kWarps + lane] : 0ull;
#pragma unroll
                for (int t = 0; t < 2; ++t) mins[t] = lane < (uint32_t)kWarps ? s_tmp[(4 + t) * kWarps + lane] : kInf;
                warp_reduce_4add_2min(sums, mins);
                if (lane == 0) {
                    const uint32_t base = tot ? atomicAdd(&ctrl->qsize[nx], tot) : 0u;
                    if ((uint64_t)base + tot > (uint64_t)n) { raise_error(&ctrl->bar, &ctrl->status, SSSP_ERR_INTERNAL); tot = 0; }
                    s_base[0] = base;
                    s_base[1] = tot;
                    const uint64_t bu = sums[0], bl = sums[1], bf = sums[2], be = sums[3], bm = mins[0], bk = mins[1];
                    if (bf) atomicAdd(&ctrl->fcount[c], (unsigned int)bf);
                    if (be) atomicAdd(&ctrl->fedges[c], (unsigned long long)be);
                    if (algo_tracks_qmin(p.algo) && bk != kInf) atomicMin(&ctrl->qmin[nx], (unsigned long long)bk);
                    if (bu) atomicAdd(&ctrl->updates[c], (unsigned long long)bu);
                    if (bl) atomicAdd(&ctrl->ledges[c], (unsigned long long)bl);
                    if (algo_tracks_qmin(p.algo) && bm != kInf) {
                        atomicMin(&ctrl->qmin[nx], (unsigned long long)bm);
                        atomicMin(&ctrl->umin[nx], (unsigned long long)bm);
                    }
                    if (p.trace && k - 1 < p.trace_cap) {
                        const unsigned long long now = global_timer_ns() - s_t_start;
                        atomicMin((unsigned long long*)&p.trace[k - 1].t_relax_end_min, now);
                        atomicMax((unsigned long long*)&p.trace[k - 1].t_relax_end_max, now);
                    }
                    // step k-1 is complete: fold its counters into the totals and
                    // recycle its slot (reused for Q_{k+2} from the next step on)
                    if (blockIdx.x == 0) fold_step(p, ctrl, pv, k - 1);
                }
            }
            __syncthreads();
            if (s_base[1] != 0) {
                const uint32_t wb = s_base[0] + s_wcnt[wid];
                for (uint32_t i = lane; i < stc; i += 32) Qnext[wb + i] = stage[i];
            }
        }
        if (!grid_sync_err(&ctrl->bar, &ctrl->status, &s_bar_target, p.timeout_ns)) break;
        prev_fused = fused;
        fre_L = fre_next;
    }

    // relabelled graph: distances back in the caller's ids
    if (p.perm)
        for (uint64_t i = gtid; i < n; i += gthreads) p.dist_out[i] = ldcg64(&dist[__ldg(&p.perm[i])]);
    if (blockIdx.x == 0 && tid == 0) {
        ctrl->steps = k - 1;
        if (p.stats_out) {
            sssp_stats so;
            so.steps = k - 1; so.queued = ctrl->queued; so.extracted = ctrl->extracted;
            so.edges = ctrl->edges; so.updates = ctrl->updates_total;
            so.status = *reinterpret_cast<volatile int*>(&ctrl->status); so.grid = 0;
            *p.stats_out = so;
        }
    }
}

const void* solve_kernel_ptr() { return reinterpret_cast<const void*>(&solve_kernel); }
int solve_kernel_threads() { return kBlock; }
unsigned int solve_kernel_smem() { return kSolveDynSmem; }

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
                                                               uint32_t dense_before, uint32_t reduced,
                                                               uint32_t max_samples, uint64_t* theta_out,
                                                               uint32_t* err_out, uint32_t cap)
{
    extern __shared__ uint64_t s_keys[];
    __shared__ int s_e;
    if (threadIdx.x == 0) s_e = 0;
    __syncthreads();
    const uint64_t th = rho_extdist_block(queue, q, dist, n, rho, seed, step, dense_before, reduced, s_keys, cap,
                                          &s_e, max_samples);
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
                                 uint32_t reduced, uint32_t max_samples, uint64_t* theta_out, uint32_t* err_out,
                                 cudaStream_t st)
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
                                                                    dense_before, reduced, max_samples, theta_out,
                                                                    err_out, cap);
    return cudaGetLastError();
}

}  // namespace sssp
