// sssp_msbatch.cu -- k <= 64 sources on one graph with one shared edge scan
// per step (batched solves, "many sources on one graph").
//
// Each instance runs the stepping loop of Algorithm 1 with its own source,
// parameter and threshold theta_i (Table 2), exactly as k separate solves
// would; what the instances share is the memory traffic:
//
//   delta     vertex-major rows, D[v*R + i] = delta_i[v] (R = k rounded up to
//             a multiple of 4, so a row's 32-byte sectors each hold four
//             instances): one vertex's distances for every instance are
//             adjacent, and a warp reads or updates them with coalesced
//             accesses.
//   queue     one union list of the vertices queued by any instance and a
//             64-bit mask per vertex (bit i: v is in instance i's LaB-PQ,
//             Sec. 3.1 / 4.3).  A vertex enters the list when its mask goes
//             from zero to non-zero, so it appears at most once.
//   records   an extracted vertex u yields records of <= 32 of its out-edges
//             carrying the mask F(u) of the instances that extracted u; the
//             relaxation reads each such edge once per step for every
//             instance in F(u).
//
// Per step:
//   phase T   |Q_i| and theta_i per instance (rho-Stepping: Sec. 6 sampling,
//             drawn from the union list and kept where the vertex is in Q_i)
//   phase E   Extract: every union entry's row is compared with the theta_i
//             of the instances whose bit it carries (lanes own instance
//             pairs); kept bits stay in the mask, extracted ones form F(u)
//   phase R   relaxation of the records: WriteMin on D[v*R + i] for the
//             instances in F(u), then one atomicOr of the improved bits on
//             v's mask (Update); v joins the next union list when its mask
//             was empty.  Masks with few instances are relaxed edge-parallel
//             (lanes = edges), others instance-parallel (lanes = instance
//             pairs, one coalesced row access per edge).
// Grid barriers separate the phases (Extract is not concurrent with Update,
// Sec. 3.1).  The distances equal k single solves; the thresholds of
// rho-Stepping come from a different sample draw than a single solve's, so
// step counts differ.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "sssp_internal.h"
#include "sssp_device.cuh"

namespace sssp {

constexpr uint32_t kMsMax = 64;        // instances per shared-scan launch
constexpr uint32_t kMsRec = 32;        // edges per relaxation record
constexpr uint32_t kMsSparse = 4;      // masks with at most this many instances: edge-parallel relaxation
#ifndef SSSP_MS_BLOCK
#define SSSP_MS_BLOCK 1024
#endif
constexpr int kMsBlock = SSSP_MS_BLOCK;  // threads per block
constexpr int kMsWarps = kMsBlock / 32;
constexpr uint32_t kMsDraws = 64u * 1024u;  // rho sampler: union-list positions drawn per instance and step
constexpr uint32_t kMsDynSmem = (uint32_t)kMsWarps * kStage * 4u > kMaxSamples * 8u
                                    ? (uint32_t)kMsWarps * kStage * 4u : kMaxSamples * 8u;

struct MsInst {                       // per instance; zeroed before the launch
    unsigned int qsize[3];            // |Q_i| of step k in slot k%3
    unsigned int dense_seen;          // rho-Stepping: dense steps so far
    unsigned long long qmin[3];       // min over Q_i of delta_i (slot k%3)
    unsigned long long fext[3], fedges[3], fupd[3];  // Extract / relaxation counters of step k (slot k%3)
    unsigned long long theta;         // theta_i of the current step
    unsigned long long delta_i;       // Delta*-Stepping bucket index
    unsigned long long queued, extracted, edges, updates;  // totals
    unsigned int last_step;           // steps the instance took
    unsigned int steps_run;           // steps run so far (rho-Stepping warm-up)
};

struct MsCtrl {
    unsigned long long bar;
    int status;
    unsigned int pad;
    unsigned int usize[3];            // union list size of step k (slot k%3)
    unsigned int nsmall[3];           // low-degree records of step k (slot k%3)
    unsigned int nbig[3];             // records of higher-degree vertices of step k (slot k%3)
    unsigned long long steps;
};

struct MsParams {
    const uint64_t* off;
    const uint2* edges;
    uint32_t n;
    uint32_t K;                       // instances
    uint32_t R;                       // row stride of D (multiple of 4, >= K)
    uint32_t rho_reduced;
    uint32_t warm_steps;              // rho-Stepping: each instance's first warm_steps steps use
    uint64_t warm_rho;                //   rho = warm_rho (at most 1024 samples, no dense reduction)
    uint64_t* D;                      // [n][R]
    uint64_t* QM;                     // [n] queue masks
    uint32_t* qa;                     // union lists [n]
    uint32_t* qb;
    uint4* rec;                       // records: x = u, y = edge count, z|w = first edge; flattened
                                      // records in [0, small_cap), per-warp records after it
    uint64_t* fm;                     // record masks F(u)
    uint64_t small_cap;               // flattened records (vertices of degree 1..32, <= kMsSparse instances)
    uint64_t big_cap;                 // per-warp records (32 edges each)
    MsInst* inst;
    MsCtrl* ctrl;
    const uint32_t* src;              // [K] sources (ids of the graph the kernel runs on)
    const uint64_t* param;            // [K]
    int algo;
    uint32_t sample_cap;
    uint32_t bidir;                   // bidirectional relaxation (symmetric graph, Sec. 6)
    uint64_t timeout_ns;
    uint64_t solve_timeout_ns;
    uint64_t* const* dist_out;        // [K] caller's outputs (caller's ids)
    const uint32_t* perm;             // caller id -> kernel id, or null
};

struct MsSmem {
    uint64_t tmp[3 * kMsWarps];
    uint32_t base[3];
    unsigned long long bar_target;
    unsigned long long t_start;
    unsigned long long cnt[4][kMsMax];   // per-instance block sums of the phase
    unsigned long long mn[kMsMax];       // per-instance block minima
    unsigned int scnt;
    int err;
};

// ---- block helpers for kMsBlock threads ----
__device__ __forceinline__ uint64_t ms_excl_scan64(uint64_t x, uint64_t* s_tmp, uint64_t* total)
{
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint64_t incl = warp_incl_scan64(x, lane);
    if (lane == 31) s_tmp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint64_t v = lane < (uint32_t)kMsWarps ? s_tmp[lane] : 0;
        v = warp_incl_scan64(v, lane);
        if (lane < (uint32_t)kMsWarps) s_tmp[lane] = v;
    }
    __syncthreads();
    *total = s_tmp[kMsWarps - 1];
    return (wid ? s_tmp[wid - 1] : 0) + incl - x;
}

// 64-bit OR over the warp of (bits2 << 2*lane): lane l contributes the two
// bits of instances 2l and 2l+1.
__device__ __forceinline__ uint64_t lane_pairs_or(uint32_t bits2, uint32_t lane)
{
    const uint32_t lo = __reduce_or_sync(FULL_MASK, lane < 16 ? bits2 << (2 * lane) : 0u);
    const uint32_t hi = __reduce_or_sync(FULL_MASK, lane >= 16 ? bits2 << (2 * lane - 32) : 0u);
    return (uint64_t)lo | ((uint64_t)hi << 32);
}

__device__ __forceinline__ ulonglong2 ld_pair_cg(const uint64_t* p)
{
    return __ldcg(reinterpret_cast<const ulonglong2*>(p));
}

// Flush the per-lane sums of the instances a lane owns (2l, 2l+1) into the
// block's per-instance counters (shared-memory atomics).
__device__ __forceinline__ void ms_lane_add(MsSmem& S, int which, uint32_t lane, uint64_t a0, uint64_t a1)
{
    if (a0) atomicAdd(&S.cnt[which][2 * lane], (unsigned long long)a0);
    if (a1) atomicAdd(&S.cnt[which][2 * lane + 1], (unsigned long long)a1);
}

// ---------------------------------------------------------------------------
// phase T: per-instance bookkeeping and theta_i (instances spread over blocks)
// ---------------------------------------------------------------------------
__device__ void ms_phase_T(const MsParams& p, uint64_t k, uint32_t U, MsSmem& S, uint64_t* s_keys)
{
    const uint32_t tid = threadIdx.x;
    const int c = (int)(k % 3), pv = (int)((k + 2) % 3);
    const uint32_t* Qcur = (k & 1) ? p.qa : p.qb;
    for (uint32_t i = blockIdx.x; i < p.K; i += gridDim.x) {
        MsInst* I = &p.inst[i];
        const uint32_t q = ldcg32(&I->qsize[c]);
        if (tid == 0) {
            if (k > 1) {
                I->queued += ldcg32(&I->qsize[pv]);
                I->extracted += ldcg64((const uint64_t*)&I->fext[pv]);
                I->edges += ldcg64((const uint64_t*)&I->fedges[pv]);
                I->updates += ldcg64((const uint64_t*)&I->fupd[pv]);
            }
            if (q == 0 && I->last_step == 0) I->last_step = (unsigned)(k - 1);
            I->qsize[pv] = 0; I->qmin[pv] = kInf; I->fext[pv] = 0; I->fedges[pv] = 0; I->fupd[pv] = 0;
        }
        uint64_t theta = kInf;
        if (q != 0 && p.algo == SSSP_DELTA_STAR) {
            const uint64_t prm = p.param[i];
            const uint64_t qmin = ldcg64((const uint64_t*)&I->qmin[c]);
            uint64_t cur = ldcg64((const uint64_t*)&I->delta_i);
            cur = cur ? cur : 1;
            theta = sat_mul(cur, prm);
            if (qmin > theta) {  // skip empty buckets
                cur = qmin / prm + ((qmin % prm) != 0);
                theta = sat_mul(cur, prm);
            }
            __syncthreads();
            if (tid == 0) I->delta_i = cur + 1;
        } else if (q != 0 && p.algo == SSSP_RHO) {
            const uint32_t dense = ldcg32(&I->dense_seen);
            // the instance's own step count: its first warm_steps steps use
            // rho = warm_rho, without the dense-step reduction
            const bool warm = ldcg32(&I->steps_run) < p.warm_steps;
            const uint64_t rho_i = warm ? p.warm_rho : p.param[i];
            uint64_t rho_eff = rho_i;
            if (!warm && (uint64_t)q * 20ull > (uint64_t)p.n && dense < p.rho_reduced)
                rho_eff = rho_eff / 10 ? rho_eff / 10 : 1;
            uint32_t s = 0, r = 0;
            if (rho_sample_plan(q, p.n, rho_i, warm ? 0xFFFFFFFFu : dense, p.rho_reduced, &s, &r,
                                warm ? kWarmSamples : kMaxSamples)) {
                // uniform samples of Q_i: positions of the union list drawn
                // uniformly (splitmix64, multiply-high), kept where the
                // vertex carries bit i; at most kMsDraws draws
                if (tid == 0) S.scnt = 0;
                __syncthreads();
                const uint64_t seed = 0x2105061450000000ull ^ (uint64_t)p.src[i];
                for (uint32_t b0 = 0; b0 < kMsDraws; b0 += kMsBlock) {
                    const uint32_t j = b0 + tid;
                    const uint32_t pos = (uint32_t)__umul64hi(splitmix64_at(seed, (k << 32) | j), (uint64_t)U);
                    const uint32_t v = ldcg32(&Qcur[pos]);
                    if ((ldcg64(&p.QM[v]) >> i) & 1ull) {
                        const uint32_t slot = atomicAdd(&S.scnt, 1u);
                        if (slot < s) s_keys[slot] = ldcg64(&p.D[(uint64_t)v * p.R + i]);
                    }
                    __syncthreads();
                    if (S.scnt >= s) break;  // block-uniform
                    __syncthreads();
                }
                const uint32_t got = S.scnt < s ? S.scnt : s;
                __syncthreads();
                if (got > 0) {
                    // the rank of the plan, scaled to the keys drawn: floor(rho' s' / q)
                    uint64_t r2 = rho_eff * (uint64_t)got / (uint64_t)q;
                    if (r2 > got - 1) r2 = got - 1;
                    const uint64_t x = tid < got ? s_keys[tid] : kInf;
                    theta = block_select(x, got, (uint32_t)r2, s_keys, p.sample_cap, &S.err);
                }
                (void)r;
            }
            if (tid == 0 && (uint64_t)q * 20ull > (uint64_t)p.n && !warm) I->dense_seen = dense + 1;
        }
        if (tid == 0) {
            I->theta = theta;
            if (q != 0) I->steps_run += 1;
        }
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------
// phase E: Extract over the union list.  A block round covers kMsBlock
// entries; lane t of a warp owns entry t of the warp's 32 for the output (keep
// flag, record count), and the rows are tested four entries at a time with
// lane l owning instances 2l and 2l+1.
// ---------------------------------------------------------------------------
__device__ void ms_phase_E(const MsParams& p, uint64_t k, uint32_t U, MsSmem& S)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
    const int c = (int)(k % 3), nx = (int)((k + 1) % 3);
    const uint32_t* Qcur = (k & 1) ? p.qa : p.qb;
    uint32_t* Qnext = (k & 1) ? p.qb : p.qa;
    const uint32_t R = p.R;
    const uint32_t i0 = 2 * lane, i1 = 2 * lane + 1;
    const uint64_t th0 = i0 < p.K ? ldcg64((const uint64_t*)&p.inst[i0].theta) : 0ull;
    const uint64_t th1 = i1 < p.K ? ldcg64((const uint64_t*)&p.inst[i1].theta) : 0ull;
    uint64_t keep0 = 0, keep1 = 0, ext0 = 0, ext1 = 0, edg0 = 0, edg1 = 0, kmin0 = kInf, kmin1 = kInf;
    for (uint64_t r0 = (uint64_t)blockIdx.x * kMsBlock; r0 < U; r0 += (uint64_t)gridDim.x * kMsBlock) {
        const uint64_t my_idx = r0 + (uint64_t)wid * 32u + lane;
        const bool valid = my_idx < U;
        uint32_t my_v = 0;
        uint64_t my_qm = 0, my_b = 0, my_e = 0, my_fm = 0;
        if (valid) my_v = ldcg32(&Qcur[my_idx]);
        if (valid) {
            my_qm = ldcg64(&p.QM[my_v]);
            my_b = __ldg(&p.off[my_v]);
            my_e = __ldg(&p.off[my_v + 1]);
        }
        const uint32_t my_deg = (uint32_t)(my_e - my_b);
        const uint32_t live = __ballot_sync(FULL_MASK, valid);
        for (uint32_t j0 = 0; j0 < 32; j0 += 4) {
            if (((live >> j0) & 0xFu) == 0) break;  // warp-uniform: the entries are a prefix
            uint32_t vv[4], dg[4];
            uint64_t qm[4];
            ulonglong2 dv[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                vv[t] = __shfl_sync(FULL_MASK, my_v, j0 + t);
                qm[t] = __shfl_sync(FULL_MASK, my_qm, j0 + t);
                dg[t] = __shfl_sync(FULL_MASK, my_deg, j0 + t);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t b2 = (uint32_t)(qm[t] >> i0) & 3u;
                dv[t] = b2 ? ld_pair_cg(&p.D[(uint64_t)vv[t] * R + i0]) : make_ulonglong2(kInf, kInf);
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t b2 = (uint32_t)(qm[t] >> i0) & 3u;
                uint32_t e2 = 0;
                if ((b2 & 1u) && dv[t].x <= th0) e2 |= 1u;
                if ((b2 & 2u) && dv[t].y <= th1) e2 |= 2u;
                const uint32_t k2 = b2 & ~e2;
                if (k2 & 1u) { ++keep0; kmin0 = dv[t].x < kmin0 ? dv[t].x : kmin0; }
                if (k2 & 2u) { ++keep1; kmin1 = dv[t].y < kmin1 ? dv[t].y : kmin1; }
                if (e2 & 1u) { ++ext0; edg0 += dg[t]; }
                if (e2 & 2u) { ++ext1; edg1 += dg[t]; }
                const uint64_t fmt = lane_pairs_or(e2, lane);
                if (lane == j0 + (uint32_t)t) my_fm = fmt;
            }
        }
        const uint64_t new_qm = my_qm & ~my_fm;
        if (valid && my_fm) p.QM[my_v] = new_qm;  // no other writer in this phase
        const bool keep = valid && new_qm != 0;
        // degree 1..32 and at most kMsSparse instances: a flattened record;
        // otherwise 32-edge records relaxed one per warp (lanes then cover
        // instance pairs when the mask is wide)
        const bool small = valid && my_fm && my_deg >= 1 && my_deg <= kMsRec && __popcll(my_fm) <= (int)kMsSparse;
        const uint64_t nrec = (valid && my_fm && !small) ? ((uint64_t)my_deg + kMsRec - 1) / kMsRec : 0;
        uint64_t tot;
        const uint64_t ex = ms_excl_scan64((uint64_t)(keep ? 1u : 0u) | ((uint64_t)(small ? 1u : 0u) << 16) |
                                           (nrec << 32), S.tmp, &tot);
        if (tid == 0) {
            const uint32_t tk = (uint32_t)(tot & 0xFFFFu), ts = (uint32_t)((tot >> 16) & 0xFFFFu);
            const uint64_t tr = tot >> 32;
            S.base[0] = tk ? atomicAdd(&p.ctrl->usize[nx], tk) : 0u;
            S.base[1] = ts ? atomicAdd(&p.ctrl->nsmall[c], ts) : 0u;
            S.base[2] = tr ? atomicAdd(&p.ctrl->nbig[c], (unsigned int)tr) : 0u;
            if ((uint64_t)S.base[0] + tk > p.n || (uint64_t)S.base[1] + ts > p.small_cap ||
                (uint64_t)S.base[2] + tr > p.big_cap)
                raise_error(&p.ctrl->bar, &p.ctrl->status, SSSP_ERR_INTERNAL);
        }
        __syncthreads();
        const uint64_t pk = (uint64_t)S.base[0] + (ex & 0xFFFFu);
        const uint64_t ps = (uint64_t)S.base[1] + ((ex >> 16) & 0xFFFFu);
        uint64_t pr = (uint64_t)S.base[2] + (ex >> 32);
        if (keep && pk < p.n) Qnext[pk] = my_v;
        if (small && ps < p.small_cap) {
            p.rec[ps] = make_uint4(my_v, my_deg, (uint32_t)my_b, (uint32_t)(my_b >> 32));
            p.fm[ps] = my_fm;
        }
        if (nrec > 0 && nrec <= 4) {
            for (uint64_t j = 0; j < nrec; ++j, ++pr) {
                if (pr >= p.big_cap) break;
                const uint64_t st = my_b + j * kMsRec;
                const uint32_t len = (uint32_t)((my_e - st) < kMsRec ? (my_e - st) : kMsRec);
                p.rec[p.small_cap + pr] = make_uint4(my_v, len, (uint32_t)st, (uint32_t)(st >> 32));
                p.fm[p.small_cap + pr] = my_fm;
            }
        }
        // vertices with many records: the whole warp writes them
        uint32_t many = __ballot_sync(FULL_MASK, nrec > 4);
        while (many) {
            const int sl = __ffs(many) - 1;
            many &= many - 1;
            const uint32_t sv = __shfl_sync(FULL_MASK, my_v, sl);
            const uint64_t sb = __shfl_sync(FULL_MASK, my_b, sl);
            const uint64_t se = __shfl_sync(FULL_MASK, my_e, sl);
            const uint64_t sf = __shfl_sync(FULL_MASK, my_fm, sl);
            const uint64_t sp = __shfl_sync(FULL_MASK, pr, sl);
            const uint64_t sn = __shfl_sync(FULL_MASK, nrec, sl);
            for (uint64_t j = lane; j < sn; j += 32) {
                if (sp + j >= p.big_cap) break;
                const uint64_t st = sb + j * kMsRec;
                const uint32_t len = (uint32_t)((se - st) < kMsRec ? (se - st) : kMsRec);
                p.rec[p.small_cap + sp + j] = make_uint4(sv, len, (uint32_t)st, (uint32_t)(st >> 32));
                p.fm[p.small_cap + sp + j] = sf;
            }
        }
        __syncthreads();  // S.tmp / S.base reuse
    }
    // per-instance sums of the block: kept bits (|Q_i| of the next step),
    // extractions, edges of the extracted vertices, smallest kept key
    if (i0 < p.K) {
        ms_lane_add(S, 0, lane, keep0, i1 < p.K ? keep1 : 0);
        ms_lane_add(S, 1, lane, ext0, i1 < p.K ? ext1 : 0);
        ms_lane_add(S, 2, lane, edg0, i1 < p.K ? edg1 : 0);
        if (kmin0 != kInf) atomicMin(&S.mn[i0], (unsigned long long)kmin0);
        if (i1 < p.K && kmin1 != kInf) atomicMin(&S.mn[i1], (unsigned long long)kmin1);
    }
    __syncthreads();
    for (uint32_t i = tid; i < p.K; i += kMsBlock) {
        MsInst* I = &p.inst[i];
        if (S.cnt[0][i]) atomicAdd(&I->qsize[nx], (unsigned int)S.cnt[0][i]);
        if (S.cnt[1][i]) atomicAdd(&I->fext[c], S.cnt[1][i]);
        if (S.cnt[2][i]) atomicAdd(&I->fedges[c], S.cnt[2][i]);
        if (S.mn[i] != kInf) atomicMin(&I->qmin[nx], S.mn[i]);
        S.cnt[0][i] = 0; S.cnt[1][i] = 0; S.cnt[2][i] = 0; S.mn[i] = kInf;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// phase R: relaxation of the step's records (one warp per record, records
// dealt round-robin to warps numbered across blocks first).
// ---------------------------------------------------------------------------
__device__ void ms_phase_R(const MsParams& p, uint64_t k, MsSmem& S, uint32_t* stage)
{
    const uint32_t tid = threadIdx.x, lane = tid & 31u, wid = tid >> 5;
    const int c = (int)(k % 3), nx = (int)((k + 1) % 3);
    uint32_t* Qnext = (k & 1) ? p.qb : p.qa;
    const uint32_t R = p.R;
    const uint32_t i0 = 2 * lane;
    const bool track_min = p.algo == SSSP_DELTA_STAR;
    uint64_t nsm = ldcg32(&p.ctrl->nsmall[c]);
    nsm = nsm < p.small_cap ? nsm : p.small_cap;
    uint64_t nrec = ldcg32(&p.ctrl->nbig[c]);
    nrec = nrec < p.big_cap ? nrec : p.big_cap;
    const uint32_t gwarp = wid * gridDim.x + blockIdx.x;
    const uint32_t nwarps = gridDim.x * kMsWarps;
    uint64_t qn0 = 0, qn1 = 0, up0 = 0, up1 = 0, um0 = kInf, um1 = kInf;
    uint32_t stc = 0;

    // (a) vertices of degree 1..32 extracted by at most kMsSparse instances:
    //     32 records per warp with their edges spread over the lanes 32 at a
    //     time; each lane walks the (short) instance mask of its edge's
    //     record (per-instance counts by shared-memory atomics)
    const uint64_t ngroups = (nsm + 31u) >> 5;
    const uint32_t lmask = lane == 31 ? FULL_MASK : ((2u << lane) - 1u);
    for (uint64_t gi = gwarp; gi < ngroups; gi += nwarps) {
        const uint64_t r = gi * 32u + lane;
        const bool valid = r < nsm;
        const uint4 rc = valid ? __ldcg(&p.rec[r]) : make_uint4(0u, 0u, 0u, 0u);
        const uint64_t fmk = valid ? ldcg64(&p.fm[r]) : 0ull;
        const uint32_t len = rc.y;
        const uint64_t start = (uint64_t)rc.z | ((uint64_t)rc.w << 32);
        const uint32_t incl = (uint32_t)warp_incl_scan64(len, lane);
        const uint32_t excl = incl - len;
        const uint32_t total = __shfl_sync(FULL_MASK, incl, 31);
        uint32_t started = 0;
        for (uint32_t r0 = 0; r0 < total; r0 += 32) {
            // owner of edge r0+lane: the record whose run of edges holds it
            const uint32_t contrib = (len > 0 && excl >= r0 && excl < r0 + 32u) ? (1u << (excl - r0)) : 0u;
            const uint32_t starts = __reduce_or_sync(FULL_MASK, contrib);
            int owner = (int)(started + __popc(starts & lmask)) - 1;
            owner = owner < 0 ? 0 : owner;
            started += __popc(starts);
            const uint32_t e = r0 + lane;
            const bool ok = e < total;
            const uint32_t ou = __shfl_sync(FULL_MASK, rc.x, owner);
            const uint64_t ofm = __shfl_sync(FULL_MASK, fmk, owner);
            const uint64_t ost = __shfl_sync(FULL_MASK, start, owner);
            const uint32_t oex = __shfl_sync(FULL_MASK, excl, owner);
            const uint2 ed = ok ? __ldcs(&p.edges[ost + (e - oex)]) : make_uint2(0u, 0u);
            uint64_t newb = 0;
            uint64_t m = ok ? ofm : 0ull;
            while (m) {  // per lane: four instances at a time, loads in flight
                uint32_t ib[4];
                uint64_t dua[4], dvb[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    ib[t] = m ? (uint32_t)(__ffsll((long long)m) - 1) : 64u;
                    m &= m - 1;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    dua[t] = ib[t] < 64u ? ldcg64(&p.D[(uint64_t)ou * R + ib[t]]) : kInf;
                    dvb[t] = ib[t] < 64u ? ld_precheck<true>(&p.D[(uint64_t)ed.x * R + ib[t]]) : 0ull;
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    if (ib[t] >= 64u || dua[t] == kInf) continue;
                    const uint64_t cand = dua[t] + ed.y;
                    if (cand < dvb[t]) {
                        atomicMin(reinterpret_cast<unsigned long long*>(&p.D[(uint64_t)ed.x * R + ib[t]]),
                                  (unsigned long long)cand);
                        newb |= 1ull << ib[t];
                        atomicAdd(&S.cnt[1][ib[t]], 1ull);
                        if (track_min) atomicMin(&S.mn[ib[t]], (unsigned long long)cand);
                    }
                }
            }
            const uint64_t old = newb ? atomicOr(reinterpret_cast<unsigned long long*>(&p.QM[ed.x]),
                                                 (unsigned long long)newb) : 0ull;
            stage_push(newb != 0 && old == 0, ed.x, stage, stc, lane);
            uint64_t newly = newb & ~old;
            while (newly) {
                const uint32_t it = (uint32_t)(__ffsll((long long)newly) - 1);
                newly &= newly - 1;
                atomicAdd(&S.cnt[0][it], 1ull);
            }
            if (stc > (uint32_t)kStage - 32u) stage_flush(stage, stc, lane, &p.ctrl->usize[nx], &p.ctrl->status, Qnext, p.n);
        }
    }

    // (b) every other record: one warp per record of <= 32 edges
    for (uint64_t r = gwarp; r < nrec; r += nwarps) {
        const uint4 rc = __ldcg(&p.rec[p.small_cap + r]);
        const uint64_t fmk = ldcg64(&p.fm[p.small_cap + r]);
        const uint32_t u = rc.x, len = rc.y;
        const uint64_t start = (uint64_t)rc.z | ((uint64_t)rc.w << 32);
        const uint32_t b2 = (uint32_t)(fmk >> i0) & 3u;
        // delta_i[u] read at relaxation time (Algorithm 1)
        const ulonglong2 du = b2 ? ld_pair_cg(&p.D[(uint64_t)u * R + i0]) : make_ulonglong2(kInf, kInf);
        const uint2 ed = lane < len ? __ldcs(&p.edges[start + lane]) : make_uint2(0u, 0u);
        const uint32_t pc = __popcll(fmk);
        uint64_t ubits = 0;  // instances whose delta[u] a pull lowered
        if (pc <= kMsSparse) {
            // lanes = the record's edges; the instances of F(u) are taken four at
            // a time with their four pre-check loads in flight (bits of one row
            // sector share a line, so later loads of the same row hit L1)
            uint64_t newb = 0;
            uint64_t m = fmk;
            while (m) {  // warp-uniform
                uint32_t ib[kMsSparse];
                uint64_t dui[kMsSparse], dv[kMsSparse];
#pragma unroll
                for (uint32_t t = 0; t < kMsSparse; ++t) {
                    ib[t] = m ? (uint32_t)(__ffsll((long long)m) - 1) : 64u;
                    m &= m - 1;
                }
#pragma unroll
                for (uint32_t t = 0; t < kMsSparse; ++t) {
                    const uint32_t it = ib[t] < 64u ? ib[t] : 0u;
                    const uint64_t mine = (it & 1u) ? du.y : du.x;
                    dui[t] = __shfl_sync(FULL_MASK, mine, it >> 1);
                    const bool ok = ib[t] < 64u && lane < len && dui[t] != kInf;
                    dv[t] = ok ? ld_precheck<true>(&p.D[(uint64_t)ed.x * R + it]) : 0ull;
                }
                if (p.bidir) {
                    // bidirectional relaxation (undirected graph): the gathered
                    // delta_i[v] first lower delta_i[u] (WriteMin + Update of u),
                    // then u pushes with the lowered value
#pragma unroll
                    for (uint32_t t = 0; t < kMsSparse; ++t) {
                        if (ib[t] >= 64u) break;  // warp-uniform
                        uint64_t pull = (lane < len && dui[t] != kInf && dv[t] != kInf) ? dv[t] + ed.y : kInf;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const uint64_t y = __shfl_xor_sync(FULL_MASK, pull, o);
                            pull = y < pull ? y : pull;
                        }
                        if (pull < dui[t]) {  // warp-uniform
                            dui[t] = pull;
                            ubits |= 1ull << ib[t];
                            if (lane == 0)
                                atomicMin(reinterpret_cast<unsigned long long*>(&p.D[(uint64_t)u * R + ib[t]]),
                                          (unsigned long long)pull);
                            if (lane == (ib[t] >> 1)) {
                                if (ib[t] & 1u) { ++up1; um1 = pull < um1 ? pull : um1; }
                                else { ++up0; um0 = pull < um0 ? pull : um0; }
                            }
                        }
                    }
                }
#pragma unroll
                for (uint32_t t = 0; t < kMsSparse; ++t) {
                    if (ib[t] >= 64u) break;  // warp-uniform
                    const uint64_t cand = dui[t] + ed.y;
                    const bool imp = lane < len && dui[t] != kInf && cand < dv[t];
                    if (imp) {
                        atomicMin(reinterpret_cast<unsigned long long*>(&p.D[(uint64_t)ed.x * R + ib[t]]),
                                  (unsigned long long)cand);
                        newb |= 1ull << ib[t];
                    }
                    const uint32_t cnt = __popc(__ballot_sync(FULL_MASK, imp));
                    if (lane == (ib[t] >> 1)) { if (ib[t] & 1u) up1 += cnt; else up0 += cnt; }
                    if (track_min) {
                        uint64_t mn = imp ? cand : kInf;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) {
                            const uint64_t y = __shfl_xor_sync(FULL_MASK, mn, o);
                            mn = y < mn ? y : mn;
                        }
                        if (lane == (ib[t] >> 1)) {
                            if (ib[t] & 1u) um1 = mn < um1 ? mn : um1; else um0 = mn < um0 ? mn : um0;
                        }
                    }
                }
            }
            // Update(v): one test-and-set of the improved bits on v's mask; the
            // bits pulled into u update u's mask (lane 0)
            const uint64_t old = newb ? atomicOr(reinterpret_cast<unsigned long long*>(&p.QM[ed.x]),
                                                 (unsigned long long)newb) : 0ull;
            const uint64_t newly = newb & ~old;
            stage_push(newb != 0 && old == 0, ed.x, stage, stc, lane);
            // newly queued bits per instance: lane l counts instances 2l, 2l+1
            {
                uint64_t mm = fmk;
                while (mm) {  // warp-uniform
                    const uint32_t it = (uint32_t)(__ffsll((long long)mm) - 1);
                    mm &= mm - 1;
                    const uint32_t cnt = __popc(__ballot_sync(FULL_MASK, (newly >> it) & 1ull));
                    if (lane == (it >> 1)) { if (it & 1u) qn1 += cnt; else qn0 += cnt; }
                }
            }
        } else {
            // many instances: lanes = instance pairs (lane l: 2l, 2l+1), four
            // edges at a time, one coalesced access to each target's row
            uint64_t du0 = du.x, du1 = du.y;
            uint32_t ub2 = 0;
            for (uint32_t e0 = 0; e0 < len; e0 += 4) {
                uint32_t vv[4], ww[4];
                ulonglong2 dv[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    vv[t] = __shfl_sync(FULL_MASK, ed.x, (e0 + t) & 31u);
                    ww[t] = __shfl_sync(FULL_MASK, ed.y, (e0 + t) & 31u);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const bool ok = e0 + t < len && b2 != 0;
                    dv[t] = ok ? __ldca(reinterpret_cast<const ulonglong2*>(&p.D[(uint64_t)vv[t] * R + i0]))
                               : make_ulonglong2(kInf, kInf);
                }
                if (p.bidir) {
                    // bidirectional relaxation: the group's gathered rows first
                    // lower this lane's delta_i[u] (the values stay in lane)
                    uint64_t p0 = kInf, p1 = kInf;
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        if (e0 + t >= len) continue;
                        if ((b2 & 1u) && dv[t].x != kInf && dv[t].x + ww[t] < p0) p0 = dv[t].x + ww[t];
                        if ((b2 & 2u) && dv[t].y != kInf && dv[t].y + ww[t] < p1) p1 = dv[t].y + ww[t];
                    }
                    uint64_t* urow = &p.D[(uint64_t)u * R + i0];
                    if (p0 < du0) {
                        du0 = p0; ub2 |= 1u; ++up0; um0 = p0 < um0 ? p0 : um0;
                        atomicMin(reinterpret_cast<unsigned long long*>(urow), (unsigned long long)p0);
                    }
                    if (p1 < du1) {
                        du1 = p1; ub2 |= 2u; ++up1; um1 = p1 < um1 ? p1 : um1;
                        atomicMin(reinterpret_cast<unsigned long long*>(urow + 1), (unsigned long long)p1);
                    }
                }
                uint32_t my_vt = 0;
                uint64_t my_nb = 0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    uint32_t imp = 0;
                    if (e0 + t < len) {
                        uint64_t* row = &p.D[(uint64_t)vv[t] * R + i0];
                        if ((b2 & 1u) && du0 != kInf) {
                            const uint64_t cnd = du0 + ww[t];
                            if (cnd < dv[t].x) {
                                atomicMin(reinterpret_cast<unsigned long long*>(row), (unsigned long long)cnd);
                                imp |= 1u; ++up0; um0 = cnd < um0 ? cnd : um0;
                            }
                        }
                        if ((b2 & 2u) && du1 != kInf) {
                            const uint64_t cnd = du1 + ww[t];
                            if (cnd < dv[t].y) {
                                atomicMin(reinterpret_cast<unsigned long long*>(row + 1), (unsigned long long)cnd);
                                imp |= 2u; ++up1; um1 = cnd < um1 ? cnd : um1;
                            }
                        }
                    }
                    const uint64_t nb = lane_pairs_or(imp, lane);
                    if (lane == (uint32_t)t) { my_vt = vv[t]; my_nb = nb; }
                }
                const uint64_t old = (lane < 4 && my_nb)
                                         ? atomicOr(reinterpret_cast<unsigned long long*>(&p.QM[my_vt]),
                                                    (unsigned long long)my_nb)
                                         : 0ull;
                const uint64_t newly = my_nb & ~old;
                stage_push(lane < 4 && my_nb != 0 && old == 0, my_vt, stage, stc, lane);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const uint64_t nw = __shfl_sync(FULL_MASK, newly, t);
                    qn0 += (nw >> i0) & 1ull;
                    qn1 += (nw >> (i0 + 1)) & 1ull;
                }
            }
            ubits = lane_pairs_or(ub2, lane);
        }
        // the bits pulled into u update u's mask (Update(u), lane 0)
        if (ubits) {  // warp-uniform
            uint64_t uold = 0;
            if (lane == 0) uold = atomicOr(reinterpret_cast<unsigned long long*>(&p.QM[u]), (unsigned long long)ubits);
            uold = __shfl_sync(FULL_MASK, uold, 0);
            stage_push(lane == 0 && uold == 0, u, stage, stc, lane);
            const uint64_t unew = ubits & ~uold;
            qn0 += (unew >> i0) & 1ull;
            qn1 += (unew >> (i0 + 1)) & 1ull;
        }
        if (stc > (uint32_t)kStage - kMsRec - 1u) stage_flush(stage, stc, lane, &p.ctrl->usize[nx], &p.ctrl->status, Qnext, p.n);
    }
    stage_flush(stage, stc, lane, &p.ctrl->usize[nx], &p.ctrl->status, Qnext, p.n);
    if (i0 < p.K) {
        const uint32_t i1 = i0 + 1;
        ms_lane_add(S, 0, lane, qn0, i1 < p.K ? qn1 : 0);
        ms_lane_add(S, 1, lane, up0, i1 < p.K ? up1 : 0);
        if (um0 != kInf) atomicMin(&S.mn[i0], (unsigned long long)um0);
        if (i1 < p.K && um1 != kInf) atomicMin(&S.mn[i1], (unsigned long long)um1);
    }
    __syncthreads();
    for (uint32_t i = tid; i < p.K; i += kMsBlock) {
        MsInst* I = &p.inst[i];
        if (S.cnt[0][i]) atomicAdd(&I->qsize[nx], (unsigned int)S.cnt[0][i]);
        if (S.cnt[1][i]) atomicAdd(&I->fupd[c], S.cnt[1][i]);
        if (S.mn[i] != kInf) atomicMin(&I->qmin[nx], S.mn[i]);
        S.cnt[0][i] = 0; S.cnt[1][i] = 0; S.mn[i] = kInf;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMsBlock, 1) ms_batch_kernel(MsParams p)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint32_t* s_stage = reinterpret_cast<uint32_t*>(s_dyn);
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_dyn);
    __shared__ MsSmem S;
    const uint32_t tid = threadIdx.x, wid = tid >> 5;
    const uint64_t gthreads = (uint64_t)gridDim.x * kMsBlock;
    const uint64_t gtid = (uint64_t)blockIdx.x * kMsBlock + tid;
    MsCtrl* ctrl = p.ctrl;
    uint32_t* stage = s_stage + wid * kStage;
    if (tid == 0) {
        S.bar_target = 0;
        S.t_start = global_timer_ns();
        S.err = 0;
    }
    for (uint32_t i = tid; i < kMsMax; i += kMsBlock) {
        S.cnt[0][i] = 0; S.cnt[1][i] = 0; S.cnt[2][i] = 0; S.cnt[3][i] = 0; S.mn[i] = kInf;
    }
    // init: delta_i <- inf for every instance, empty masks
    const uint64_t cells = (uint64_t)p.n * p.R / 2;
    ulonglong2* D2 = reinterpret_cast<ulonglong2*>(p.D);
    for (uint64_t x = gtid; x < cells; x += gthreads) D2[x] = make_ulonglong2(kInf, kInf);
    for (uint64_t v = gtid; v < p.n; v += gthreads) p.QM[v] = 0ull;
    if (!grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns)) return;
    // delta_i[s_i] <- 0, Q_i.Update(s_i) (Algorithm 1)
    for (uint64_t i = gtid; i < p.K; i += gthreads) {
        const uint32_t s = p.src[i];
        p.D[(uint64_t)s * p.R + i] = 0ull;
        const unsigned long long old = atomicOr(reinterpret_cast<unsigned long long*>(&p.QM[s]), 1ull << i);
        if (old == 0) p.qa[atomicAdd(&ctrl->usize[1], 1u)] = s;
        MsInst* I = &p.inst[i];
        I->qsize[1] = 1;
        I->qmin[0] = kInf; I->qmin[1] = 0; I->qmin[2] = kInf;
    }
    if (!grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns)) return;

    uint64_t k = 1;
    bool ok = true;
    for (;; ++k) {
        const int c = (int)(k % 3), pv = (int)((k + 2) % 3);
        uint32_t U = ldcg32(&ctrl->usize[c]);
        U = U < p.n ? U : p.n;
        if (U == 0) break;  // every instance's queue is empty (all blocks agree)
        ms_phase_T(p, k, U, S, s_keys);
        if (blockIdx.x == 0 && tid == 0) {
            ctrl->usize[pv] = 0;
            ctrl->nsmall[pv] = 0;
            ctrl->nbig[pv] = 0;
            if (S.err) raise_error(&ctrl->bar, &ctrl->status, SSSP_ERR_INTERNAL);
            if (global_timer_ns() - S.t_start > p.solve_timeout_ns) raise_error(&ctrl->bar, &ctrl->status, SSSP_ERR_TIMEOUT);
        }
        if (!(ok = grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns))) break;
        ms_phase_E(p, k, U, S);
        if (!(ok = grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns))) break;
        ms_phase_R(p, k, S, stage);
        if (!(ok = grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns))) break;
    }
    if (!ok) return;
    // the last step's counters; instances still unmarked ran to the last step
    const int last = (int)((k + 2) % 3);
    for (uint64_t i = gtid; i < p.K; i += gthreads) {
        MsInst* I = &p.inst[i];
        if (k > 1) {
            I->queued += I->qsize[last];
            I->extracted += I->fext[last];
            I->edges += I->fedges[last];
            I->updates += I->fupd[last];
        }
        if (I->last_step == 0) I->last_step = (unsigned)(k - 1);
    }
    if (gtid == 0) ctrl->steps = k - 1;
    // distances out, in the caller's ids and layout (instance-major)
    for (uint64_t v = gtid; v < p.n; v += gthreads) {
        const uint64_t kv = p.perm ? (uint64_t)__ldg(&p.perm[v]) : v;
        const uint64_t* row = &p.D[kv * p.R];
        for (uint32_t i = 0; i < p.K; ++i) p.dist_out[i][v] = __ldcg(reinterpret_cast<const unsigned long long*>(row + i));
    }
}

// ---------------------------------------------------------------------------
// Serving with the shared scan: a long-lived loop over S <= 64 query slots
// that are the kernel's instances.  At each step boundary block 0 retires the
// slots whose queue emptied (their column of D is copied to the caller's
// output by every block before the completion record is released) and admits
// newly submitted queries into free slots (their column is reset by every
// block, then the source is queued); admitted queries join the running ones
// at that step (continuous batching).  With no query left the loop waits a
// bounded idle time for a command, then the kernel returns.
// ---------------------------------------------------------------------------
struct MsServeState {                 // device memory, kept across launches
    unsigned long long seen_submitted;
    unsigned long long step;          // last global step run
    unsigned int nretire, nadmit, exit_flag, pad;
    unsigned int retire[kMsMax], admit[kMsMax];
    unsigned int running[kMsMax], seq[kMsMax];
    unsigned long long ticket[kMsMax], t_admit[kMsMax], admit_step[kMsMax], dist_ptr[kMsMax];
    unsigned int source[kMsMax];      // caller's id
    unsigned long long seen_ns[kMsMax];  // device time a slot's waiting command was first seen (0: none)
};

struct MsServeParams {
    MsParams p;                       // p.src / p.param: device arrays of S entries, written at admission
    uint32_t* src_w;
    SlotCmd* cmd;
    SlotDone* done;
    ServeShared* shared;
    MsServeState* st;
    uint64_t idle_ns;
    uint64_t param;
    uint32_t gang;                    // admit when this many commands wait, the device is idle,
    uint64_t gang_wait_ns;            // or the oldest waiting command is this old
};

// Block 0: which slots retire (queue empty at step k) and which free slots
// take a new command; exit_flag when the loop should return.
__device__ void ms_serve_decide(const MsServeParams& sp, uint64_t k, MsSmem& S)
{
    const MsParams& p = sp.p;
    MsServeState* st = sp.st;
    const uint32_t tid = threadIdx.x;
    const int c = (int)(k % 3);
    if (tid == 0) { st->nretire = 0; st->nadmit = 0; }
    __syncthreads();
    for (uint32_t i = tid; i < p.K; i += kMsBlock)
        if (st->running[i] && ldcg32(&p.inst[i].qsize[c]) == 0) st->retire[atomicAdd(&st->nretire, 1u)] = i;
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            const unsigned long long sub = ld_acquire_sys_u64(&sp.shared->submitted);
            S.scnt = sub != st->seen_submitted;
            st->seen_submitted = sub;
        }
        __syncthreads();
        // free slots holding a command not yet admitted (queries that start
        // together stay aligned step by step, which is what the shared scan
        // shares, so they are admitted as a gang: when sp.gang of them wait,
        // when nothing else runs, or when the oldest has waited gang_wait_ns)
        if (tid == 0) { S.base[1] = 0; S.t_start = ~0ull; }
        __syncthreads();
        const unsigned long long now = global_timer_ns();
        for (uint32_t i = tid; i < p.K; i += kMsBlock) {
            if (st->running[i]) continue;
            const unsigned int cs = ld_acquire_sys_u32(&sp.cmd[i].seq);
            if (cs == st->seq[i]) continue;
            if (st->seen_ns[i] == 0) st->seen_ns[i] = now;
            atomicAdd(&S.base[1], 1u);
            atomicMin(&S.t_start, (unsigned long long)st->seen_ns[i]);
        }
        uint32_t live0 = 0;
        for (uint32_t i = tid; i < p.K; i += kMsBlock) {
            bool retiring = false;
            for (uint32_t r = 0; r < st->nretire; ++r) retiring |= st->retire[r] == i;
            live0 += (st->running[i] && !retiring) ? 1u : 0u;
        }
        live0 = __syncthreads_count(live0 != 0);
        const bool take = S.base[1] >= sp.gang || live0 == 0 ||
                          (S.base[1] > 0 && now - S.t_start >= sp.gang_wait_ns);
        if (take) {
            for (uint32_t i = tid; i < p.K; i += kMsBlock) {
                if (st->running[i]) continue;
                const unsigned int cs = ld_acquire_sys_u32(&sp.cmd[i].seq);
                if (cs == st->seq[i]) continue;
                const volatile SlotCmd* cm = &sp.cmd[i];
                st->dist_ptr[i] = cm->dist_ptr;
                st->source[i] = cm->source < p.n ? cm->source : 0u;
                st->ticket[i] = cm->ticket;
                st->seq[i] = cs;
                st->seen_ns[i] = 0;
                st->admit[atomicAdd(&st->nadmit, 1u)] = i;
            }
        }
        __syncthreads();
        uint32_t live = 0;
        for (uint32_t i = tid; i < p.K; i += kMsBlock) {
            bool retiring = false;
            for (uint32_t r = 0; r < st->nretire; ++r) retiring |= st->retire[r] == i;
            live += (st->running[i] && !retiring) ? 1u : 0u;
        }
        live = __syncthreads_count(live != 0);
        if (tid == 0) {
            S.base[0] = 0;  // 0: run, 1: a command came while idle, 2: leave
            if (ld_acquire_sys_u32(&sp.shared->stop)) {
                S.base[0] = 2;
            } else if (live == 0 && st->nadmit == 0 && st->nretire == 0) {
                const unsigned long long t0 = global_timer_ns();
                S.base[0] = 2;
                while (global_timer_ns() - t0 < sp.idle_ns) {
                    if (ld_acquire_sys_u64(&sp.shared->submitted) != st->seen_submitted) { S.base[0] = 1; break; }
                    if (ld_acquire_sys_u32(&sp.shared->stop)) break;
                    __nanosleep(2000);
                }
            }
            st->exit_flag = S.base[0] == 2 ? 1u : 0u;
        }
        __syncthreads();
        if (S.base[0] != 1) return;
    }
}

// Block 0, after the columns were copied / reset: completion records of the
// retired slots, then the admitted queries' sources are queued.
__device__ void ms_serve_publish(const MsServeParams& sp, uint64_t k)
{
    const MsParams& p = sp.p;
    MsServeState* st = sp.st;
    const uint32_t tid = threadIdx.x;
    const int c = (int)(k % 3), pv = (int)((k + 2) % 3);
    uint32_t* Qcur = (k & 1) ? p.qa : p.qb;
    for (uint32_t r = tid; r < st->nretire; r += kMsBlock) {
        const uint32_t i = st->retire[r];
        MsInst* I = &p.inst[i];
        SlotDone* D = &sp.done[i];
        D->ticket = st->ticket[i];
        D->t_admit_ns = st->t_admit[i];
        D->t_done_ns = global_timer_ns();
        D->edges = I->edges + I->fedges[pv];
        D->extracted = I->extracted + I->fext[pv];
        D->steps = (unsigned int)(k - st->admit_step[i]);
        D->status = *reinterpret_cast<volatile int*>(&p.ctrl->status);
        __threadfence_system();
        st_release_sys_u32(&D->seq, st->seq[i]);
        st->running[i] = 0;
        memset(I, 0, sizeof(MsInst));
        I->qmin[0] = kInf; I->qmin[1] = kInf; I->qmin[2] = kInf;
    }
    for (uint32_t a = tid; a < st->nadmit; a += kMsBlock) {
        const uint32_t i = st->admit[a];
        const uint32_t caller = st->source[i];
        const uint32_t s = p.perm ? p.perm[caller] : caller;
        sp.src_w[i] = s;
        p.D[(uint64_t)s * p.R + i] = 0ull;
        const unsigned long long old = atomicOr(reinterpret_cast<unsigned long long*>(&p.QM[s]), 1ull << i);
        if (old == 0) Qcur[atomicAdd(&p.ctrl->usize[c], 1u)] = s;
        MsInst* I = &p.inst[i];
        memset(I, 0, sizeof(MsInst));
        I->qmin[0] = kInf; I->qmin[1] = kInf; I->qmin[2] = kInf;
        I->qsize[c] = 1;
        I->qmin[c] = 0;
        st->admit_step[i] = k;
        st->t_admit[i] = global_timer_ns();
        st->running[i] = 1;
    }
}

__global__ void __launch_bounds__(kMsBlock, 1) ms_serve_kernel(MsServeParams sp)
{
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint32_t* s_stage = reinterpret_cast<uint32_t*>(s_dyn);
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(s_dyn);
    __shared__ MsSmem S;
    const MsParams& p = sp.p;
    const uint32_t tid = threadIdx.x, wid = tid >> 5;
    const uint64_t gthreads = (uint64_t)gridDim.x * kMsBlock;
    const uint64_t gtid = (uint64_t)blockIdx.x * kMsBlock + tid;
    MsCtrl* ctrl = p.ctrl;
    MsServeState* st = sp.st;
    uint32_t* stage = s_stage + wid * kStage;
    if (tid == 0) {
        S.bar_target = 0;
        S.err = 0;
    }
    for (uint32_t i = tid; i < kMsMax; i += kMsBlock) {
        S.cnt[0][i] = 0; S.cnt[1][i] = 0; S.cnt[2][i] = 0; S.cnt[3][i] = 0; S.mn[i] = kInf;
    }
    __syncthreads();
    uint64_t k = ldcg64((const uint64_t*)&st->step) + 1;
    for (;;) {
        const int c = (int)(k % 3), pv = (int)((k + 2) % 3);
        if (blockIdx.x == 0) ms_serve_decide(sp, k, S);
        if (!grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns)) return;
        if (ldcg32(&st->exit_flag)) break;
        const uint32_t nret = ldcg32(&st->nretire), nadm = ldcg32(&st->nadmit);
        if (nret + nadm != 0) {
            // finished queries' columns to their callers (caller's ids), new
            // queries' columns reset
            for (uint32_t r = 0; r < nret; ++r) {
                const uint32_t i = ldcg32(&st->retire[r]);
                uint64_t* out = reinterpret_cast<uint64_t*>(ldcg64((const uint64_t*)&st->dist_ptr[i]));
                for (uint64_t v = gtid; v < p.n; v += gthreads) {
                    const uint64_t kv = p.perm ? (uint64_t)__ldg(&p.perm[v]) : v;
                    out[v] = __ldcg(reinterpret_cast<const unsigned long long*>(&p.D[kv * p.R + i]));
                }
            }
            for (uint32_t a = 0; a < nadm; ++a) {
                const uint32_t i = ldcg32(&st->admit[a]);
                for (uint64_t v = gtid; v < p.n; v += gthreads) p.D[v * p.R + i] = kInf;
            }
            if (!grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns)) return;
            if (blockIdx.x == 0) ms_serve_publish(sp, k);
            if (!grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns)) return;
        }
        uint32_t U = ldcg32(&ctrl->usize[c]);
        U = U < p.n ? U : p.n;
        if (U == 0) {
            // nothing queued (all blocks agree): every slot is idle, back to
            // admission at the same step; a running slot here would be an
            // internal fault, reported instead of looping
            if (blockIdx.x == 0 && tid == 0) {
                bool any = false;
                for (uint32_t i = 0; i < p.K; ++i) any |= ldcg32(&st->running[i]) != 0;
                if (any) raise_error(&ctrl->bar, &ctrl->status, SSSP_ERR_INTERNAL);
            }
            continue;
        }
        ms_phase_T(p, k, U, S, s_keys);
        if (blockIdx.x == 0 && tid == 0) {
            ctrl->usize[pv] = 0;
            ctrl->nsmall[pv] = 0;
            ctrl->nbig[pv] = 0;
            if (S.err) raise_error(&ctrl->bar, &ctrl->status, SSSP_ERR_INTERNAL);
        }
        if (!grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns)) return;
        ms_phase_E(p, k, U, S);
        if (!grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns)) return;
        ms_phase_R(p, k, S, stage);
        if (blockIdx.x == 0 && tid == 0) st->step = k;
        if (!grid_sync_err(&ctrl->bar, &ctrl->status, &S.bar_target, p.timeout_ns)) return;
        ++k;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

struct MsWorkspace {
    int device = -1;
    void* buf = nullptr;
    size_t bytes = 0;
    MsInst* d_inst = nullptr;
    MsCtrl* d_ctrl = nullptr;
    uint32_t* d_src = nullptr;
    uint64_t* d_param = nullptr;
    uint64_t** d_out = nullptr;
    // pinned staging (sources, parameters, output pointers), reused after the copy event
    uint32_t* h_src = nullptr;
    uint64_t* h_param = nullptr;
    uint64_t** h_out = nullptr;
    MsInst* h_inst = nullptr;
    MsCtrl* h_ctrl = nullptr;
    cudaEvent_t copied = nullptr;
    uint32_t grid = 0;
    uint32_t last_k = 0;
};
std::mutex g_ms_mu;
MsWorkspace g_ms[64];

int ms_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? SSSP_ERR_OUT_OF_MEMORY : SSSP_ERR_CUDA; }
size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int ms_setup(MsWorkspace& w, int dev)
{
    if (w.device >= 0) return SSSP_OK;
    cudaError_t e;
    if ((e = cudaEventCreateWithFlags(&w.copied, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&w.d_inst), sizeof(MsInst) * kMsMax)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&w.d_ctrl), sizeof(MsCtrl))) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&w.d_src), sizeof(uint32_t) * kMsMax)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&w.d_param), sizeof(uint64_t) * kMsMax)) != cudaSuccess ||
        (e = cudaMalloc(reinterpret_cast<void**>(&w.d_out), sizeof(uint64_t*) * kMsMax)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void**>(&w.h_src), sizeof(uint32_t) * kMsMax)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void**>(&w.h_param), sizeof(uint64_t) * kMsMax)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void**>(&w.h_out), sizeof(uint64_t*) * kMsMax)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void**>(&w.h_inst), sizeof(MsInst) * kMsMax)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void**>(&w.h_ctrl), sizeof(MsCtrl))) != cudaSuccess)
        return ms_fail(e);
    const void* fn = reinterpret_cast<const void*>(&ms_batch_kernel);
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMsDynSmem)) != cudaSuccess)
        return ms_fail(e);
    int bps = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kMsBlock, kMsDynSmem)) != cudaSuccess) return ms_fail(e);
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return ms_fail(e);
    if (bps < 1) return SSSP_ERR_CUDA;
    w.grid = (uint32_t)(bps * sms);
    w.device = dev;
    return SSSP_OK;
}

}  // namespace

bool ms_batch_supported(sssp_algo algo, uint32_t k)
{
    return k >= 1 && k <= kMsMax && (algo == SSSP_RHO || algo == SSSP_DELTA_STAR || algo == SSSP_BELLMAN_FORD);
}

int ms_solve_sources(const sssp_graph* g, const uint32_t* sources, uint32_t k, sssp_algo algo,
                     const uint64_t* params, uint64_t* const* outs, uint32_t rho_reduced, uint32_t warm_steps,
                     uint64_t warm_rho, bool bidir, void* stream)
{
    if (!g || !sources || !outs || !ms_batch_supported(algo, k)) return SSSP_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < k; ++i) {
        if (sources[i] >= g->n || !outs[i]) return SSSP_ERR_INVALID_ARG;
        if (algo_needs_param(algo) && (params ? params[i] : 1) == 0) return SSSP_ERR_INVALID_ARG;
    }
    const int dev = g->device;
    if (dev < 0 || dev >= 64) return SSSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_ms_mu);
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return ms_fail(e);
    MsWorkspace& w = g_ms[dev];
    int rc = ms_setup(w, dev);
    if (rc != SSSP_OK) return rc;
    const uint32_t R = (k + 3) & ~3u;
    const uint64_t n = g->n;
    const uint64_t rec_cap = g->fsmall_cap + g->ms_rec_cap;  // degree 1..32: one each; larger: 32 edges each
    const size_t need = a256(8ull * n * R) + a256(8ull * n) + 2 * a256(4ull * n) + a256(16ull * rec_cap) +
                        a256(8ull * rec_cap);
    if (need > w.bytes) {
        cudaDeviceSynchronize();
        cudaFree(w.buf);
        w.buf = nullptr;
        w.bytes = 0;
        if ((e = cudaMalloc(&w.buf, need)) != cudaSuccess) return ms_fail(e);
        w.bytes = need;
    }
    unsigned char* b = static_cast<unsigned char*>(w.buf);
    MsParams p;
    memset(&p, 0, sizeof p);
    p.D = reinterpret_cast<uint64_t*>(b); b += a256(8ull * n * R);
    p.QM = reinterpret_cast<uint64_t*>(b); b += a256(8ull * n);
    p.qa = reinterpret_cast<uint32_t*>(b); b += a256(4ull * n);
    p.qb = reinterpret_cast<uint32_t*>(b); b += a256(4ull * n);
    p.rec = reinterpret_cast<uint4*>(b); b += a256(16ull * rec_cap);
    p.fm = reinterpret_cast<uint64_t*>(b);
    p.small_cap = g->fsmall_cap;
    p.big_cap = g->ms_rec_cap;
    // the staging is reused: wait until the previous call's copy has left it
    if ((e = cudaEventSynchronize(w.copied)) != cudaSuccess) return ms_fail(e);
    uint64_t max_param = 1;
    for (uint32_t i = 0; i < k; ++i) {
        w.h_src[i] = g->reordered ? g->h_perm[sources[i]] : sources[i];
        w.h_param[i] = params ? params[i] : sssp_graph_batch_param(g, algo);
        if (algo_needs_param(algo) && w.h_param[i] == 0) return SSSP_ERR_INVALID_ARG;
        w.h_out[i] = outs[i];
        max_param = w.h_param[i] > max_param ? w.h_param[i] : max_param;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if ((e = cudaMemcpyAsync(w.d_src, w.h_src, sizeof(uint32_t) * k, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(w.d_param, w.h_param, sizeof(uint64_t) * k, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(w.d_out, w.h_out, sizeof(uint64_t*) * k, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaEventRecord(w.copied, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.d_inst, 0, sizeof(MsInst) * k, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(w.d_ctrl, 0, sizeof(MsCtrl), st)) != cudaSuccess)
        return ms_fail(e);
    p.off = g->reordered ? g->d_off2 : g->d_off;
    p.edges = g->reordered ? g->d_edges2 : g->d_edges;
    p.perm = g->reordered ? g->d_perm : nullptr;
    p.n = g->n;
    p.K = k;
    p.R = R;
    p.rho_reduced = rho_reduced;
    p.warm_steps = warm_rho ? warm_steps : 0u;
    p.warm_rho = warm_rho;
    p.bidir = (bidir && (g->flags & SSSP_GRAPH_SYMMETRIC)) ? 1u : 0u;
    p.inst = w.d_inst;
    p.ctrl = w.d_ctrl;
    p.src = w.d_src;
    p.param = w.d_param;
    p.algo = (int)algo;
    p.sample_cap = kMaxSamples;
    p.timeout_ns = 2000000000ull;
    p.solve_timeout_ns = 120000000000ull;
    p.dist_out = w.d_out;
    void* args[] = {&p};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&ms_batch_kernel), dim3(w.grid), dim3(kMsBlock), args,
                                    kMsDynSmem, st);
    if (e != cudaSuccess) return ms_fail(e);
    w.last_k = k;
    (void)max_param;
    return SSSP_OK;
}

int ms_last_stats(int dev, sssp_stats* out, uint32_t k, cudaStream_t st)
{
    if (dev < 0 || dev >= 64) return SSSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_ms_mu);
    MsWorkspace& w = g_ms[dev];
    if (w.device < 0 || k > w.last_k || (k > 0 && !out)) return SSSP_ERR_INVALID_ARG;
    cudaError_t e = cudaMemcpyAsync(w.h_ctrl, w.d_ctrl, sizeof(MsCtrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && k) e = cudaMemcpyAsync(w.h_inst, w.d_inst, sizeof(MsInst) * k, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ms_fail(e);
    for (uint32_t i = 0; i < k; ++i) {
        const MsInst& c = w.h_inst[i];
        out[i].steps = c.last_step;
        out[i].queued = c.queued;
        out[i].extracted = c.extracted;
        out[i].edges = c.edges;
        out[i].updates = c.updates;
        out[i].status = w.h_ctrl->status;
        out[i].grid = w.grid;
    }
    return w.h_ctrl->status;
}


// ---------------------------------------------------------------------------
// host side of the shared-scan server
// ---------------------------------------------------------------------------
struct MsServer {
    void* buf = nullptr;
    MsServeParams sp;
    uint32_t grid = 0;
};

size_t ms_server_bytes(const sssp_graph* g, uint32_t S)
{
    const uint64_t n = g->n, R = (S + 3) & ~3u;
    const uint64_t rec_cap = g->fsmall_cap + g->ms_rec_cap;
    return a256(8ull * n * R) + a256(8ull * n) + 2 * a256(4ull * n) + a256(16ull * rec_cap) + a256(8ull * rec_cap) +
           a256(sizeof(MsInst) * kMsMax) + a256(sizeof(MsCtrl)) + a256(sizeof(MsServeState)) + 2 * a256(8ull * kMsMax);
}

int ms_server_create(const sssp_graph* g, uint32_t S, sssp_algo algo, uint64_t param, uint32_t rho_reduced,
                     uint32_t warm_steps, uint64_t warm_rho, bool bidir, SlotCmd* d_cmd, SlotDone* d_done, ServeShared* d_shared, uint64_t idle_ns,
                     uint32_t gang, uint64_t gang_wait_ns, MsServer** out)
{
    if (!g || !out || S == 0 || S > kMsMax || !ms_batch_supported(algo, S)) return SSSP_ERR_INVALID_ARG;
    MsServer* m = new (std::nothrow) MsServer();
    if (!m) return SSSP_ERR_OUT_OF_MEMORY;
    const size_t bytes = ms_server_bytes(g, S);
    cudaError_t e = cudaMalloc(&m->buf, bytes);
    if (e != cudaSuccess) { delete m; return ms_fail(e); }
    const uint64_t n = g->n;
    const uint32_t R = (S + 3) & ~3u;
    const uint64_t rec_cap = g->fsmall_cap + g->ms_rec_cap;
    unsigned char* b = static_cast<unsigned char*>(m->buf);
    MsParams& p = m->sp.p;
    memset(&m->sp, 0, sizeof m->sp);
    p.D = reinterpret_cast<uint64_t*>(b); b += a256(8ull * n * R);
    p.QM = reinterpret_cast<uint64_t*>(b); b += a256(8ull * n);
    p.qa = reinterpret_cast<uint32_t*>(b); b += a256(4ull * n);
    p.qb = reinterpret_cast<uint32_t*>(b); b += a256(4ull * n);
    p.rec = reinterpret_cast<uint4*>(b); b += a256(16ull * rec_cap);
    p.fm = reinterpret_cast<uint64_t*>(b); b += a256(8ull * rec_cap);
    p.inst = reinterpret_cast<MsInst*>(b); b += a256(sizeof(MsInst) * kMsMax);
    p.ctrl = reinterpret_cast<MsCtrl*>(b); b += a256(sizeof(MsCtrl));
    m->sp.st = reinterpret_cast<MsServeState*>(b); b += a256(sizeof(MsServeState));
    m->sp.src_w = reinterpret_cast<uint32_t*>(b); b += a256(8ull * kMsMax);
    uint64_t* d_param = reinterpret_cast<uint64_t*>(b);
    p.small_cap = g->fsmall_cap;
    p.big_cap = g->ms_rec_cap;
    p.off = g->reordered ? g->d_off2 : g->d_off;
    p.edges = g->reordered ? g->d_edges2 : g->d_edges;
    p.perm = g->reordered ? g->d_perm : nullptr;
    p.n = g->n;
    p.K = S;
    p.R = R;
    p.rho_reduced = rho_reduced;
    p.warm_steps = warm_rho ? warm_steps : 0u;
    p.warm_rho = warm_rho;
    p.bidir = (bidir && (g->flags & SSSP_GRAPH_SYMMETRIC)) ? 1u : 0u;
    p.src = m->sp.src_w;
    p.param = d_param;
    p.algo = (int)algo;
    p.sample_cap = kMaxSamples;
    p.timeout_ns = 2000000000ull;
    p.solve_timeout_ns = ~0ull;
    m->sp.cmd = d_cmd;
    m->sp.done = d_done;
    m->sp.shared = d_shared;
    m->sp.idle_ns = idle_ns;
    m->sp.param = param;
    m->sp.gang = gang ? (gang < S ? gang : S) : S;
    m->sp.gang_wait_ns = gang_wait_ns ? gang_wait_ns : 20000000ull;
    // zero state: empty masks, no query in any slot; every slot's parameter
    std::vector<uint64_t> prm(kMsMax, param);
    std::vector<MsInst> inst(kMsMax);
    memset(inst.data(), 0, sizeof(MsInst) * kMsMax);
    for (MsInst& x : inst) { x.qmin[0] = kInf; x.qmin[1] = kInf; x.qmin[2] = kInf; }
    if ((e = cudaMemset(p.QM, 0, 8ull * n)) != cudaSuccess ||
        (e = cudaMemset(m->sp.st, 0, sizeof(MsServeState))) != cudaSuccess ||
        (e = cudaMemset(p.ctrl, 0, sizeof(MsCtrl))) != cudaSuccess ||
        (e = cudaMemcpy(d_param, prm.data(), 8ull * kMsMax, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(p.inst, inst.data(), sizeof(MsInst) * kMsMax, cudaMemcpyHostToDevice)) != cudaSuccess) {
        cudaFree(m->buf);
        delete m;
        return ms_fail(e);
    }
    const void* fn = reinterpret_cast<const void*>(&ms_serve_kernel);
    int bps = 0, sms = 0;
    if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMsDynSmem)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, kMsBlock, kMsDynSmem)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device)) != cudaSuccess || bps < 1) {
        cudaFree(m->buf);
        delete m;
        return e != cudaSuccess ? ms_fail(e) : SSSP_ERR_CUDA;
    }
    m->grid = (uint32_t)(bps * sms);
    *out = m;
    return SSSP_OK;
}

int ms_server_launch(MsServer* m, cudaStream_t st)
{
    // the barrier word and status start from zero; the ring slots are zero
    // whenever the loop has returned (it returns only with no query queued)
    cudaError_t e = cudaMemsetAsync(m->sp.p.ctrl, 0, sizeof(MsCtrl), st);
    if (e != cudaSuccess) return ms_fail(e);
    void* args[] = {&m->sp};
    e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(&ms_serve_kernel), dim3(m->grid), dim3(kMsBlock), args,
                                    kMsDynSmem, st);
    return e == cudaSuccess ? SSSP_OK : ms_fail(e);
}

int ms_server_status(MsServer* m)
{
    MsCtrl hc;
    if (cudaMemcpy(&hc, m->sp.p.ctrl, sizeof hc, cudaMemcpyDeviceToHost) != cudaSuccess) return SSSP_ERR_CUDA;
    return hc.status;
}

void ms_server_destroy(MsServer* m)
{
    if (!m) return;
    cudaFree(m->buf);
    delete m;
}

}  // namespace sssp
