/*
 * sssp.h -- C ABI of the GB300 stepping-SSSP library (libsssp.so).
 *
 * The library computes exact single-source shortest-path distances on a
 * directed graph with unsigned 32-bit integer weights by running the stepping
 * framework of Dong, Gu, Sun, Zhang, "Efficient Stepping Algorithms and
 * Implementations for Parallel Shortest Paths" (SPAA'21; Algorithm 1 and
 * Table 2): each step picks a threshold theta (ExtDist), extracts every queued
 * vertex whose tentative distance is <= theta (Extract of the LaB-PQ, Sec. 3.1),
 * relaxes their out-edges with WriteMin and re-queues improved targets
 * (Update, Sec. 3.1).  Three ExtDist rules are offered (Table 2): rho-Stepping,
 * Delta*-Stepping and Bellman-Ford.  Every rule reaches the same, unique
 * output d(s, v) (Sec. 1 problem statement): the sum of weights of a lightest
 * s->v path, UINT64_MAX when v is unreachable.
 *
 * Conventions shared by every call:
 *   - Return value: SSSP_OK (0) or a negative sssp_status.  The library never
 *     aborts, traps or prints.
 *   - Memory: "host" pointers are ordinary CPU memory; "device" pointers are
 *     CUDA global memory of the current device (e.g. a torch CUDA tensor's
 *     data_ptr()).  Graph storage and solver scratch are owned by the library;
 *     distance outputs are owned by the caller.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy
 *     default stream).  Device work is enqueued asynchronously on it.
 *   - Threading: a graph handle may be read by many threads, but solves that
 *     share one graph handle share its scratch, so they must be ordered (one
 *     stream, or host synchronisation between them).
 */
#ifndef SSSP_H
#define SSSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sssp_graph sssp_graph; /* opaque; device copy of one CSR graph */

/* ExtDist rule (Table 2). */
typedef enum {
    SSSP_RHO = 0,           /* theta = sampled rho-th smallest queued distance (Sec. 6, App. B) */
    SSSP_DELTA_STAR = 1,    /* theta = i * Delta, i advancing every step (Table 2, Thm. 5.5)    */
    SSSP_BELLMAN_FORD = 2,  /* theta = +infinity (Table 2)                                       */
    SSSP_DELTA = 3,         /* theta = i * Delta with FinishCheck: i advances only after a step  */
                            /* that wrote no distance below i * Delta (Table 2, Delta-Stepping)  */
    SSSP_DIJKSTRA = 4       /* theta = min over Q of delta (Table 2, Dijkstra)                   */
} sssp_algo;

typedef enum {
    SSSP_OK = 0,
    SSSP_ERR_INVALID_ARG = -1,   /* a pointer, size, id or parameter is out of range            */
    SSSP_ERR_OUT_OF_MEMORY = -2, /* a device or host allocation failed                          */
    SSSP_ERR_CUDA = -3,          /* a CUDA runtime call failed (no device, launch failure, ...) */
    SSSP_ERR_TIMEOUT = -4,       /* a bounded device-wide wait ran out; outputs are undefined   */
    SSSP_ERR_INTERNAL = -5       /* a device-side capacity or step guard fired                  */
} sssp_status;

/* Per-step record written when sssp_options.trace is set (device memory). */
typedef struct {
    uint64_t theta;     /* ExtDist threshold of the step (UINT64_MAX = extract all)        */
    uint32_t queued;    /* |Q| at the start of the step                                    */
    uint32_t extracted; /* |Extract(theta)|                                                */
    uint64_t edges;     /* out-edges scanned by the extracted vertices                     */
    uint64_t updates;   /* WriteMin calls that passed the pre-check cand < delta[v]         */
    uint64_t t_ns;      /* device time from the start of the solve to the start of the step */
    uint64_t t_relax_ns;/* device time from the start of the solve to the step's relaxation */
    uint64_t t_extract_end_max; /* latest time a block finished its Extract work         */
    uint64_t t_relax_end_min;   /* earliest time a block finished its relaxation work    */
    uint64_t t_relax_end_max;   /* latest time a block finished its relaxation work      */
} sssp_step_trace;

/* Totals of the last solve (sssp_last_stats). */
typedef struct {
    uint64_t steps;     /* iterations of Algorithm 1's while loop                          */
    uint64_t queued;    /* sum over steps of |Q|                                           */
    uint64_t extracted; /* sum over steps of |Extract(theta)|                              */
    uint64_t edges;     /* sum over steps of the out-edges scanned (relaxations attempted) */
    uint64_t updates;   /* WriteMin calls that passed the pre-check cand < delta[v]        */
    int32_t status;     /* device status of the solve (an sssp_status)                     */
    uint32_t grid;      /* thread blocks of the persistent launch                          */
} sssp_stats;

/* Optional knobs of sssp_solve_ex.  Zero-initialise, then set what you need. */
typedef struct {
    uint64_t seed;           /* rho sampler seed; 0 derives it from the source            */
    uint64_t timeout_ns;     /* bound on every device-wide wait; 0 = 2 s                  */
    uint64_t max_steps;      /* 0 = no limit beyond the internal guard                    */
    uint32_t* ext_count;     /* device uint32[n] or NULL: times each vertex was extracted */
    sssp_step_trace* trace;  /* device array or NULL: one record per step                 */
    uint32_t trace_cap;      /* records available in `trace`                              */
    uint32_t grid_limit;     /* 0 = full device; else at most this many thread blocks     */
    uint32_t test_exit_block;/* testing only: 1 + index of a block that leaves before the
                                first device-wide wait (0 = none); the other blocks then
                                time out and the solve reports SSSP_ERR_TIMEOUT           */
    sssp_stats* stats_out;   /* device sssp_stats or NULL: the solve's totals are written
                                here when it ends (grid is left 0), so a sequence of
                                solves can be measured without host synchronisation       */
    uint64_t solve_timeout_ns; /* bound on the whole solve; 0 = 60 s (SSSP_ERR_TIMEOUT)  */
    uint32_t flags;          /* SSSP_SOLVE_* bits                                         */
    uint32_t local_budget;   /* local relaxation of super-sparse steps (Sec. 6, "local
                                BFS"); 0 = off.  rho- and Delta*-Stepping only
                                (INVALID_ARG for another rule when nonzero).  In a step
                                with 20*|Q| <= n whose extracted vertices have average
                                out-degree < 20, every warp keeps relaxing from the
                                vertices it has just queued while their distance is
                                <= theta (degree <= 32 each), 32 at a time, until it has
                                relaxed local_budget such vertices or runs out of
                                them in that step.  The distances are the same;
                                steps, edges and updates change (edges then counts the
                                local relaxations too).                                  */
    uint32_t shape;          /* kernel shape, SSSP_SHAPE_*; the distances do not depend on it */
    uint32_t rho_reduced;    /* rho-Stepping: how many dense steps (20*|Q| > n) use
                                rho' = max(1, rho/10) instead of rho (Sec. 6, "Threshold
                                estimation", uses the first two).  0 = 2 (the paper's
                                count); SSSP_RHO_REDUCED_NONE = none; else the count.
                                Other rules ignore it.                                   */
    uint32_t small_deg;      /* degree-bin cut-off: extracted vertices of out-degree
                                1..small_deg are relaxed as warp-flattened groups of 32,
                                larger ones as chunk records.  0 = 32; else 8..128     */
    uint32_t chunk;          /* edges per chunk record (a chunk never crosses a multiple
                                of this in the edge array).  0 = 256; else 128, 256, 512
                                or 1024.  Neither cut-off changes the distances.       */
    uint32_t rho_warmup_steps; /* rho-Stepping: the first rho_warmup_steps steps use
                                rho = rho_warmup instead, from at most 1024 samples
                                (without the dense-step reduction, and not counted among
                                the dense steps of rho_reduced), so that the first,
                                sparse waves -- which
                                on power-law graphs hold the high-degree vertices --
                                advance in small, nearly ordered groups.  0 = none (the
                                paper's schedule); rho_warmup must then be 0 too.  An
                                extension of Sec. 6's reduced rho for early steps; the
                                distances are the same.  Other rules ignore both.      */
    uint32_t rho_warmup;     /* rho of the warm-up steps (>= 1 when rho_warmup_steps > 0) */
} sssp_options;

#define SSSP_RHO_REDUCED_NONE 0xFFFFFFFFu /* sssp_options.rho_reduced: plain rho on every step */

/* sssp_options.flags */
#define SSSP_SOLVE_BIDIRECTIONAL 1u /* bidirectional relaxation (Sec. 6, "Bidirectional
                                       relaxation for undirected graphs"): before an extracted
                                       vertex u pushes to its neighbours it first takes
                                       min(delta[u], delta[v] + w) over them (WriteMin on u with
                                       the usual Update).  Needs a graph created with
                                       SSSP_GRAPH_SYMMETRIC (INVALID_ARG otherwise).  Applied to
                                       vertices relaxed as chunk records (out-degree above the
                                       small_deg cut-off).  It pulls over u's OUT-edges as if
                                       they were in-edges, so the distances are correct only
                                       when every edge (u,v,w) really has its reverse (v,u,w):
                                       on a graph declared SSSP_GRAPH_SYMMETRIC that is not
                                       symmetric the results are wrong.  Create the graph with
                                       SSSP_GRAPH_VERIFY as well unless symmetry is known.      */
#define SSSP_SOLVE_FUSED 2u         /* super-sparse steps (20*|Q| <= n, at most 4 queued ids per
                                       thread, theta the same for every block: every rule
                                       except a rho-Stepping step that samples theta) run
                                       Extract and the relaxation without the device-wide wait
                                       between them: each block relaxes the vertices it has
                                       just extracted.  Extract then overlaps other blocks'
                                       WriteMin, so an extracted vertex may be relaxed with a
                                       distance that another block lowers at the same time;
                                       each block re-checks its extracted vertices after the
                                       step and re-queues those whose distance dropped.  The
                                       distances are the same; steps and edges may differ.
                                       Used by the narrow kernel shape (SSSP_SHAPE_NARROW; the
                                       wide shape runs every step unfused), where it allocates
                                       128 bytes per thread of the launch on the graph's first
                                       such solve.  Best on graphs whose solves take thousands
                                       of small steps (road-like grids).                       */

/* sssp_options.shape: thread-block shape of the persistent solve kernel.  WIDE
   keeps the most memory operations in flight (best when steps relax many
   edges); NARROW has fewer threads with more registers each, so the per-step
   block-wide work is cheaper (best when a solve takes thousands of small
   steps, e.g. road-like graphs).  sssp_autotune measures both. */
#define SSSP_SHAPE_WIDE 0u   /* 1024 threads per block, one block per SM (default) */
#define SSSP_SHAPE_NARROW 1u /* 512 threads per block, one block per SM            */

/* sssp_graph_create_ex flags */
#define SSSP_GRAPH_SYMMETRIC 1u     /* every edge (u,v,w) has its reverse (v,u,w); taken
                                       on trust unless SSSP_GRAPH_VERIFY is also given (a
                                       false claim makes SSSP_SOLVE_BIDIRECTIONAL solves
                                       return wrong distances)                            */
#define SSSP_GRAPH_VERIFY 2u        /* check SSSP_GRAPH_SYMMETRIC on the host, O(m log d);
                                       INVALID_ARG when it does not hold                  */
#define SSSP_GRAPH_REORDER 4u       /* single solves run on a relabelled device copy: new id
                                       = rank by decreasing out-degree (ties by id), each
                                       adjacency sorted by new target, so the most frequent
                                       edge targets share cache lines; distances are
                                       returned in the caller's ids (one more pass over n
                                       at the end of the solve).  Costs a second copy of
                                       the graph and 16 bytes per vertex on the device, and
                                       O(m log d) host time at creation.  Batched and
                                       serving calls use the caller's order.              */

/*
 * Copy a CSR graph (host arrays) to the device.
 *   n        vertices, 1 <= n <= 2^32-1
 *   m        directed edges, m < 2^40
 *   offsets  host uint64[n+1]: offsets[0] = 0, non-decreasing, offsets[n] = m;
 *            the out-edges of u are [offsets[u], offsets[u+1])
 *   targets  host uint32[m], every entry < n (the graph notation of Sec. 2: N(u))
 *   weights  host uint32[m], any value (0 allowed; the paper assumes >= 1)
 *   out      receives the handle
 * Self-loops and parallel edges are accepted.  The arrays are validated in
 * O(n + m) and copied; the caller keeps ownership of them.  Errors:
 * INVALID_ARG (bad sizes, non-monotone offsets, target >= n), OUT_OF_MEMORY,
 * CUDA.  Synchronous.
 */
int sssp_graph_create(uint32_t n, uint64_t m, const uint64_t* offsets, const uint32_t* targets,
                      const uint32_t* weights, sssp_graph** out);

/* sssp_graph_create with SSSP_GRAPH_* flags (0 = sssp_graph_create). */
int sssp_graph_create_ex(uint32_t n, uint64_t m, const uint64_t* offsets, const uint32_t* targets,
                         const uint32_t* weights, uint32_t flags, sssp_graph** out);

/* Release a graph and its scratch.  Synchronises the device first. */
int sssp_graph_destroy(sssp_graph* g);

/* Vertex and edge counts of a graph (host outputs; either may be NULL). */
int sssp_graph_info(const sssp_graph* g, uint32_t* n, uint64_t* m);

/*
 * Distances from `source` (Algorithm 1 with the ExtDist of Table 2).
 *   source    vertex id < n
 *   algo      SSSP_RHO (param = rho >= 1), SSSP_DELTA_STAR and SSSP_DELTA
 *             (param = Delta >= 1), SSSP_BELLMAN_FORD and SSSP_DIJKSTRA (param ignored)
 *   dist_out  caller-owned DEVICE uint64[n]; receives d(source, v), UINT64_MAX if
 *             unreachable.  It doubles as the tentative-distance array delta of
 *             Algorithm 1 during the solve.
 *   stream    cudaStream_t as void*
 * Asynchronous: the return value covers argument checks and the launch only.
 * Device-side failures (TIMEOUT, INTERNAL) are reported by sssp_last_status
 * after the stream has completed the solve.  The whole solve is one
 * persistent kernel launch: step count, theta and queue sizes stay on the
 * device.
 */
int sssp_solve(const sssp_graph* g, uint32_t source, sssp_algo algo, uint64_t param,
               uint64_t* dist_out, void* stream);

/* sssp_solve with options (opt may be NULL = defaults). */
int sssp_solve_ex(const sssp_graph* g, uint32_t source, sssp_algo algo, uint64_t param,
                  uint64_t* dist_out, const sssp_options* opt, void* stream);

/*
 * End-to-end convenience: solve into library-owned device memory and copy the
 * distances to HOST memory `host_dist_out` (uint64[n]; pinned memory copies
 * fastest).  Synchronous; returns the device status of the solve.
 */
int sssp_solve_host(const sssp_graph* g, uint32_t source, sssp_algo algo, uint64_t param,
                    uint64_t* host_dist_out, void* stream);

/* sssp_solve_host with options (opt may be NULL = defaults). */
int sssp_solve_host_ex(const sssp_graph* g, uint32_t source, sssp_algo algo, uint64_t param,
                       uint64_t* host_dist_out, const sssp_options* opt, void* stream);

/* Waits for `stream`, then returns the device status of the last solve on g. */
int sssp_last_status(const sssp_graph* g, void* stream);

/* Waits for `stream`, then copies the totals of the last solve on g to *out. */
int sssp_last_stats(const sssp_graph* g, sssp_stats* out, void* stream);

/*
 * ExtDist of rho-Stepping alone, on the device (Sec. 6 "Threshold estimation",
 * App. B; the same device code the solve runs).  Reads the queue queue[0..q)
 * (device uint32 ids < n) and their keys dist[] (device uint64[n]); writes
 * theta to *theta_out (device uint64).  n is the vertex count, step the
 * 1-based step number, dense_before the number of earlier dense steps and
 * reduced the number of dense steps that use rho/10 (the exact count: 2 is
 * the paper's); max_samples caps the sample count (0 = 4096, the solve's
 * rule; its warm-up steps use 1024 with dense_before beyond reduced; at most
 * 4096, INVALID_ARG above).  The sample count s, its cap, the sample positions
 * (splitmix64 output step*2^32 + j from state `seed`, reduced by
 * multiply-high), the rank floor(rho'*s/q) and the dense-step rule (rho' =
 * max(1, rho/10) when 20*q > n and dense_before < reduced) are those of the
 * solve.  q <= rho' gives UINT64_MAX (extract every queued vertex).
 * Asynchronous on `stream`.
 */
int sssp_rho_threshold(const uint32_t* queue, uint32_t q, const uint64_t* dist, uint32_t n,
                       uint64_t rho, uint64_t seed, uint64_t step, uint32_t dense_before,
                       uint32_t reduced, uint32_t max_samples, uint64_t* theta_out, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched solves: many independent instances of the stepping loop (each its */
/* own source, parameter, LaB-PQ and threshold; Algorithm 1 / Table 2) in   */
/* one persistent launch.  The results equal k separate sssp_solve calls.    */
/* ------------------------------------------------------------------------ */

#define SSSP_MAX_BATCH 2048   /* instances per batched call */

/*
 * k sources on one graph (mode SSSP_BATCH_AUTO of sssp_solve_sources_ex).
 *   sources   HOST uint32[k], each < n (repeats allowed)
 *   params    HOST uint64[k] per-instance rho / Delta (as for sssp_solve), or
 *             NULL: rho = max(64, n/16), Delta = max(1, mean weight / 4)
 *   dist_out  DEVICE uint64[k * n], instance-major: instance i's distances at
 *             dist_out[i*n .. i*n + n)
 * When the graph has a tuning for `algo` (sssp_graph_get_tuning), each
 * instance also uses its bidirectional relaxation and, on graphs of at least
 * 2^20 vertices, its local-relaxation budget (sssp_options); the distances
 * do not depend on them.
 * Asynchronous on `stream`.  Working memory (per instance: queue bitmap, two
 * queue lists, extraction records) is a library-owned per-device workspace
 * grown to the largest batch seen; batched calls on one device share it, so
 * they must be ordered (one stream, or host synchronisation).  Errors:
 * INVALID_ARG (k = 0 or > SSSP_MAX_BATCH, bad source or parameter, graphs on
 * different devices), OUT_OF_MEMORY, CUDA; device-side status via
 * sssp_batch_last_stats.
 */
int sssp_solve_sources(const sssp_graph* g, const uint32_t* sources, uint32_t k, sssp_algo algo,
                       const uint64_t* params, uint64_t* dist_out, void* stream);

/* How a batch of sources on one graph is run (sssp_solve_sources_ex). */
#define SSSP_BATCH_AUTO 0u     /* the graph's batch tuning (sssp_autotune_batch) decides; without
                                  one, SHARED where it applies, else SEPARATE                    */
#define SSSP_BATCH_SHARED 1u   /* one edge scan per step shared by every instance that extracted
                                  the vertex (k <= 64; rho-Stepping, Delta*-Stepping,
                                  Bellman-Ford): distances are kept vertex-major inside, so one
                                  vertex's k distances share cache lines.  Uses the graph's
                                  bidirectional relaxation setting (batch tuning); no local
                                  relaxation.  INVALID_ARG when it does not apply               */
#define SSSP_BATCH_SEPARATE 2u /* independent instances (any k and rule; each instance uses its
                                  graph's bidirectional and local relaxation settings)           */

/* sssp_solve_sources with an explicit SSSP_BATCH_* mode.  The distances do not
   depend on the mode. */
int sssp_solve_sources_ex(const sssp_graph* g, const uint32_t* sources, uint32_t k, sssp_algo algo,
                          const uint64_t* params, uint32_t mode, uint64_t* dist_out, void* stream);

/*
 * k independent graphs, one source each (instance i solves gs[i] from
 * sources[i] into dist_outs[i], a DEVICE uint64[n_i]).  gs and dist_outs are
 * HOST arrays of k entries; graphs may repeat.  Otherwise as
 * sssp_solve_sources.
 */
int sssp_solve_multi(const sssp_graph* const* gs, const uint32_t* sources, uint32_t k, sssp_algo algo,
                     const uint64_t* params, uint64_t* const* dist_outs, void* stream);

/*
 * Waits for `stream`, then copies the per-instance totals of the last batched
 * call on the current device to HOST out[0..k) (k <= that call's k) and
 * returns its device status (SSSP_OK, SSSP_ERR_TIMEOUT, SSSP_ERR_INTERNAL).
 */
int sssp_batch_last_stats(sssp_stats* out, uint32_t k, void* stream);

/* ------------------------------------------------------------------------ */
/* Serving: a query server with continuous batching over resident graphs.    */
/* Queries (one source each) are admitted into device slots as slots free up;*/
/* a query that arrives while others run joins them at the next step        */
/* boundary of a long-lived persistent launch, so their steps overlap on the */
/* device.  Each result equals the single solve of the same source.         */
/* ------------------------------------------------------------------------ */

typedef struct sssp_server sssp_server;

typedef struct {
    uint32_t slots;        /* queries on the device at once; 0 = the graph's batch   */
                           /* tuning's slots, else as many as fit                    */
    sssp_algo algo;        /* ExtDist rule of every query                            */
    uint64_t param;        /* rho / Delta; 0 = max(64, n/16) / max(1, mean weight/4) */
    uint64_t idle_ns;      /* the device loop exits after this long without a query  */
                           /* (0 = 2 ms; at most 1 s); it restarts on the next query */
    double hbm_fraction;   /* share of free HBM the slots may take (0 = 0.5)         */
    uint32_t batch_mode;   /* SSSP_BATCH_*: SHARED runs the slots as the instances of */
                           /* one shared edge scan (at most 64 slots; rho, Delta*,    */
                           /* Bellman-Ford), SEPARATE as independent instances; AUTO */
                           /* (0) follows the graph's batch tuning, else SHARED where */
                           /* it applies                                              */
    uint32_t gang;         /* SHARED: waiting queries are admitted together once this */
                           /* many wait (queries that start together stay aligned,    */
                           /* which is what the shared scan shares), when nothing    */
                           /* else runs, or after gang_wait_ns; 0 = every slot        */
    uint64_t gang_wait_ns; /* 0 = 20 ms; at most 1 s                                  */
} sssp_server_config;

typedef struct {
    int32_t status;        /* device status of the query (SSSP_OK, ...)              */
    uint32_t steps;        /* steps the query took                                   */
    uint64_t latency_ns;   /* host: submit -> completion seen by the server thread   */
    uint64_t device_ns;    /* device: admission -> completion                        */
    uint64_t device_admit_ns, device_done_ns; /* device clock at admission / completion */
    uint64_t edges;        /* edges the query scanned                                */
} sssp_query_info;

/*
 * Create a server for graph g.  Slots are admitted by free HBM: the slots'
 * working memory comes out of hbm_fraction of the free device memory, capped
 * at cfg->slots (and at SSSP_MAX_BATCH, or 64 in SSSP_BATCH_SHARED mode).  In
 * SHARED mode the slots are the instances of one shared edge scan (per slot
 * one vertex-major distance column: a query's column is reset when it is
 * admitted and copied to its dist_out when its queue empties); in SEPARATE
 * mode each slot has its own queue bitmap, lists and records.  Starts a host
 * thread that assigns queries to slots, keeps the device loop running while
 * there is work and collects completions (through host-mapped memory).  While
 * the device loop runs it occupies every SM.  Errors: INVALID_ARG (also SHARED
 * for a rule it does not cover), OUT_OF_MEMORY (not one slot fits), CUDA.
 */
int sssp_server_create(const sssp_graph* g, const sssp_server_config* cfg, sssp_server** out);

/* Number of slots the server got. */
int sssp_server_slots(const sssp_server* s, uint32_t* slots);

/* The SSSP_BATCH_* mode the server runs its slots in (SHARED or SEPARATE). */
int sssp_server_mode(const sssp_server* s, uint32_t* mode);

/*
 * Queue a query; non-blocking, thread-safe.  dist_out: caller-owned DEVICE
 * uint64[n] that receives the distances (it must stay valid and untouched
 * until the query completes).  *ticket identifies the query.
 */
int sssp_server_submit(sssp_server* s, uint32_t source, uint64_t* dist_out, uint64_t* ticket);

/* 1 and *info when the query is complete (the ticket is then released), 0 while
 * pending, a negative status on error. */
int sssp_server_poll(sssp_server* s, uint64_t ticket, sssp_query_info* info);

/* As sssp_server_poll, but blocks until completion or timeout_ns (0 = 60 s;
 * SSSP_ERR_TIMEOUT then). */
int sssp_server_wait(sssp_server* s, uint64_t ticket, uint64_t timeout_ns, sssp_query_info* info);

/* Completion queue: copies up to max completed, not yet collected queries to
 * HOST tickets[] / infos[] (in completion order; they are then released) and
 * returns how many (0 when none; a negative status after a device failure). */
int sssp_server_drain(sssp_server* s, uint64_t* tickets, sssp_query_info* infos, uint32_t max);

/* Device-loop launches so far, slots in use, queries waiting for a slot. */
int sssp_server_stats(const sssp_server* s, uint64_t* launches, uint32_t* busy_slots, uint64_t* pending);

/* Stop the device loop and the host thread, release everything.  Queries not
 * yet complete are abandoned. */
int sssp_server_destroy(sssp_server* s);

/* Largest graph sssp_solve_noalloc accepts. */
#define SSSP_NOALLOC_MAX_VERTICES (1u << 18)   /* 262,144 vertices            */
#define SSSP_NOALLOC_MAX_EDGES (1ull << 22)    /* 4,194,304 directed edges     */

/*
 * A solve that allocates nothing.  (The paper has no counterpart: this is a
 * systems entry point of this library.)  It is meant for callers that cannot
 * allocate device memory when they need a solve -- a plugin whose enqueue step
 * runs inside a framework that owns all device memory through its own pool,
 * or a latency-critical loop that cannot take the implicit device
 * synchronisation of cudaMalloc/cudaFree.  It calls no cudaMalloc, cudaFree
 * or other allocating routine.
 *
 * The solver's working memory is a file-scope device array of about 10.4 MB,
 * sized for SSSP_NOALLOC_MAX_VERTICES and SSSP_NOALLOC_MAX_EDGES; every GPU
 * that loads it keeps it until the process exits.  All calls on a device
 * share that array and it keeps the last call's contents (each call clears
 * what must start from zero): calls that overlap on the GPU (different
 * streams, or host threads without ordering) race and give undefined results;
 * order them.  The first call on a device does a one-time set-up with that
 * device current: it looks up the array's device address and the launch
 * grid, and keeps both for the life of the process; make that first call
 * before any stream capture begins.  A cudaDeviceReset of the device discards
 * the array, so the entry point must not be called on that device after one.
 *
 *   n, m       vertex and edge counts; n in [1, SSSP_NOALLOC_MAX_VERTICES],
 *              m <= SSSP_NOALLOC_MAX_EDGES, otherwise SSSP_ERR_INVALID_ARG
 *   offsets    DEVICE uint64[n+1], a valid CSR (offsets[0] = 0, non-decreasing,
 *              offsets[n] = m); not checked (it is in device memory)
 *   edges      DEVICE uint32 array of (target, weight) pairs, pair e at
 *              edges[2e], edges[2e+1]; 16-byte aligned; it must hold an even
 *              number of pairs (when m is odd, the pair slot m is read and
 *              ignored); every target < n (not checked)
 *   source, algo, param   as for sssp_solve
 *   dist_out   DEVICE uint64[n], receives the distances
 *   stats_out  DEVICE sssp_stats or NULL: the solve's totals and device status
 *              (SSSP_OK, SSSP_ERR_TIMEOUT, SSSP_ERR_INTERNAL) once the stream
 *              has run the solve
 *   stream     cudaStream_t as void*
 * Asynchronous; the return value covers the argument checks and the launch.
 * Results are identical to sssp_solve's.
 */
int sssp_solve_noalloc(uint32_t n, uint64_t m, const uint64_t* offsets, const uint32_t* edges,
                       uint32_t source, sssp_algo algo, uint64_t param, uint64_t* dist_out,
                       sssp_stats* stats_out, void* stream);

/* ------------------------------------------------------------------------ */
/* Autotuner.  (The paper fixes rho per graph family -- 2^21 for social and  */
/* web graphs, 2^15 for road networks, Sec. 7 -- and sweeps it; this library */
/* measures instead.)                                                       */
/* ------------------------------------------------------------------------ */

/* A solve configuration: the ExtDist rule and its parameter (Table 2), the
   kernel shape, the SSSP_SOLVE_* flags and the local-relaxation budget
   (sssp_options).  The distances do not depend on it. */
typedef struct {
    sssp_algo algo;          /* SSSP_RHO or SSSP_DELTA_STAR (or SSSP_BELLMAN_FORD)          */
    uint32_t shape;          /* SSSP_SHAPE_*                                                */
    uint64_t param;          /* rho or Delta                                                */
    uint32_t flags;          /* SSSP_SOLVE_* (bidirectional relaxation on symmetric graphs,
                                fused super-sparse steps)                                 */
    uint32_t local_budget;   /* sssp_options.local_budget                                   */
    double ms;               /* autotuner: mean solve time of the choice on the samples     */
    uint32_t candidates;     /* autotuner: configurations timed                             */
    uint32_t slots;          /* batch autotuner: concurrent queries with the highest
                                throughput (the server's slot count when its config
                                gives none); 0 = not measured                          */
    uint32_t rho_reduced;    /* sssp_options.rho_reduced (0 = the paper's 2)                */
    uint32_t small_deg;      /* sssp_options.small_deg (0 = 32; single solves only)         */
    uint32_t chunk;          /* sssp_options.chunk (0 = 256; single solves only)            */
    uint32_t batch_mode;     /* batch autotuner: SSSP_BATCH_SHARED or SSSP_BATCH_SEPARATE   */
    uint32_t rho_warmup_steps; /* sssp_options.rho_warmup_steps (single solves and
                                shared-scan batches; the separate-instance kernel and the
                                server ignore it)                                          */
    uint32_t rho_warmup;     /* sssp_options.rho_warmup                                     */
} sssp_tuning;

/*
 * Time candidate configurations on the k sample sources (HOST uint32[k], each
 * < n) and keep the fastest: rho in {n/4, n/8, ..., n/1024} (at least 64) and
 * Delta in mean-weight x {1/8, 1/4, ..., 8} in the wide shape on the first
 * source; the two best in both shapes on up to three sources (as every
 * later stage); on graphs with mean
 * out-degree < 20 the three best parameters of each rule in the winning shape
 * with local budgets 64, 256, 1024 and in the narrow shape with
 * SSSP_SOLVE_FUSED and local budgets 0, 64, 256, 1024; for a rho winner the
 * count of dense steps at rho/10 (2, 4, 6, 8, none), then 4, 6 or 8 warm-up
 * steps at rho 256 (rho_warmup_steps; with that count, 2, 4 or 6 reduced
 * dense steps after them); the degree-bin cut-offs
 * (small_deg 16, 32, 64, then chunk 128, 256, 512); the winner is re-timed on
 * all k sources.
 * Bidirectional relaxation is used when the graph was created
 * SSSP_GRAPH_SYMMETRIC.  The result is stored on the graph and in
 * a per-class table (sssp_graph_class) that sssp_solve_tuned, sssp_solve_sources,
 * sssp_solve_multi (params == NULL) and the server (param == 0) use for graphs
 * of the same class that were not tuned themselves.  Synchronous on `stream`;
 * allocates a temporary distance array.  out may be NULL.
 */
int sssp_autotune(sssp_graph* g, const uint32_t* sources, uint32_t k, sssp_tuning* out, void* stream);

/* sssp_autotune over a subset of the rules: `rules` is a bit mask of
   (1 << SSSP_RHO) and (1 << SSSP_DELTA_STAR) (e.g. rho only, for batched calls
   that run every instance with rho-Stepping); INVALID_ARG for other bits or 0. */
int sssp_autotune_ex(sssp_graph* g, const uint32_t* sources, uint32_t k, uint32_t rules, sssp_tuning* out,
                     void* stream);

/* The best configuration of batched launches of k sources on g (HOST
   uint32[k], k <= SSSP_MAX_BATCH): rho / Delta candidates as in
   sssp_autotune's first stage (rules: as sssp_autotune_ex), each timed as one
   sssp_solve_sources launch over up to 8 of the sources, the two best of each
   rule re-timed on all k (for k <= 64 also with one shared edge scan,
   SSSP_BATCH_SHARED, with 2 or 6 reduced dense steps, or 8 warm-up steps at
   rho 256 and 4 reduced steps); on graphs of >= 2^20 vertices and mean degree < 20
   local budgets 0, 64, 256 for each of those of the separate-instance
   kernel; for a rho winner the count of dense steps at rho/10 (4, 6, 8,
   none); then the winner's throughput
   with 1, 4 and 16 concurrent sources (those < k) against k, the best count
   recorded as `slots`.  Kept as the graph's batch tuning, which
   sssp_solve_sources / sssp_solve_multi (params == NULL) and the server
   (param == 0) use before the single-solve tuning.  Synchronous; allocates k*n
   distances for the measurements.  ms = time of one batched launch. */
int sssp_autotune_batch(sssp_graph* g, const uint32_t* sources, uint32_t k, uint32_t rules, sssp_tuning* out,
                        void* stream);

/* The tuning that applies to g (its own, else its class's); INVALID_ARG when none. */
int sssp_graph_get_tuning(const sssp_graph* g, sssp_tuning* out);

/* Attach a configuration to g (e.g. one tuned on another graph). */
int sssp_graph_set_tuning(sssp_graph* g, const sssp_tuning* t);

/* Class key of a graph: bits 0-7 ceil(log2 n), 8-15 round(4 log2(m/n)),
   16-23 floor(log2(max out-degree / mean out-degree)), bit 24 symmetric. */
int sssp_graph_class(const sssp_graph* g, uint64_t* key);

/* sssp_solve with the configuration that applies to g (sssp_graph_get_tuning),
   else rho-Stepping with rho = max(64, n/16). */
int sssp_solve_tuned(const sssp_graph* g, uint32_t source, uint64_t* dist_out, void* stream);

/* ------------------------------------------------------------------------ */
/* Tournament-tree LaB-PQ (Sec. 4.2, Algorithm 2, Theorem 4.1) on the device, */
/* as a stand-alone data structure: a complete binary tree over the records  */
/* 0..n-1 whose interior nodes keep the smallest key below them.  Keys are    */
/* read from a caller's key array (device uint64[n], "delta" of Sec. 3.1);    */
/* every change of a record's key must be followed by an update of that       */
/* record (as Algorithm 1 does with Update).  Calls are asynchronous on       */
/* `stream` and must be ordered on one stream.                                */
/* ------------------------------------------------------------------------ */

typedef struct sssp_tourney sssp_tourney;

/* An empty tree over n records (1 <= n <= 2^31).  Synchronous. */
int sssp_tourney_create(uint32_t n, sssp_tourney** out);
int sssp_tourney_destroy(sssp_tourney* t);

/* LazyInsert / Update (Algorithm 2: Mark(id, 1)) of a batch of b record ids
   (DEVICE uint32[b]; ids >= n are ignored; repeats allowed). */
int sssp_tourney_update(sssp_tourney* t, const uint32_t* ids, uint32_t b, void* stream);

/* Extract(theta) (Algorithm 2): every record in Q whose key is <= theta leaves
   Q; their ids go to out (DEVICE uint32[n], in no particular order) and their
   number to *count_out (DEVICE uint32). */
int sssp_tourney_extract(sssp_tourney* t, const uint64_t* keys, uint64_t theta, uint32_t* out,
                         uint32_t* count_out, void* stream);

/* Reduce (Sec. 3.1, min): the smallest key in Q (UINT64_MAX when Q is empty)
   to *min_out (DEVICE uint64). */
int sssp_tourney_min(sssp_tourney* t, const uint64_t* keys, uint64_t* min_out, void* stream);

/* Copy of the inQ flags (DEVICE uint32[ceil(n/32)], bit id of word id/32). */
int sssp_tourney_inq(const sssp_tourney* t, uint32_t* inq_out, void* stream);

/* Extract of the array-based LaB-PQ (Sec. 4.3) as a stand-alone operation, for
   comparison with the tree (App. F): the ids of list[0..q) (DEVICE) whose key
   is <= theta go to ext, the others to keep (DEVICE uint32[q] each), their
   numbers to *ext_count / *keep_count (DEVICE uint32). */
int sssp_array_extract(const uint32_t* list, uint32_t q, const uint64_t* keys, uint64_t theta, uint32_t* ext,
                       uint32_t* ext_count, uint32_t* keep, uint32_t* keep_count, void* stream);

/* Static description of a status code (never NULL). */
const char* sssp_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* SSSP_H */
