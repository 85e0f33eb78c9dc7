/*
 * sssp.h -- C ABI of the GB300 library for Garg's bound-based single-source
 * shortest paths (arXiv 1812.10499, "Removing Sequential Bottleneck of
 * Dijkstra's Algorithm for the Shortest Path Problem").
 *
 * Problem (Sec. I and Sec. II): a directed graph with n vertices and m edges
 * and strictly positive integer weights; find cost[x], the minimum weight of a
 * path from the source v0 to every vertex x.  The library runs the
 * data-parallel round of SP_3/SP_4 (Sec. V, Sec. VI): each round
 *   (a) relaxes the out-edges of the vertices fixed in the previous round,
 *       lowering the upper bounds D (SP_4 step 3, label-setting as in SP_3);
 *   (b) raises the lower bounds C of the discovered, unfixed vertices with
 *       Eq. (1) of Lemma 6 over their in-edges, clamped by
 *       min(D, threshold) from Lemmas 7 and 8 (SP_4 steps 1 and 4);
 *   (c) fixes every vertex whose C equals its D (SP_4 step 5) and makes the
 *       newly fixed vertices the next round's frontier.
 * All arithmetic is exact 64-bit integer; results are bit-identical to a
 * sequential execution of the same rounds.
 *
 * Conventions for every entry point:
 *   - Return value: SSSP_OK (0) on success, a negative SSSP_E_* code on
 *     failure; sssp_strerror() names it.  On failure, outputs are unspecified
 *     and no input is modified.
 *   - Host pointers are caller-owned and only read during the call (inputs)
 *     or written before the call returns (outputs); nothing is retained.
 *   - Device pointers ("_dev", "_device") are CUDA global-memory addresses on
 *     the handle's device; the caller owns them.
 *   - A handle may be used by one host thread at a time.
 *   - Unreachable vertices get distance SSSP_DIST_INF (UINT64_MAX).
 */
#ifndef SSSP_H
#define SSSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SSSP_OK                 0
#define SSSP_E_INVAL           (-1)  /* malformed argument (NULL, bad CSR, n = 0, ...)      */
#define SSSP_E_ZERO_WEIGHT     (-2)  /* an edge weight is 0; Sec. I requires w > 0          */
#define SSSP_E_SOURCE_RANGE    (-3)  /* source vertex >= n                                  */
#define SSSP_E_OVERFLOW        (-4)  /* n * max weight does not fit the packed distance     */
#define SSSP_E_NOMEM           (-5)  /* device allocation failed or budget exhausted        */
#define SSSP_E_DEVICE_TIMEOUT  (-6)  /* a bounded device-side wait gave up                  */
#define SSSP_E_CUDA            (-7)  /* a CUDA runtime call failed                          */
#define SSSP_E_ROUND_LIMIT     (-8)  /* more rounds than vertices: internal invariant broken */
#define SSSP_E_BUSY            (-9)  /* server has no free slot / budget for this query      */
#define SSSP_E_NOT_FOUND      (-10)  /* unknown ticket                                      */
#define SSSP_E_INTERNAL       (-11)  /* a device-side consistency guard tripped (library bug) */
#define SSSP_E_NOALLOC_LIMIT  (-12)  /* graph larger than the fixed scratch of sssp_solve_noalloc */
#define SSSP_PENDING            1    /* sssp_serve_poll: query still running                 */

#define SSSP_DIST_INF UINT64_MAX

/* Lower-bound clamp used in step (b).
 *   SSSP_RULE_THRESHOLD: C[y] >= min(D[y], threshold), the combination of
 *     Lemma 7 (crule2) and Lemma 8 (Crauser et al. out-version); subsumes
 *     SP_4 step 2's "fix D <= threshold".
 *   SSSP_RULE_MIND: C[y] >= minD over the unfixed set (SP_4 step 4 as
 *     printed) plus SP_4 step 2 (fix D <= threshold).  Same distances, the
 *     round count may differ. */
#define SSSP_RULE_THRESHOLD 0u
#define SSSP_RULE_MIND      1u
/* Flag OR-ed into the rule: label-correcting relaxation, SP_4 step 3 as
 * printed (Sec. VI) -- every round relaxes the out-edges of every vertex whose
 * D changed in the previous round's relaxation (with its D from the start of
 * the relaxation), not only of the vertices fixed in the previous round; the
 * loop ends when a relaxation changes nothing.  Distances are the same; the
 * rounds, the work and the fixing rounds differ (vertices whose D is final
 * may stay unfixed: fixed_round -1 for a reachable vertex is possible).
 * Not available for the server (sssp_serve_submit returns SSSP_E_INVAL). */
#define SSSP_RULE_LABEL_CORRECTING 2u
/* Flag OR-ed into the rule: before scanning the in-edges of an active y, fix
 * y at once when D[y] <= minD + inWeight[y] (the in-version rule of SP_2,
 * Sec. IV, inWeight = least in-edge weight) or D[y] <= threshold (Lemma 8).
 * Both imply that Eq. (1) gives C[y] = D[y], so every output is unchanged;
 * only in_scanned (the in-edges actually read) drops. */
#define SSSP_RULE_CHEAP_FIRST 4u
/* Flag OR-ed into the rule: windowed relaxation, a combination of the lower
 * bounds with Delta-stepping (Sec. I notes that the two can be combined).
 * Delta-stepping's current bucket becomes a window of width
 * sssp_options.delta above minD: after step (c) the next frontier is every
 * vertex whose D changed since it last relaxed and that is either fixed now
 * or still active with D < minD + delta.  The loop runs while a frontier or
 * an active vertex is left.  delta = 0 gives exactly the default
 * label-setting round; a delta above every distance relaxes every changed
 * vertex as SSSP_RULE_LABEL_CORRECTING does (but every reachable vertex is
 * fixed in the end).  Distances are the same; rounds, work and fixing
 * rounds depend on delta.  Not combinable with SSSP_RULE_LABEL_CORRECTING;
 * not available for the server. */
#define SSSP_RULE_WINDOWED 16u
/* Flag OR-ed into the rule: SP_1's predecessor counts (Sec. III).  Each
 * vertex counts its in-edges that have not yet been relaxed; the relaxation
 * of an edge into an unfixed vertex decrements the count (one atomic per such
 * edge).  An active y whose count is 0 -- every in-neighbour is fixed and
 * has relaxed into y, so D[y] is final -- is fixed without reading its
 * in-edges.  Eq. (1) fixes such a y in the same round (every term is
 * D[x] + w >= D[y]), so every output is unchanged; only in_scanned drops.
 * Combinable with SSSP_RULE_MIND and SSSP_RULE_CHEAP_FIRST; not with
 * SSSP_RULE_LABEL_CORRECTING or SSSP_RULE_WINDOWED (sssp_create returns
 * SSSP_E_INVAL); not available for the server.  Costs 4 bytes of device
 * memory per vertex (per record in a batch). */
#define SSSP_RULE_PRED_COUNT 32u

/* How the rounds are sequenced.  All modes give identical results. */
#define SSSP_LOOP_GRAPH      0u  /* two kernels per round in a CUDA graph with a device-side
                                    while loop (default)                                  */
#define SSSP_LOOP_HOST       1u  /* host launches the two kernels in groups of rounds and
                                    polls a status word                                   */
#define SSSP_LOOP_PERSISTENT 2u  /* one cooperative launch runs every round, phases
                                    separated by grid barriers whose waits time out
                                    (SSSP_E_DEVICE_TIMEOUT) instead of hanging            */

/* Per-vertex state layout of the round kernels.  Results are identical.
 *   SSSP_LAYOUT_AUTO     compact when n * max weight < 2^31, else wide (default)
 *   SSSP_LAYOUT_WIDE     32-byte records: packed D, two C words, outWeight and
 *                        in-degree of the vertex
 *   SSSP_LAYOUT_COMPACT  16-byte records: packed D and two 31-bit C words;
 *                        outWeight and in-degree are read from the graph.
 *                        sssp_create fails with SSSP_E_OVERFLOW when
 *                        n * max weight >= 2^31. */
#define SSSP_LAYOUT_AUTO    0u
#define SSSP_LAYOUT_WIDE    1u
#define SSSP_LAYOUT_COMPACT 2u

typedef struct sssp_graph* sssp_handle;
typedef struct sssp_server sssp_server;

/* Device-memory allocator hook.  alloc returns a device pointer aligned to at
 * least 256 bytes or NULL; free releases it.  Both are called only from
 * sssp_create / sssp_destroy / sssp_serve_open / sssp_serve_close.  NULL
 * hooks mean cudaMalloc / cudaFree. */
typedef void* (*sssp_alloc_fn)(size_t bytes, void* ctx);
typedef void (*sssp_free_fn)(void* ptr, void* ctx);

typedef struct sssp_options {
    uint32_t rule;           /* SSSP_RULE_*                                                */
    uint32_t loop_mode;      /* SSSP_LOOP_*                                                */
    uint32_t hub_degree;     /* vertices of degree > hub_degree are split into chunks
                                processed by many warps (0 = library default, 256)         */
    uint32_t chunk_edges;    /* edges per hub chunk (0 = default 1024, must be a multiple
                                of 32)                                                     */
    uint32_t block_threads;  /* threads per CTA of the round kernels (0 = 256)             */
    uint32_t ctas_per_sm;    /* CTAs per SM of the round kernels (0 = from occupancy)      */
    int32_t device;          /* CUDA device ordinal (-1 = the calling thread's current)    */
    uint32_t layout;         /* SSSP_LAYOUT_* (batched solves use the compact layout only
                                when every graph of the batch does)                        */
    sssp_alloc_fn alloc;     /* NULL = cudaMalloc                                          */
    sssp_free_fn free;       /* NULL = cudaFree                                            */
    void* alloc_ctx;
    uint64_t delta;          /* window width of SSSP_RULE_WINDOWED, in weight units
                                (0 = the label-setting round)                              */
} sssp_options;

/* Fills *opt with the defaults described above.  hub_degree, chunk_edges
 * and ctas_per_sm are left 0: the library chooses them (from the tuning
 * cache when it holds the graph's class, else its defaults). */
void sssp_options_default(sssp_options* opt);

/* Launch shape of the round kernels for one graph (or one batch).  None of
 * these changes any result (every output is bit-identical); they change only
 * how the work is spread over the GPU.  The paper has no counterpart: this
 * is the GPU's tuning. */
typedef struct sssp_tuning {
    uint32_t hub_degree;     /* vertices of degree > hub_degree are split into chunks of
                                chunk_edges edges, each handled by one warp (1..2^20)     */
    uint32_t chunk_edges;    /* edges per hub chunk: a multiple of 32, 32..2^20           */
    uint32_t ctas_per_sm;    /* CTAs of 256 threads per SM of the round kernels
                                (0 = as many as fit)                                       */
    uint32_t tail_items;     /* rounds whose frontier and active set each make at most this
                                many work items (32-vertex tiles and hub chunks) run in the
                                16-CTA cluster kernel (0 = never)                          */
} sssp_tuning;

/* The tuning a handle's solves use.  Errors: SSSP_E_INVAL. */
int sssp_get_tuning(sssp_handle h, sssp_tuning* out);

/* Sets a handle's tuning (recomputes the hub flags, list capacities and
 * solve contexts; the graph is not copied again).  Errors: SSSP_E_INVAL for
 * a value out of range, SSSP_E_NOMEM, SSSP_E_CUDA. */
int sssp_set_tuning(sssp_handle h, const sssp_tuning* t);

/* The key of a graph's class in the tuning cache, from its vertex and edge
 * counts, largest out- and in-degree, largest weight and state layout
 * (compact when n * max weight < 2^31), each rounded to a power of two (the
 * average degree to a half power): graphs of one class share a tuning.
 * Writes a NUL-terminated string of at most 95 characters.  Host-only.
 * Errors: SSSP_E_INVAL (cap < 96). */
int sssp_tune_key(uint32_t n, uint64_t m, uint32_t max_out_degree, uint32_t max_in_degree,
                  uint32_t max_weight, char* key, size_t cap);

/* The key of a handle's graph (as sssp_tune_key).  Errors: SSSP_E_INVAL. */
int sssp_graph_key(sssp_handle h, char* key, size_t cap);

/* Process-wide tuning cache, persisted as a JSON object {key: {"hub_degree":
 * .., "chunk_edges": .., "ctas_per_sm": .., "tail_items": ..}, ...}.  sssp_tune_cache_open loads `path` (a missing file is an empty
 * cache) and makes later puts write it back (NULL: an in-memory cache only);
 * without a call, the first use opens the file named by the environment
 * variable SSSP_TUNE_CACHE, if set.  sssp_create looks up the graph's class
 * when its options leave hub_degree and chunk_edges 0; sssp_solve_batch
 * looks up the batch's class.  Host-only; thread-safe.  Errors:
 * SSSP_E_INVAL (unreadable or malformed file), SSSP_E_NOT_FOUND (get: no
 * entry), SSSP_E_CUDA never. */
int sssp_tune_cache_open(const char* path);
int sssp_tune_cache_get(const char* key, sssp_tuning* out);
int sssp_tune_cache_put(const char* key, const sssp_tuning* t);

typedef struct sssp_tune_result {
    sssp_tuning best;        /* the fastest tuning found                                   */
    double start_ms;         /* device time of one pass over the sources with the tuning
                                in place before the sweep                                  */
    double best_ms;          /* the same with `best`                                       */
    uint32_t evaluated;      /* tunings timed                                              */
    uint32_t reserved;
} sssp_tune_result;

/* Autotuner: times single-source solves from `sources` (nsrc >= 1) on the
 * device for candidate tunings -- hub degree with chunk size, then the
 * cluster-tail work-item limit, then CTAs per SM, one parameter
 * group at a time starting from the handle's current tuning -- keeping the
 * fastest (best of `reps` passes, reps 0 = 3).  The winner is set on the
 * handle and put in the tuning cache under the graph's key.  Results of
 * every solve are unchanged.  Errors: as sssp_solve, SSSP_E_INVAL. */
int sssp_autotune(sssp_handle h, const uint32_t* sources, uint32_t nsrc, uint32_t reps,
                  sssp_tune_result* out);

/* The same for a batch (as sssp_solve_batch: query i is (g[i], sources[i])):
 * times whole batched solves and puts the winner in the cache under the
 * batch's key (its query count, vertex and edge totals and largest graph,
 * rounded to powers of two), where sssp_solve_batch finds it.  The handles'
 * own tunings are not changed. */
int sssp_autotune_batch(const sssp_handle* g, const uint32_t* sources, uint32_t k, uint32_t reps,
                        sssp_tune_result* out);

/* The key of a batch's class (see sssp_autotune_batch).  Errors: SSSP_E_INVAL. */
int sssp_batch_key(const sssp_handle* g, uint32_t k, char* key, size_t cap);

/* Builds a device-resident graph (Sec. II: out-edges for relaxation; Sec. IV:
 * in-edges, needed by the lower-bound rule of Lemma 6).
 *   n        number of vertices, 1 <= n < 2^32 - 1
 *   m        number of edges (entries of col / w)
 *   row_ptr  host u64[n+1], CSR offsets: out-edges of u are
 *            col[row_ptr[u] .. row_ptr[u+1]); row_ptr[0] = 0, row_ptr[n] = m,
 *            non-decreasing
 *   col      host u32[m], edge targets (< n)
 *   w        host u32[m], edge weights (> 0)
 *   col_ptr, row, w_in: optional host CSC of the same edge multiset (in-edges
 *            of v are row/w_in[col_ptr[v] .. col_ptr[v+1])); pass all three
 *            NULL to have the library transpose on the device.
 *   opt      NULL for defaults.
 * Self-loops (u, u) are dropped (Sec. II assumes a loop-free graph; a loop
 * never lies on a shortest path).  Multi-edges are kept.  Vertices without
 * in-edges are allowed (they are unreachable unless they are the source).
 * Errors: SSSP_E_INVAL, SSSP_E_ZERO_WEIGHT, SSSP_E_OVERFLOW (when
 * n * max(w) >= 2^(64 - ceil(log2 n)) - 1: distance and parent share one
 * 64-bit word), SSSP_E_NOMEM, SSSP_E_CUDA.  *out is set only on success. */
int sssp_create(uint32_t n, uint64_t m, const uint64_t* row_ptr, const uint32_t* col,
                const uint32_t* w, const uint64_t* col_ptr, const uint32_t* row,
                const uint32_t* w_in, const sssp_options* opt, sssp_handle* out);

/* Single-source shortest paths from `source` (Sec. VI, rounds until no vertex
 * is left to explore).  dist_out: host u64[n], written on success (an array
 * from sssp_host_alloc is written directly by the device, any other through
 * a copy).  rounds_out (nullable): number of rounds executed (relaxation
 * steps, including the last one that finds nothing new).  Blocks until done.
 * Errors: SSSP_E_INVAL, SSSP_E_SOURCE_RANGE, SSSP_E_ROUND_LIMIT,
 * SSSP_E_DEVICE_TIMEOUT (a bounded device wait of the persistent loop gave
 * up), SSSP_E_INTERNAL (a device-side guard tripped), SSSP_E_CUDA. */
int sssp_solve(sssp_handle h, uint32_t source, uint64_t* dist_out, uint32_t* rounds_out);

/* Same as sssp_solve, but dist_dev is a device u64[n] and the work is
 * enqueued on `cuda_stream` (a cudaStream_t; NULL = the legacy default
 * stream).  If rounds_out is NULL the call returns without synchronising;
 * otherwise it waits for the stream and reports the round count. */
int sssp_solve_device(sssp_handle h, uint32_t source, uint64_t* dist_dev, uint32_t* rounds_out,
                      void* cuda_stream);

/* Optional outputs and counters of one solve (all output pointers nullable;
 * "dev" selects device pointers instead of host pointers). */
typedef struct sssp_solve_args {
    uint64_t* dist;          /* u64[n]: cost[x] or SSSP_DIST_INF                           */
    uint32_t* parent;        /* u32[n]: predecessor on a shortest path (source: itself;
                                unreachable: UINT32_MAX); among equal distances the
                                smallest predecessor id                                    */
    int32_t* fixed_round;    /* i32[n]: round in which x was fixed (source 0, never: -1)   */
    uint64_t* lower;         /* u64[n]: final lower bound C[x]                             */
    uint32_t max_rounds;     /* stop after this many rounds (0 = run to completion); the
                                outputs then hold the state after that round               */
    uint32_t dev;            /* 1: output pointers are device pointers                     */
    void* cuda_stream;       /* stream for the work (NULL = legacy default stream)         */
    uint32_t has_target;     /* 1: single-target query (Sec. I): stop after the round that
                                fixes `target`; dist[target] is then exact, the other
                                outputs hold the state after that round                    */
    uint32_t target;         /* vertex id, < n (checked: SSSP_E_SOURCE_RANGE)              */
} sssp_solve_args;

typedef struct sssp_solve_info {
    uint32_t rounds;         /* rounds executed                                            */
    uint32_t finished;       /* 1 if the rounds ran to completion: no frontier left (and,
                                windowed, no active vertex); 0 if stopped by max_rounds or
                                a target                                                   */
    uint64_t reached;        /* vertices fixed (reachable, source included)                */
    uint64_t out_scanned;    /* out-edges scanned by step (a)                              */
    uint64_t in_scanned;     /* in-edges scanned by step (b)                               */
    uint64_t active_visits;  /* sum over rounds of the discovered-unfixed set size         */
    uint64_t front_visits;   /* sum over rounds of the frontier size                       */
    uint64_t kernel_launches;/* kernels the solve launched (start, rounds, output)          */
} sssp_solve_info;

/* General form of sssp_solve.  Synchronises the stream before returning.
 * info (nullable) receives the counters. */
int sssp_solve_ex(sssp_handle h, uint32_t source, const sssp_solve_args* args,
                  sssp_solve_info* info);

/* k independent queries solved together in lock-step rounds by the same
 * kernels: query i is (g[i], sources[i]); g[i] may repeat (many sources on
 * one graph) or differ (many graphs).  Each query's rounds depend only on its
 * own graph and source, so every result equals the one sssp_solve returns.
 * All handles must live on the same device and have the same rule and
 * window (SSSP_E_INVAL otherwise); their tunings may differ: the batch runs
 * with the tuning cached for its class (sssp_autotune_batch), else the first
 * handle's.  dist_out[i]: host u64[n_i]; rounds_out: host u32[k] (nullable).
 * Errors: as sssp_solve, plus SSSP_E_NOMEM for the batch workspace. */
int sssp_solve_batch(const sssp_handle* g, const uint32_t* sources, uint32_t k,
                     uint64_t* const* dist_out, uint32_t* rounds_out);

/* Device-pointer form of sssp_solve_batch: dist_dev[i] is a device u64[n_i].
 * Synchronises `cuda_stream` before returning. */
int sssp_solve_batch_device(const sssp_handle* g, const uint32_t* sources, uint32_t k,
                            uint64_t* const* dist_dev, uint32_t* rounds_out, void* cuda_stream);

/* Continuous-batching query server (the serving form of Sec. VI's round:
 * independent queries share its rounds).  Queries (graph handle, source)
 * are admitted into free slots while earlier queries are in flight, as long
 * as their state fits the device-memory budget; all admitted queries advance
 * together, a few rounds per device step, on one stream owned by the
 * server; between steps finished queries are written out and newly arrived
 * ones are admitted.  A query's result does not depend on which other
 * queries share its rounds.  By default a host thread owned by the server
 * runs the steps whenever a query is queued or in flight, so queries
 * complete without any call from the client. */
#define SSSP_SERVE_MANUAL 1u  /* no server thread: sssp_serve_poll, _wait and _drain
                                 run the steps (the caller drives the server)     */
#define SSSP_SERVE_WIDE   2u  /* 32-byte records: admits graphs whose
                                 n * max weight >= 2^31 (default: 16-byte records,
                                 which such graphs cannot use: SSSP_E_OVERFLOW)   */

typedef struct sssp_serve_cfg {
    uint64_t budget_bytes;   /* device bytes for query state (0 = 32 GiB)                  */
    uint32_t max_slots;      /* queries in flight at once (0 = 1024)                       */
    uint32_t rounds_per_step;/* rounds per device step between admissions (0 = 8)          */
    int32_t device;          /* -1 = current                                               */
    uint32_t flags;          /* SSSP_SERVE_* bits                                          */
    sssp_alloc_fn alloc;     /* NULL = cudaMalloc (one allocation per state array)         */
    sssp_free_fn free;
    void* alloc_ctx;
} sssp_serve_cfg;

/* Opens a server (and, unless SSSP_SERVE_MANUAL, starts its thread).  The
 * graphs passed to sssp_serve_submit must stay alive until their queries
 * complete; they must have the SSSP_RULE_THRESHOLD rule (any tuning).
 * Errors: SSSP_E_INVAL, SSSP_E_NOMEM, SSSP_E_CUDA. */
int sssp_serve_open(const sssp_serve_cfg* cfg, sssp_server** out);

/* Queues a query.  dist_out: host u64[n] written when the query completes
 * (owned by the caller, must stay valid until the query is reported done).
 * *ticket identifies the query.  Does not block on the device; callable from
 * any host thread.  Errors: SSSP_E_INVAL (also a graph with other options
 * than the server's), SSSP_E_SOURCE_RANGE, SSSP_E_OVERFLOW (a graph that
 * needs 32-byte records on a server without SSSP_SERVE_WIDE), SSSP_E_BUSY
 * (the query alone exceeds the budget), or the error that stopped the
 * server. */
int sssp_serve_submit(sssp_server* s, sssp_handle g, uint32_t source, uint64_t* dist_out,
                      uint64_t* ticket);

/* Reports on `ticket`: SSSP_OK when its dist_out is written (rounds_out set,
 * nullable; the ticket is then released), SSSP_PENDING while it is queued or
 * running, SSSP_E_NOT_FOUND for an unknown or already reported ticket, or
 * the error that stopped the server.  With SSSP_SERVE_MANUAL it first
 * advances the server by one step; otherwise it does not block. */
int sssp_serve_poll(sssp_server* s, uint64_t ticket, uint32_t* rounds_out);

/* Timing of one completed query.  Times are nanoseconds of the host's
 * monotonic clock (std::chrono::steady_clock, CLOCK_MONOTONIC on Linux). */
typedef struct sssp_query_info {
    uint32_t rounds;         /* rounds the query ran                                       */
    uint32_t reserved;
    uint64_t submit_ns;      /* sssp_serve_submit returned                                 */
    uint64_t admit_ns;       /* its state was set up on the device                         */
    uint64_t done_ns;        /* its distances were in dist_out                             */
    uint64_t first_step;     /* server step in which it was admitted (steps count from 1)  */
    uint64_t last_step;      /* server step in which it finished                           */
} sssp_query_info;

/* Waits up to timeout_ms for `ticket` to complete: then as sssp_serve_poll's
 * SSSP_OK, with info (nullable) filled in; SSSP_PENDING when the time ran
 * out.  With SSSP_SERVE_MANUAL the calling thread runs the steps meanwhile.
 * Other results as sssp_serve_poll. */
int sssp_serve_wait(sssp_server* s, uint64_t ticket, uint32_t timeout_ms, sssp_query_info* info);

/* Blocks until every submitted query is complete.  Errors: SSSP_E_BUSY when
 * a queued query can never be admitted, or the error that stopped the
 * server. */
int sssp_serve_drain(sssp_server* s);

typedef struct sssp_serve_stats {
    uint64_t steps;          /* device steps run                                           */
    uint64_t rounds;         /* engine rounds run (all queries in flight share a round)    */
    uint64_t submitted;      /* queries submitted                                          */
    uint64_t completed;      /* queries whose distances were written out                   */
    uint32_t queued;         /* waiting for a slot or pages now                            */
    uint32_t inflight;       /* on the device now                                          */
    uint32_t max_inflight;   /* most queries on the device together in one step            */
    uint32_t layout;         /* SSSP_LAYOUT_COMPACT or SSSP_LAYOUT_WIDE                    */
} sssp_serve_stats;

/* Counters of the server since it was opened.  Errors: SSSP_E_INVAL. */
int sssp_serve_stats_get(sssp_server* s, sssp_serve_stats* out);

/* Stops the server thread and closes the server; queries still queued or in
 * flight are abandoned (their dist_out is not written). */
void sssp_serve_close(sssp_server* s);

/* Per-kernel timing of the round kernels (tracing; the paper has no
 * counterpart).  While enabled on a handle, its single-query solves launch
 * the round kernels from the host and bracket every launch with CUDA events
 * on the solve stream.  With the default loop mode (SSSP_LOOP_GRAPH) the
 * host launches exactly the device loop's iterations -- k_relax, k_cupdate,
 * then the cluster tail kernel k_tail, which runs the following small rounds
 * -- so the times describe the schedule of an unprofiled solve; with
 * SSSP_LOOP_HOST every iteration is one round of k_relax and k_cupdate.
 * Launches after the last round are not counted.  The work counters of
 * sssp_solve_info are split by the kernel that did the work.  Results are
 * bit-identical to an unprofiled solve. */
typedef struct sssp_kernel_profile {
    uint64_t relax_launches;
    uint64_t cupdate_launches;
    double relax_ms;         /* summed event time of k_relax launches    */
    double cupdate_ms;       /* summed event time of k_cupdate launches  */
    uint64_t tail_launches;
    double tail_ms;          /* summed event time of k_tail launches     */
    uint64_t tail_rounds;    /* rounds finished inside k_tail            */
    uint64_t grid_counters[4];  /* out_scanned, in_scanned, active_visits, front_visits
                                   of the work done by k_relax and k_cupdate */
    uint64_t tail_counters[4];  /* the same for the work done by k_tail   */
} sssp_kernel_profile;

/* enable: 1 = on, 0 = off.  out (nullable) receives the totals gathered
 * since the last call, which are then reset.  Errors: SSSP_E_INVAL. */
int sssp_profile(sssp_handle h, int enable, sssp_kernel_profile* out);

/* Per-iteration event times of the most recent profiled solve (iterations
 * of the device loop, or rounds with SSSP_LOOP_HOST): iteration i's
 * k_relax / k_cupdate / k_tail milliseconds go to relax_ms[i] /
 * cupdate_ms[i] / tail_ms[i], the rounds k_tail finished to tail_rounds[i],
 * and (device-loop schedule only, else 0) the work counters of its k_relax
 * and k_cupdate -- out_scanned, in_scanned, active_visits, front_visits --
 * to grid_counters[4i .. 4i+3], for i < cap (tail_ms, tail_rounds and
 * grid_counters nullable); *count receives the number of iterations
 * recorded.  Errors: SSSP_E_INVAL. */
int sssp_profile_rounds(sssp_handle h, float* relax_ms, float* cupdate_ms, float* tail_ms,
                        uint32_t* tail_rounds, uint64_t* grid_counters, uint32_t cap,
                        uint32_t* count);

/* Single-source solve that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * when they solve -- code running inside another framework's memory pool
 * (which owns all device memory), services whose memory budget is fixed at
 * start-up, and latency-critical loops in which a cudaMalloc / cudaFree
 * would synchronise the device.  The caller passes the graph and the output
 * in its own device memory; all working state lives in one fixed scratch
 * array inside the library image (about SSSP_NOALLOC_MAX_VERTICES * 100
 * bytes), which every GPU that loads the library holds until the process
 * exits.  No cudaMalloc, cudaFree or other allocating routine is called.
 *   n          vertices, 1 <= n <= SSSP_NOALLOC_MAX_VERTICES; larger graphs
 *              get SSSP_E_NOALLOC_LIMIT
 *   out_off    device u64[n+1]: out-edges of u are entries out_off[u] ..
 *              out_off[u+1]-1 of out_adj
 *   out_adj    device u32[2m]: (target, weight) pairs
 *   in_off, in_adj: the same edges by target: (source, weight) pairs
 *   The graph must be loop-free with weights > 0 and ids < n (not checked:
 *   it is never copied to the host).
 *   max_weight the largest weight (for the SSSP_E_OVERFLOW check; an edge
 *              heavier than it is detected on the device during the solve
 *              and also gives SSSP_E_OVERFLOW)
 *   dist_dev   device u64[n] output, as sssp_solve
 *   rounds_out host u32 (nullable)
 *   cuda_stream the stream for the work (NULL = legacy default stream)
 * The call returns after the stream has finished the solve, also when it
 * fails after enqueuing work (no kernel of a failed call is left running on
 * the scratch).  The first call
 * on a device sets up that device (looks up the scratch's device address and
 * the kernels' launch limits); make that first call before any stream
 * capture.  Every call shares the scratch and leaves its contents behind
 * (each call clears what it needs), so calls that overlap on the GPU -- from
 * several host threads or streams -- race and must be serialised by the
 * caller. */
#define SSSP_NOALLOC_MAX_VERTICES 131072u
int sssp_solve_noalloc(uint32_t n, const uint64_t* out_off, const uint32_t* out_adj,
                       const uint64_t* in_off, const uint32_t* in_adj, uint32_t source,
                       uint32_t max_weight, uint64_t* dist_dev, uint32_t* rounds_out,
                       void* cuda_stream);

/* Releases a graph and its device memory.  NULL is ignored. */
void sssp_destroy(sssp_handle h);

/* Page-locked host memory, mapped into the device's address space, for
 * outputs written every solve: given as the dist_out of sssp_solve /
 * sssp_solve_ex, it is written directly by the output kernel (no device
 * staging, no copy); a pageable destination gets a copy from device scratch.
 * bytes > 0 (else SSSP_E_INVAL); *out receives the pointer, owned by the
 * caller until sssp_host_free.  SSSP_E_NOMEM when the allocation fails.
 * sssp_host_free(NULL) is ignored. */
int sssp_host_alloc(size_t bytes, void** out);
void sssp_host_free(void* p);

/* Static string naming an SSSP_* status code. */
const char* sssp_strerror(int code);

/* Number of vertices / edges (after self-loop removal) of a handle. */
uint32_t sssp_num_vertices(sssp_handle h);
uint64_t sssp_num_edges(sssp_handle h);

/* Single-target query (Sec. I: the distance from source to one vertex): the
 * rounds stop as soon as `target` is fixed, which is when its distance is
 * known.  *dist_target (host) receives cost[target] or SSSP_DIST_INF when
 * target is unreachable (then every round runs).  rounds_out (nullable):
 * rounds executed (0 when target = source).  Synchronous.  Errors: as
 * sssp_solve; SSSP_E_SOURCE_RANGE also for target >= n. */
int sssp_solve_to(sssp_handle h, uint32_t source, uint32_t target, uint64_t* dist_target,
                  uint32_t* rounds_out);

/* Self-test of the device-side wait limit (failure detection without a
 * fault): launches the persistent kernel's grid barrier over four CTAs of
 * which one never arrives; the other three must give up after timeout_ms
 * (1..10000), flag the timeout and exit, leaving the context usable.  Returns
 * SSSP_E_DEVICE_TIMEOUT when the limit worked (the expected result),
 * SSSP_E_INTERNAL if the wait ended otherwise, SSSP_E_CUDA on a CUDA error,
 * SSSP_E_INVAL for a timeout out of range.  Uses the current device. */
int sssp_selftest_barrier_timeout(uint32_t timeout_ms);

/* State layout the handle's single-query solves run with:
 * SSSP_LAYOUT_WIDE or SSSP_LAYOUT_COMPACT (0 for a NULL handle). */
uint32_t sssp_layout(sssp_handle h);

#ifdef __cplusplus
}
#endif
#endif /* SSSP_H */
