/*
 * oracle.h -- plain, single-threaded CPU oracle for Garg's bound-based
 * single-source shortest paths (arXiv 1812.10499).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant
 * with the CUDA path.
 *
 * Graphs are given as CSR out-adjacency: row_ptr[n+1] (u64 offsets),
 * col[m] (u32 targets), w[m] (u32 weights, strictly positive, Sec. I).
 * Inputs must be loop-free (Sec. II); orc_strip_self_loops() makes them so.
 * Distances are u64 with ORC_INF = UINT64_MAX for "unreachable / infinity".
 *
 * Parity status per function (what pins it is in tests/test_oracle_pins.py):
 *   orc_dijkstra        pinned: Bellman-Ford, Floyd-Warshall, scipy, worked example
 *   orc_bellman_ford    pinned: Floyd-Warshall, scipy, exhaustive tiny graphs
 *   orc_floyd_warshall  pinned: brute-force path enumeration on tiny graphs
 *   orc_round           pinned: distances vs the above; per-round invariants
 *                       C <= cost <= D (Lemmas 6-8); BFS closed form on unit
 *                       weights; hand-derived worked-example trace (3 rounds).
 *                       Round counts on general graphs: parity unpinned
 *                       beyond those invariants (the paper prints none).
 *   orc_round_delta     pinned: delta = 0 equals orc_round; an unbounded delta
 *                       equals ORC_LABEL_CORRECT round by round; hand-derived
 *                       window9 / window10 traces (the strict minD + delta
 *                       bound); per-round invariants for several deltas.
 *   orc_sp1 / orc_sp2   pinned: distances; heap-op claims of Theorems 2-3.
 *   orc_transpose       pinned: edge multiset equality.
 */
#ifndef SSSP_ORACLE_H
#define SSSP_ORACLE_H
#include <stdint.h>

#define ORC_INF UINT64_MAX

#define ORC_OK      0
#define ORC_EINVAL  (-1)
#define ORC_ENOMEM  (-2)

/* Round-R variants (mode bits of orc_round). */
#define ORC_RULE_THR      0u  /* clamp C by min(D, threshold)  (Lemmas 7-8)   */
#define ORC_RULE_MIND     1u  /* clamp C by minD, fix D <= threshold (Fig. SP_4 steps 2, 4) */
#define ORC_LABEL_CORRECT 2u  /* relax from every vertex whose D changed (SP_4 step 3) */
#define ORC_ALL_UNFIXED   8u  /* ablation: step 4 also raises C of undiscovered vertices (Fig. SP_4
                                 step 4 "for all unfixed"); they are never fixed (D = infinity) */
#define ORC_CHEAP_FIRST   4u  /* before scanning y's in-edges, fix y at once when
                                 D[y] <= minD + inWeight[y] (the in-version rule of SP_2,
                                 Sec. IV) or D[y] <= threshold (Lemma 8); both imply
                                 Cn[y] = D[y], so only in_scanned changes */

#define ORC_DELTA        16u  /* windowed relaxation (orc_round_delta only): see oracle.c */
#define ORC_PRED_COUNT   32u  /* SP_1's predecessor counts (Sec. III): count, per vertex, the
                                 in-edges whose source has not yet relaxed them; an active y
                                 whose count is 0 (every in-neighbour fixed and relaxed, so
                                 D[y] is final) is fixed without reading its in-edges.  Eq. (1)
                                 fixes such a y in the same round, so only in_scanned changes.
                                 Label-setting only (not with ORC_LABEL_CORRECT or ORC_DELTA) */
#define ORC_WITNESS      64u  /* (orc_round_ex only) a stored minimum witness per vertex: after a
                                 full in-edge scan of y, its argmin in-edge k* (least term, then
                                 least source, then least weight) and m2, the least term of its
                                 other in-edges.  Every Eq. (1) term only grows from round to
                                 round (C grows, D falls but stays >= the distance >= the last
                                 bound, the threshold and minD grow), so at y's next visit, if
                                 the term of k* is still <= m2, it is the exact minimum: the
                                 visit reads one in-edge instead of all of them.  Otherwise y
                                 is scanned in full and gets a new witness.  Applies to vertices
                                 with in-degree <= witness_deg; a visit counts 1 in-edge read for
                                 the check plus the in-degree if the check fails.  Only
                                 in_scanned changes.  Label-setting only, not with
                                 ORC_ALL_UNFIXED */

/* Per-round statistics written by orc_round (array of ORC_NSTATS u64). */
#define ORC_ST_OUT_SCANNED   0  /* out-edges scanned in relax steps          */
#define ORC_ST_IN_SCANNED    1  /* in-edges scanned in C-update steps        */
#define ORC_ST_ACTIVE_VISITS 2  /* sum over rounds of |active|               */
#define ORC_ST_FRONT_VISITS  3  /* sum over rounds of |frontier|             */
#define ORC_ST_REACHED       4  /* vertices fixed at the end (incl. source)  */
#define ORC_ST_MAX_ACTIVE    5  /* largest active set                        */
#define ORC_NSTATS           6

/* Called after every round with the state at the end of that round. */
typedef void (*orc_round_cb)(void* ctx, uint32_t round, uint64_t thr, uint64_t minD,
                             const uint64_t* D, const uint64_t* C,
                             const int32_t* fixed_round);

#ifdef __cplusplus
extern "C" {
#endif

/* Removes edges (u,u); returns the new edge count.  Arrays rewritten in place. */
uint64_t orc_strip_self_loops(uint32_t n, uint64_t* row_ptr, uint32_t* col, uint32_t* w);

/* CSR -> CSC (in-adjacency), stable by source id. */
int orc_transpose(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                  uint64_t* col_ptr, uint32_t* row, uint32_t* w_in);

/* Fig. 1: binary-heap Dijkstra.  ops[3] (nullable) = {inserts, adjusts, removeMins}. */
int orc_dijkstra(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                 uint32_t s, uint64_t* dist, uint64_t* ops);

/* Bellman-Ford by repeated full relaxation sweeps. */
int orc_bellman_ford(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                     uint32_t s, uint64_t* dist);

/* Floyd-Warshall on a dense n x n matrix (n <= 512); row s copied to dist. */
int orc_floyd_warshall(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                       uint32_t s, uint64_t* dist);

/* The data-parallel round of SP_3/SP_4 executed sequentially ("Round R").
 * Outputs (all nullable except dist): dist, parent (u32, UINT32_MAX if
 * unreachable), C (final lower bounds), fixed_round (-1 if never fixed),
 * rounds_out, stats[ORC_NSTATS].  cb (nullable) is called after each round.
 * target >= 0: single-target query (Sec. I: the method also answers the
 * distance to one vertex): stop after the round in which target is fixed
 * (no round when target = s). */
int orc_round(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
              uint32_t s, uint32_t mode, int64_t target,
              uint64_t* dist, uint32_t* parent, uint64_t* C_out, int32_t* fixed_round,
              uint32_t* rounds_out, uint64_t* stats, orc_round_cb cb, void* ctx);

/* orc_round with ORC_DELTA allowed in mode: delta is the width of the window
 * of distances above minD whose changed vertices relax before they are fixed
 * (ignored without ORC_DELTA; ORC_DELTA with ORC_LABEL_CORRECT is invalid). */
int orc_round_delta(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                    uint32_t s, uint32_t mode, int64_t target, uint64_t delta,
                    uint64_t* dist, uint32_t* parent, uint64_t* C_out, int32_t* fixed_round,
                    uint32_t* rounds_out, uint64_t* stats, orc_round_cb cb, void* ctx);

/* orc_round_delta with ORC_WITNESS allowed in mode, for vertices of
 * in-degree <= witness_deg. */
int orc_round_ex(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                 uint32_t s, uint32_t mode, int64_t target, uint64_t delta, uint32_t witness_deg,
                 uint64_t* dist, uint32_t* parent, uint64_t* C_out, int32_t* fixed_round,
                 uint32_t* rounds_out, uint64_t* stats, orc_round_cb cb, void* ctx);

/* Sec. III pre-processing: iteratively delete non-source vertices with no
 * in-edges.  removed[v] = 1 for deleted vertices. */
int orc_prune(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, uint32_t s,
              uint8_t* removed);

/* Fig. SP_1 (pred counts) and Fig. SP_2 (pred counts + inWeight).
 * prune != 0 applies orc_prune first (edges out of deleted vertices ignored).
 * ops[4] (nullable) = {heap inserts, heap adjusts, heap removeMins, outer iterations}. */
int orc_sp1(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
            uint32_t s, int prune, uint64_t* dist, uint64_t* ops);
int orc_sp2(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
            uint32_t s, int prune, uint64_t* dist, uint64_t* ops);

#ifdef __cplusplus
}
#endif
#endif
