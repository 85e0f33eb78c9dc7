/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for the bound-based
 * SSSP method of Garg (arXiv 1812.10499).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, by __graft_entry__.smoke() and by
 * the CPU-baseline leg of bench.py.  It shares no code with the CUDA path.
 *
 * Every function names the passage of the paper it restates.  The method
 * itself is a pure-integer computation (add, min, max, compare), so the
 * oracle is exact; there is no floating point anywhere.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- helpers */

/* Addition that saturates at infinity (an unreachable bound stays unreachable). */
static uint64_t sat_add(uint64_t a, uint64_t b) {
    if (a == ORC_INF || b == ORC_INF) return ORC_INF;
    uint64_t s = a + b;
    return (s < a) ? ORC_INF : s;
}
static uint64_t min_u64(uint64_t a, uint64_t b) { return a < b ? a : b; }
static uint64_t max_u64(uint64_t a, uint64_t b) { return a > b ? a : b; }

uint64_t orc_strip_self_loops(uint32_t n, uint64_t* row_ptr, uint32_t* col, uint32_t* w) {
    /* Sec. II assumes the graph is loop-free; a self-loop never lies on a
     * shortest path when weights are positive, so dropping it keeps cost[]. */
    uint64_t out = 0;
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t b = row_ptr[u], e = row_ptr[u + 1];
        row_ptr[u] = out;
        for (uint64_t k = b; k < e; ++k) {
            if (col[k] == u) continue;
            col[out] = col[k];
            w[out] = w[k];
            ++out;
        }
    }
    row_ptr[n] = out;
    return out;
}

int orc_transpose(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                  uint64_t* col_ptr, uint32_t* row, uint32_t* w_in) {
    /* In-edge lists, needed from SP_2 on (Sec. IV: "requires access to
     * incoming edges").  Counting sort by target; sources ascend in a list. */
    uint64_t m = row_ptr[n];
    uint64_t* cursor = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!cursor) return ORC_ENOMEM;
    for (uint64_t k = 0; k < m; ++k) cursor[col[k] + 1]++;
    col_ptr[0] = 0;
    for (uint32_t v = 0; v < n; ++v) col_ptr[v + 1] = col_ptr[v] + cursor[v + 1];
    for (uint32_t v = 0; v < n; ++v) cursor[v] = col_ptr[v];
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
            uint64_t at = cursor[col[k]]++;
            row[at] = u;
            w_in[at] = w[k];
        }
    free(cursor);
    return ORC_OK;
}

/* ------------------------------------------------------------ binary heap */
/* A textbook indexed binary min-heap of (vertex, key) with insertOrAdjust,
 * as used by Fig. 1 and the heap-based algorithms SP_1 / SP_2. */
typedef struct {
    uint32_t* v;     /* heap slots: vertex */
    uint64_t* key;   /* heap slots: key    */
    int64_t* pos;    /* pos[vertex] = slot or -1 */
    uint64_t size;
    uint64_t n_insert, n_adjust, n_remove;
} heap_t;

static int heap_init(heap_t* h, uint32_t n) {
    h->v = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    h->key = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    h->pos = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
    if (!h->v || !h->key || !h->pos) return ORC_ENOMEM;
    for (uint32_t i = 0; i < n; ++i) h->pos[i] = -1;
    h->size = 0;
    h->n_insert = h->n_adjust = h->n_remove = 0;
    return ORC_OK;
}
static void heap_free(heap_t* h) { free(h->v); free(h->key); free(h->pos); }

/* Heap order: smaller key first, ties broken by smaller vertex id. */
static int heap_less(const heap_t* h, uint64_t a, uint64_t b) {
    if (h->key[a] != h->key[b]) return h->key[a] < h->key[b];
    return h->v[a] < h->v[b];
}
static void heap_swap(heap_t* h, uint64_t a, uint64_t b) {
    uint32_t tv = h->v[a]; h->v[a] = h->v[b]; h->v[b] = tv;
    uint64_t tk = h->key[a]; h->key[a] = h->key[b]; h->key[b] = tk;
    h->pos[h->v[a]] = (int64_t)a;
    h->pos[h->v[b]] = (int64_t)b;
}
static void heap_up(heap_t* h, uint64_t i) {
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (!heap_less(h, i, p)) break;
        heap_swap(h, i, p);
        i = p;
    }
}
static void heap_down(heap_t* h, uint64_t i) {
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < h->size && heap_less(h, l, s)) s = l;
        if (r < h->size && heap_less(h, r, s)) s = r;
        if (s == i) break;
        heap_swap(h, i, s);
        i = s;
    }
}
static void heap_insert_or_adjust(heap_t* h, uint32_t v, uint64_t key) {
    if (h->pos[v] < 0) {
        uint64_t i = h->size++;
        h->v[i] = v;
        h->key[i] = key;
        h->pos[v] = (int64_t)i;
        h->n_insert++;
        heap_up(h, i);
    } else {
        uint64_t i = (uint64_t)h->pos[v];
        if (key < h->key[i]) {
            h->key[i] = key;
            h->n_adjust++;
            heap_up(h, i);
        }
    }
}
static void heap_remove_min(heap_t* h, uint32_t* v, uint64_t* key) {
    *v = h->v[0];
    *key = h->key[0];
    h->n_remove++;
    h->pos[*v] = -1;
    h->size--;
    if (h->size > 0) {
        h->v[0] = h->v[h->size];
        h->key[0] = h->key[h->size];
        h->pos[h->v[0]] = 0;
        heap_down(h, 0);
    }
}

/* --------------------------------------------------------------- Dijkstra */

int orc_dijkstra(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                 uint32_t s, uint64_t* dist, uint64_t* ops) {
    /* Fig. 1 with the loop body's "z" read as "j" (the vertex just removed). */
    if (s >= n) return ORC_EINVAL;
    heap_t H;
    uint8_t* fixed = (uint8_t*)calloc(n, 1);
    if (!fixed || heap_init(&H, n) != ORC_OK) { free(fixed); return ORC_ENOMEM; }
    for (uint32_t i = 0; i < n; ++i) dist[i] = ORC_INF;
    dist[s] = 0;
    heap_insert_or_adjust(&H, s, 0);
    while (H.size > 0) {
        uint32_t j; uint64_t d;
        heap_remove_min(&H, &j, &d);
        fixed[j] = 1;
        for (uint64_t k = row_ptr[j]; k < row_ptr[j + 1]; ++k) {
            uint32_t y = col[k];
            if (fixed[y]) continue;
            uint64_t nd = dist[j] + w[k];
            if (dist[y] > nd) {
                dist[y] = nd;
                heap_insert_or_adjust(&H, y, nd);
            }
        }
    }
    if (ops) { ops[0] = H.n_insert; ops[1] = H.n_adjust; ops[2] = H.n_remove; }
    heap_free(&H);
    free(fixed);
    return ORC_OK;
}

/* ----------------------------------------------------------- Bellman-Ford */

int orc_bellman_ford(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                     uint32_t s, uint64_t* dist) {
    /* Sweep every edge until nothing changes (at most n-1 useful sweeps). */
    if (s >= n) return ORC_EINVAL;
    for (uint32_t i = 0; i < n; ++i) dist[i] = ORC_INF;
    dist[s] = 0;
    for (uint32_t it = 0; it < n; ++it) {
        int changed = 0;
        for (uint32_t u = 0; u < n; ++u) {
            if (dist[u] == ORC_INF) continue;
            for (uint64_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
                uint64_t nd = dist[u] + w[k];
                if (nd < dist[col[k]]) { dist[col[k]] = nd; changed = 1; }
            }
        }
        if (!changed) break;
    }
    return ORC_OK;
}

/* ---------------------------------------------------------- Floyd-Warshall */

int orc_floyd_warshall(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                       uint32_t s, uint64_t* dist) {
    if (s >= n || n > 512) return ORC_EINVAL;
    uint64_t* M = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)n * n);
    if (!M) return ORC_ENOMEM;
    for (uint64_t i = 0; i < (uint64_t)n * n; ++i) M[i] = ORC_INF;
    for (uint32_t i = 0; i < n; ++i) M[(uint64_t)i * n + i] = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k)
            M[(uint64_t)u * n + col[k]] = min_u64(M[(uint64_t)u * n + col[k]], w[k]);
    for (uint32_t k = 0; k < n; ++k)
        for (uint32_t i = 0; i < n; ++i)
            for (uint32_t j = 0; j < n; ++j) {
                uint64_t via = sat_add(M[(uint64_t)i * n + k], M[(uint64_t)k * n + j]);
                if (via < M[(uint64_t)i * n + j]) M[(uint64_t)i * n + j] = via;
            }
    for (uint32_t j = 0; j < n; ++j) dist[j] = M[(uint64_t)s * n + j];
    free(M);
    return ORC_OK;
}

/* ----------------------------------------------------------------- Round R */

/* Eq. (1)'s minimum for vertex y over its in-edges (x, y) of lb(x) + w,
 * reading the C of the previous round:
 *   lb(x) = max(C[x], min(D[x], threshold))          (Lemmas 7 and 8)
 *   lb(x) = C[x] if x is fixed, else max(C[x], minD)  (minD rule, SP_4 step 4). */
/* One Eq. (1) term lb(x) + w of in-edge k = (x, y). */
static uint64_t eq1_term(uint64_t k, const uint32_t* row, const uint32_t* w_in, const uint64_t* C,
                         const uint64_t* D, const int32_t* fr, uint64_t thr, uint64_t minD,
                         int rule_mind) {
    uint32_t x = row[k];
    uint64_t lb;
    if (rule_mind)
        lb = (fr[x] >= 0) ? C[x] : max_u64(C[x], minD);
    else
        lb = max_u64(C[x], min_u64(D[x], thr));
    return sat_add(lb, w_in[k]);
}

static uint64_t eq1_min(uint32_t y, const uint64_t* col_ptr, const uint32_t* row,
                        const uint32_t* w_in, const uint64_t* C, const uint64_t* D,
                        const int32_t* fr, uint64_t thr, uint64_t minD, int rule_mind) {
    uint64_t best = ORC_INF;
    for (uint64_t k = col_ptr[y]; k < col_ptr[y + 1]; ++k)
        best = min_u64(best, eq1_term(k, row, w_in, C, D, fr, thr, minD, rule_mind));
    return best;
}

/* eq1_min that also records the witness (ORC_WITNESS): *kw = the in-edge
 * with the least (term, source, weight) -- a choice that does not depend on
 * the order of the in-edges -- and *m2 = the least term of the other
 * in-edges (equal to the minimum when two in-edges share it). */
static uint64_t eq1_min_witness(uint32_t y, const uint64_t* col_ptr, const uint32_t* row,
                                const uint32_t* w_in, const uint64_t* C, const uint64_t* D,
                                const int32_t* fr, uint64_t thr, uint64_t minD, int rule_mind,
                                uint64_t* kw, uint64_t* m2) {
    uint64_t best = ORC_INF, second = ORC_INF, kb = col_ptr[y];
    for (uint64_t k = col_ptr[y]; k < col_ptr[y + 1]; ++k) {
        const uint64_t t = eq1_term(k, row, w_in, C, D, fr, thr, minD, rule_mind);
        if (t < best) {
            second = min_u64(second, best);
            best = t;
            kb = k;
        } else {
            second = min_u64(second, t);
            if (t == best && k != kb &&
                (row[k] < row[kb] || (row[k] == row[kb] && w_in[k] < w_in[kb])))
                kb = k;
        }
    }
    *kw = kb;
    *m2 = second;
    return best;
}

int orc_round(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
              uint32_t s, uint32_t mode, int64_t target,
              uint64_t* dist, uint32_t* parent, uint64_t* C_out, int32_t* fixed_round,
              uint32_t* rounds_out, uint64_t* stats, orc_round_cb cb, void* ctx) {
    if (mode & ORC_DELTA) return ORC_EINVAL;   /* needs a window: orc_round_delta */
    return orc_round_delta(n, row_ptr, col, w, s, mode, target, 0, dist, parent, C_out,
                           fixed_round, rounds_out, stats, cb, ctx);
}

int orc_round_delta(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                    uint32_t s, uint32_t mode, int64_t target, uint64_t delta,
                    uint64_t* dist, uint32_t* parent, uint64_t* C_out, int32_t* fixed_round,
                    uint32_t* rounds_out, uint64_t* stats, orc_round_cb cb, void* ctx) {
    if (mode & ORC_WITNESS) return ORC_EINVAL;   /* needs a degree limit: orc_round_ex */
    return orc_round_ex(n, row_ptr, col, w, s, mode, target, delta, 0, dist, parent, C_out,
                        fixed_round, rounds_out, stats, cb, ctx);
}

int orc_round_ex(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                 uint32_t s, uint32_t mode, int64_t target, uint64_t delta, uint32_t witness_deg,
                 uint64_t* dist, uint32_t* parent, uint64_t* C_out, int32_t* fixed_round,
                 uint32_t* rounds_out, uint64_t* stats, orc_round_cb cb, void* ctx) {
    /*
     * One round of the parallel SP_3/SP_4 scheme, done one vertex at a time
     * on a snapshot (Sec. VI, SP_4 steps 1-5, label-setting as in SP_3):
     *   1. relax the out-edges of the frontier (vertices fixed in the
     *      previous round) into unfixed targets (SP_4 step 3); a target whose
     *      D was infinite becomes active (discovered and not fixed);
     *   2. threshold = min{D[u] + outWeight[u]} and minD = min{D[u]} over the
     *      active set (SP_4 step 1; Lemma 8 and Lemma 7), taken after the
     *      relaxation so that every fixed vertex has been explored;
     *   3. for every active y, from the PRE-round C and the post-relax D:
     *        lb(x) = max(C[x], min(D[x], threshold))    (Lemmas 7 and 8)
     *        Cn[y] = max(C[y], min(D[y], threshold),
     *                    min over in-edges (x,y) of lb(x) + w[x,y])   (Eq. 1)
     *      (ORC_RULE_MIND: clamp by minD instead, SP_4 step 4, and fix
     *      D <= threshold as in SP_4 step 2);
     *   4. C := Cn; fix y iff Cn[y] = D[y] (SP_4 step 5); the vertices fixed
     *      now form the next frontier, the others stay active.
     * The loop ends when a round fixes nothing new to explore.
     * D is kept as the pair (distance, parent) ordered lexicographically, so
     * equal distances keep the smaller parent id.
     *
     * ORC_LABEL_CORRECT: step 1 instead relaxes from every vertex whose D
     * changed in the previous round's step 1 (SP_4 step 3 relaxes all
     * discovered vertices; a vertex whose D is unchanged has nothing new to
     * relax), each with the D it had at the start of the step.
     *
     * ORC_DELTA (a reading of Sec. I's remark that Delta-stepping can be
     * combined with the lower bounds): a vertex is "pending" while its D has
     * changed since it last relaxed.  After step 4 the next frontier is every
     * pending vertex that is fixed, plus every pending active vertex with
     * D < minD + delta (minD of this round, saturating): the window plays the
     * part of Delta-stepping's current bucket.  Vertices outside the window
     * wait, so the loop runs while the frontier or the active set is
     * non-empty.  delta = 0 is the label-setting round exactly; a large
     * delta relaxes every changed vertex as ORC_LABEL_CORRECT does.
     */
    if (s >= n || target >= (int64_t)n) return ORC_EINVAL;
    const int rule_mind = (mode & ORC_RULE_MIND) != 0;
    const int label_correct = (mode & ORC_LABEL_CORRECT) != 0;
    const int cheap_first = (mode & ORC_CHEAP_FIRST) != 0;
    const int all_unfixed = (mode & ORC_ALL_UNFIXED) != 0;
    const int windowed = (mode & ORC_DELTA) != 0;
    const int pred_count = (mode & ORC_PRED_COUNT) != 0;
    const int witness = (mode & ORC_WITNESS) != 0;
    if (windowed && label_correct) return ORC_EINVAL;
    if (pred_count && (windowed || label_correct)) return ORC_EINVAL;
    if (witness && (windowed || label_correct || all_unfixed)) return ORC_EINVAL;
    uint64_t m = row_ptr[n];

    uint64_t* col_ptr = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint32_t* row = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* w_in = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint64_t* outW = (uint64_t*)malloc(sizeof(uint64_t) * n);
    uint64_t* inW = (uint64_t*)malloc(sizeof(uint64_t) * n);
    uint64_t* D = dist;
    uint32_t* par = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint64_t* C = (uint64_t*)malloc(sizeof(uint64_t) * n);
    int32_t* fr = (int32_t*)malloc(sizeof(int32_t) * n);
    uint32_t* front = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint32_t* front2 = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint64_t* front_d = (uint64_t*)malloc(sizeof(uint64_t) * n);
    uint32_t* act = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint32_t* act2 = (uint32_t*)malloc(sizeof(uint32_t) * n);
    uint64_t* Cn = (uint64_t*)malloc(sizeof(uint64_t) * n);
    uint64_t* Cu = (uint64_t*)malloc(sizeof(uint64_t) * n);   /* undiscovered (ablation) */
    uint8_t* changed = (uint8_t*)calloc(n, 1);
    uint64_t* pcnt = (uint64_t*)malloc(sizeof(uint64_t) * n);   /* SP_1 predecessor counts */
    uint64_t* wk = (uint64_t*)malloc(sizeof(uint64_t) * n);     /* witness in-edge */
    uint64_t* wm2 = (uint64_t*)malloc(sizeof(uint64_t) * n);    /* witness bound m2 */
    uint32_t* list_mem[4] = {front, front2, act, act2};   /* freed at the end */
    if (!col_ptr || !row || !w_in || !outW || !inW || !par || !C || !fr || !front || !front2 ||
        !front_d || !act || !act2 || !Cn || !Cu || !changed || !pcnt || !wk || !wm2) {
        free(col_ptr); free(row); free(w_in); free(outW); free(inW); free(par); free(C); free(fr);
        free(front); free(front2); free(front_d); free(act); free(act2); free(Cn); free(Cu);
        free(changed); free(pcnt); free(wk); free(wm2);
        return ORC_ENOMEM;
    }
    orc_transpose(n, row_ptr, col, w, col_ptr, row, w_in);
    /* Every in-edge of y still has to be relaxed by its source. */
    for (uint32_t y = 0; y < n; ++y) pcnt[y] = col_ptr[y + 1] - col_ptr[y];

    /* outWeight[x] = min out-edge weight (Fig. SP_3 / SP_4 declarations);
     * a vertex without out-edges contributes nothing to the threshold. */
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t mw = ORC_INF;
        for (uint64_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) mw = min_u64(mw, w[k]);
        outW[u] = mw;
    }
    /* inWeight[y] = min in-edge weight (SP_2, Sec. IV). */
    for (uint32_t y = 0; y < n; ++y) {
        uint64_t mw = ORC_INF;
        for (uint64_t k = col_ptr[y]; k < col_ptr[y + 1]; ++k) mw = min_u64(mw, w_in[k]);
        inW[y] = mw;
    }

    uint64_t st[ORC_NSTATS];
    memset(st, 0, sizeof(st));

    /* Initial state (Fig. SP_4 declarations; the source is fixed at once). */
    for (uint32_t i = 0; i < n; ++i) { D[i] = ORC_INF; par[i] = UINT32_MAX; C[i] = 0; fr[i] = -1; }
    D[s] = 0; par[s] = s; fr[s] = 0;
    uint64_t nf = 1, na = 0;
    front[0] = s;
    uint32_t r = 0;
    if (target == (int64_t)s) nf = 0;   /* the source is fixed before round 1 */

    while (nf > 0 || (windowed && na > 0)) {
        r++;
        st[ORC_ST_FRONT_VISITS] += nf;

        /* Step 1: relaxation.  Sources read their D from the snapshot. */
        for (uint64_t i = 0; i < nf; ++i) front_d[i] = D[front[i]];
        for (uint64_t i = 0; i < nf; ++i) changed[front[i]] = 0;
        uint64_t nchg = 0;
        for (uint64_t i = 0; i < nf; ++i) {
            uint32_t x = front[i];
            uint64_t dx = front_d[i];
            st[ORC_ST_OUT_SCANNED] += row_ptr[x + 1] - row_ptr[x];
            for (uint64_t k = row_ptr[x]; k < row_ptr[x + 1]; ++k) {
                uint32_t y = col[k];
                pcnt[y]--;                                /* (x, y) is relaxed now */
                if (fr[y] >= 0) continue;                 /* only unfixed targets */
                uint64_t nd = dx + w[k];
                if (nd < D[y] || (nd == D[y] && x < par[y])) {
                    if (D[y] == ORC_INF) act[na++] = y;    /* newly discovered */
                    D[y] = nd;
                    par[y] = x;
                    if (label_correct && !changed[y]) { changed[y] = 1; front2[nchg++] = y; }
                    if (windowed) changed[y] = 1;          /* pending */
                }
            }
        }

        /* Step 2: the two global minima over the discovered, unfixed set. */
        uint64_t minD = ORC_INF, thr = ORC_INF;
        for (uint64_t i = 0; i < na; ++i) {
            uint32_t y = act[i];
            minD = min_u64(minD, D[y]);
            thr = min_u64(thr, sat_add(D[y], outW[y]));
        }
        st[ORC_ST_ACTIVE_VISITS] += na;
        if (na > st[ORC_ST_MAX_ACTIVE]) st[ORC_ST_MAX_ACTIVE] = na;

        /* Step 3: Jacobi lower bounds (reads pre-round C only). */
        for (uint64_t i = 0; i < na; ++i) {
            uint32_t y = act[i];
            uint64_t self = rule_mind ? minD : min_u64(D[y], thr);
            uint64_t best = ORC_INF;
            if ((cheap_first && (D[y] <= sat_add(minD, inW[y]) || D[y] <= thr)) ||
                (pred_count && pcnt[y] == 0)) {
                Cn[i] = D[y];            /* fixed without reading the in-edges */
                continue;
            }
            const int witnessed = witness && col_ptr[y + 1] - col_ptr[y] <= witness_deg;
            if (witnessed && C[y] != 0) {
                /* Visited before (every visit leaves C >= 1), so the witness
                 * is set: if its term is still <= m2 it is the minimum. */
                st[ORC_ST_IN_SCANNED] += 1;
                const uint64_t t = eq1_term(wk[y], row, w_in, C, D, fr, thr, minD, rule_mind);
                if (t <= wm2[y]) {
                    Cn[i] = max_u64(C[y], max_u64(self, t));
                    continue;
                }
            }
            st[ORC_ST_IN_SCANNED] += col_ptr[y + 1] - col_ptr[y];
            if (witnessed)
                best = eq1_min_witness(y, col_ptr, row, w_in, C, D, fr, thr, minD, rule_mind,
                                       &wk[y], &wm2[y]);
            else
                best = eq1_min(y, col_ptr, row, w_in, C, D, fr, thr, minD, rule_mind);
            Cn[i] = max_u64(C[y], max_u64(self, best));
        }
        /* Ablation: the same bound for every undiscovered vertex (D = infinity,
         * so its own clamp is the threshold, or minD with the minD rule). */
        if (all_unfixed) {
            for (uint32_t y = 0; y < n; ++y) {
                if (fr[y] >= 0 || D[y] != ORC_INF) continue;
                st[ORC_ST_IN_SCANNED] += col_ptr[y + 1] - col_ptr[y];
                const uint64_t best = eq1_min(y, col_ptr, row, w_in, C, D, fr, thr, minD, rule_mind);
                Cu[y] = max_u64(C[y], max_u64(rule_mind ? minD : thr, best));
            }
        }

        /* Step 4: apply C, fix C = D, split into next frontier / active. */
        uint64_t nf2 = 0, na2 = 0;
        const uint64_t window = sat_add(minD, delta);
        for (uint64_t i = 0; i < na; ++i) {
            uint32_t y = act[i];
            C[y] = Cn[i];
            int fix = (Cn[i] == D[y]) || (rule_mind && D[y] <= thr);
            if (fix) {
                C[y] = D[y];
                fr[y] = (int32_t)r;
                if (windowed ? changed[y] : !label_correct) front2[nf2++] = y;
            } else {
                act2[na2++] = y;
                if (windowed && changed[y] && D[y] < window) front2[nf2++] = y;
            }
        }
        if (all_unfixed)
            for (uint32_t y = 0; y < n; ++y)
                if (fr[y] < 0 && D[y] == ORC_INF) C[y] = Cu[y];
        if (label_correct) nf2 = nchg;
        { uint32_t* t = front; front = front2; front2 = t; }
        { uint32_t* t = act; act = act2; act2 = t; }
        nf = nf2;
        na = na2;
        if (cb) cb(ctx, r, thr, minD, D, C, fr);
        if (target >= 0 && fr[target] >= 0) break;   /* single-target query answered */
    }

    uint64_t reached = 0;
    for (uint32_t i = 0; i < n; ++i) reached += (fr[i] >= 0);
    st[ORC_ST_REACHED] = reached;

    if (parent) memcpy(parent, par, sizeof(uint32_t) * n);
    if (C_out) memcpy(C_out, C, sizeof(uint64_t) * n);
    if (fixed_round) memcpy(fixed_round, fr, sizeof(int32_t) * n);
    if (rounds_out) *rounds_out = r;
    if (stats) memcpy(stats, st, sizeof(st));

    free(col_ptr); free(row); free(w_in); free(outW); free(inW); free(par); free(C); free(fr);
    free(list_mem[0]); free(list_mem[1]); free(front_d); free(list_mem[2]); free(list_mem[3]);
    free(Cn); free(Cu); free(changed); free(pcnt); free(wk); free(wm2);
    return ORC_OK;
}

/* ------------------------------------------------------------ SP_1 / SP_2 */

int orc_prune(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, uint32_t s,
              uint8_t* removed) {
    /* Sec. III: list L of non-source vertices without in-edges; delete them
     * and their out-edges; repeat while deletions create new such vertices. */
    if (s >= n) return ORC_EINVAL;
    uint64_t* indeg = (uint64_t*)calloc(n, sizeof(uint64_t));
    uint32_t* L = (uint32_t*)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!indeg || !L) { free(indeg); free(L); return ORC_ENOMEM; }
    for (uint64_t k = 0; k < row_ptr[n]; ++k) indeg[col[k]]++;
    uint64_t top = 0;
    for (uint32_t v = 0; v < n; ++v) {
        removed[v] = 0;
        if (v != s && indeg[v] == 0) { L[top++] = v; removed[v] = 1; }
    }
    while (top > 0) {
        uint32_t u = L[--top];
        for (uint64_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) {
            uint32_t y = col[k];
            if (--indeg[y] == 0 && y != s && !removed[y]) { removed[y] = 1; L[top++] = y; }
        }
    }
    free(indeg);
    free(L);
    return ORC_OK;
}

/* Shared body of Fig. SP_1 and Fig. SP_2; use_inweight selects processEdge2. */
static int sp12(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
                uint32_t s, int prune, int use_inweight, uint64_t* dist, uint64_t* ops) {
    if (s >= n) return ORC_EINVAL;
    uint64_t m = row_ptr[n];
    uint8_t* removed = (uint8_t*)calloc(n, 1);
    uint8_t* fixed = (uint8_t*)calloc(n, 1);
    uint8_t* inQ = (uint8_t*)calloc(n, 1);
    uint64_t* pred = (uint64_t*)calloc(n, sizeof(uint64_t));
    uint64_t* inWeight = (uint64_t*)malloc(sizeof(uint64_t) * n);
    uint32_t* R = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint32_t* Q = (uint32_t*)malloc(sizeof(uint32_t) * ((size_t)n + 1));
    uint64_t* col_ptr = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n + 1));
    uint32_t* row = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint32_t* w_in = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    heap_t H;
    memset(&H, 0, sizeof(H));
    int rc = ORC_OK;
    if (!removed || !fixed || !inQ || !pred || !inWeight || !R || !Q || !col_ptr || !row ||
        !w_in || heap_init(&H, n) != ORC_OK) {
        rc = ORC_ENOMEM;
        goto done;
    }
    orc_transpose(n, row_ptr, col, w, col_ptr, row, w_in);
    if (prune) orc_prune(n, row_ptr, col, s, removed);

    /* pred[i] = number of in-edges (from vertices that were not deleted). */
    for (uint32_t u = 0; u < n; ++u) {
        if (removed[u]) continue;
        for (uint64_t k = row_ptr[u]; k < row_ptr[u + 1]; ++k) pred[col[k]]++;
    }
    for (uint32_t i = 0; i < n; ++i) { dist[i] = ORC_INF; inWeight[i] = ORC_INF; }

    uint64_t outer = 0, r_head = 0, r_tail = 0, q_len = 0;
    dist[s] = 0;
    heap_insert_or_adjust(&H, s, 0);
    while (H.size > 0) {
        /* H.empty() counts non-fixed entries only (Sec. III); fixed entries
         * are popped and skipped. */
        uint32_t j; uint64_t d;
        heap_remove_min(&H, &j, &d);
        if (fixed[j]) continue;
        outer++;
        fixed[j] = 1;
        r_head = r_tail = 0;
        R[r_tail++] = j;
        while (r_head < r_tail) {
            uint32_t z = R[r_head++];
            for (uint64_t k = row_ptr[z]; k < row_ptr[z + 1]; ++k) {
                uint32_t y = col[k];
                if (fixed[y]) continue;
                /* processEdge1 / processEdge2 */
                int chg = 0;
                pred[y]--;
                if (use_inweight && dist[y] == ORC_INF && pred[y] > 0) {
                    /* Step 1: minimum in-weight over predecessors other than z. */
                    uint64_t mw = ORC_INF;
                    for (uint64_t q = col_ptr[y]; q < col_ptr[y + 1]; ++q)
                        if (row[q] != z && !removed[row[q]]) mw = min_u64(mw, w_in[q]);
                    inWeight[y] = mw;
                }
                uint64_t nd = dist[z] + w[k];
                if (dist[y] > nd) { dist[y] = nd; chg = 1; }
                int fix = (pred[y] == 0);
                if (use_inweight && !fix && dist[y] <= sat_add(d, inWeight[y])) fix = 1;
                if (fix) {
                    fixed[y] = 1;
                    R[r_tail++] = y;
                } else if (chg && !inQ[y]) {
                    inQ[y] = 1;
                    Q[q_len++] = y;
                }
            }
        }
        for (uint64_t i = 0; i < q_len; ++i) {
            uint32_t z = Q[i];
            inQ[z] = 0;
            if (!fixed[z]) heap_insert_or_adjust(&H, z, dist[z]);
        }
        q_len = 0;
    }
    if (ops) { ops[0] = H.n_insert; ops[1] = H.n_adjust; ops[2] = H.n_remove; ops[3] = outer; }
done:
    heap_free(&H);
    free(removed); free(fixed); free(inQ); free(pred); free(inWeight); free(R); free(Q);
    free(col_ptr); free(row); free(w_in);
    return rc;
}

int orc_sp1(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
            uint32_t s, int prune, uint64_t* dist, uint64_t* ops) {
    return sp12(n, row_ptr, col, w, s, prune, 0, dist, ops);
}

int orc_sp2(uint32_t n, const uint64_t* row_ptr, const uint32_t* col, const uint32_t* w,
            uint32_t s, int prune, uint64_t* dist, uint64_t* ops) {
    return sp12(n, row_ptr, col, w, s, prune, 1, dist, ops);
}
