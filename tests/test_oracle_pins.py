"""Pins of the CPU oracle against things other than itself.

Each check ties the oracle to a fact fixed by the paper or by mathematics:
the worked example printed in Sec. III / Sec. IV, textbook shortest-path
algorithms (Bellman-Ford, Floyd-Warshall, brute-force path enumeration,
scipy's Dijkstra), closed forms (BFS depth on unit weights, Manhattan
distance on a unit grid) and the invariants of Lemmas 6-8 (C <= cost <= D
after every round).  test_oracle_mutants.py shows that plausible mistakes in
oracle.c fail at least one of these checks.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.golden.fixtures import worked_example

INF = int(oracle.INF)


# ----------------------------------------------------------------- helpers

def edges_of(g):
    src, col, w = g.edges()
    return list(zip(src.tolist(), col.tolist(), w.tolist()))


def brute_force_dist(g, s):
    """Minimum over all simple paths by explicit enumeration (tiny graphs)."""
    adj = {u: [] for u in range(g.n)}
    for u, v, w in edges_of(g):
        if u != v:
            adj[u].append((v, w))
    best = [INF] * g.n
    best[s] = 0

    def dfs(u, cost, seen):
        for v, w in adj[u]:
            if v in seen:
                continue
            c = cost + w
            if c < best[v]:
                best[v] = c
            dfs(v, c, seen | {v})

    dfs(s, 0, {s})
    return np.array(best, dtype=np.uint64)


def bfs_depth(g, s):
    depth = np.full(g.n, -1, dtype=np.int64)
    depth[s] = 0
    frontier = [s]
    while frontier:
        nxt = []
        for u in frontier:
            for k in range(int(g.row_ptr[u]), int(g.row_ptr[u + 1])):
                v = int(g.col[k])
                if depth[v] < 0:
                    depth[v] = depth[u] + 1
                    nxt.append(v)
        frontier = nxt
    return depth


def random_small(n, deg, wmax, seed):
    return gg.random_graph(n, deg, 1, wmax, seed)


SMALL_CASES = [(n, d, wmax, seed) for n, d, wmax in
               [(2, 1, 3), (5, 2, 3), (8, 3, 5), (17, 2, 10), (33, 4, 100), (64, 6, 1000)]
               for seed in range(3)]


# ------------------------------------------------------- worked example pins

@pytest.mark.parametrize("variant", ["A", "B"])
def test_worked_example(variant):
    ex = worked_example()[variant]
    g = gg.from_edges(ex["n"], ex["edges"])
    s = ex["source"]
    assert oracle.dijkstra(g, s)[0].tolist() == ex["dist"]
    d1, ops1 = oracle.sp1(g, s)
    d2, ops2 = oracle.sp2(g, s)
    assert d1.tolist() == ex["dist"] and d2.tolist() == ex["dist"]
    assert ops1["inserts"] == ex["sp1_inserts"] and ops1["outer"] == ex["sp1_outer"]
    assert ops2["inserts"] == ex["sp2_inserts"] and ops2["outer"] == ex["sp2_outer"]
    r = oracle.round_r(g, s)
    assert r.dist.tolist() == ex["dist"]
    assert r.fixed_round.tolist() == ex["fixed_round"]
    assert r.parent.tolist() == ex["parent"]
    assert r.rounds == ex["rounds"]


@pytest.mark.parametrize("variant", ["threshold", "jacobi", "inclamp"])
def test_hand_derived_round_traces(variant):
    """Round traces derived by hand from Lemma 8 and the Jacobi reading of
    SP_4 step 4 (see the comments in tests/golden/worked_example.txt)."""
    ex = worked_example()[variant]
    g = gg.from_edges(ex["n"], ex["edges"])
    r = oracle.round_r(g, ex["source"])
    assert r.dist.tolist() == ex["dist"]
    assert r.fixed_round.tolist() == ex["fixed_round"]
    assert r.parent.tolist() == ex["parent"]
    assert r.rounds == ex["rounds"]


# ---------------------------------------- distances vs textbook algorithms

def test_exhaustive_three_vertex_digraphs():
    """Every digraph on 3 vertices with weights in {1,2,3} (4^6 graphs), every
    source: Dijkstra = Bellman-Ford = Floyd-Warshall = enumeration = Round R."""
    pairs = [(u, v) for u in range(3) for v in range(3) if u != v]
    lib = oracle.load()
    for choice in itertools.product(range(4), repeat=len(pairs)):
        edges = [(u, v, c) for (u, v), c in zip(pairs, choice) if c]
        g = gg.from_edges(3, edges)
        for s in range(3):
            ref = brute_force_dist(g, s)
            assert np.array_equal(oracle.dijkstra(g, s, lib=lib)[0], ref)
            assert np.array_equal(oracle.bellman_ford(g, s, lib=lib), ref)
            assert np.array_equal(oracle.floyd_warshall(g, s, lib=lib), ref)
            assert np.array_equal(oracle.round_r(g, s, lib=lib).dist, ref)


@pytest.mark.parametrize("case", SMALL_CASES)
def test_distances_agree(case):
    n, d, wmax, seed = case
    g = random_small(n, d, wmax, seed)
    scipy_sp = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sp
    for s in range(min(n, 4)):
        dj, _ = oracle.dijkstra(g, s)
        assert np.array_equal(dj, oracle.bellman_ford(g, s))
        assert np.array_equal(dj, oracle.floyd_warshall(g, s))
        if n <= 8:
            assert np.array_equal(dj, brute_force_dist(g, s))
        # scipy's Dijkstra keeps the minimum of parallel edges when summing
        # duplicates is avoided; build the matrix from the min weight per pair.
        src, col, w = g.edges()
        M = {}
        for u, v, ww in zip(src.tolist(), col.tolist(), w.tolist()):
            M[(u, v)] = min(M.get((u, v), ww), ww)
        mat = sp.csr_matrix((np.array(list(M.values()), dtype=np.float64),
                             ([k[0] for k in M], [k[1] for k in M])), shape=(n, n))
        ref = scipy_sp.dijkstra(mat, directed=True, indices=s)
        fin = ~np.isinf(ref)
        assert np.array_equal(dj == INF, ~fin)
        assert np.array_equal(dj[fin], ref[fin].astype(np.uint64))
        for mode in (oracle.RULE_THR, oracle.RULE_MIND, oracle.LABEL_CORRECT,
                     oracle.LABEL_CORRECT | oracle.RULE_MIND):
            assert np.array_equal(oracle.round_r(g, s, mode=mode).dist, dj)
        assert np.array_equal(oracle.sp1(g, s)[0], dj)
        assert np.array_equal(oracle.sp2(g, s)[0], dj)


def test_transpose_is_the_same_edge_multiset():
    g = gg.random_var_graph(300, 1, 9, 1, 50, 7)
    col_ptr, row, w_in = oracle.transpose(g)
    fwd = sorted(edges_of(g))
    bwd = sorted((int(row[k]), v, int(w_in[k]))
                 for v in range(g.n) for k in range(int(col_ptr[v]), int(col_ptr[v + 1])))
    assert fwd == bwd


# ---------------------------------------------------- Round R invariants

def check_round_invariants(g, s, mode=oracle.RULE_THR, lib=None, delta=None):
    cost, _ = oracle.dijkstra(g, s, lib=lib)
    seen = []

    def on_round(r, thr, minD, D, C, F):
        fixed = F >= 0
        # Lemmas 6-8: every C is a lower bound, every D an upper bound.
        assert np.all(C <= cost), f"round {r}: C > cost"
        assert np.all(D >= cost), f"round {r}: D < cost"
        # Fixed vertices carry their final cost (Lemma 1(a) analogue).
        assert np.all(D[fixed] == cost[fixed]) and np.all(C[fixed] == cost[fixed])
        # Fixing is C = D (SP_4 step 5).
        unf = ~fixed & (D != INF)
        assert np.all(C[unf] < D[unf])
        seen.append(int(np.count_nonzero(F == r)))

    r = oracle.round_r(g, s, mode=mode, on_round=on_round, lib=lib, delta=delta)
    reach = cost != INF
    assert np.array_equal(r.dist, cost)
    assert np.array_equal(r.fixed_round >= 0, reach)
    # every round but the last fixes at least one vertex (windowed: the last
    # round may fix vertices that have nothing left to relax)
    assert all(c >= 1 for c in seen[:-1]) and (delta is not None or seen[-1] == 0)
    assert r.rounds == len(seen) <= max(1, int(reach.sum()))
    assert r.stats["reached"] == int(reach.sum())
    # parent edges are tight and come from vertices fixed earlier
    for v in np.flatnonzero(reach):
        p = int(r.parent[v])
        if v == s:
            assert p == s
            continue
        ws = [int(g.w[k]) for k in range(int(g.row_ptr[p]), int(g.row_ptr[p + 1]))
              if int(g.col[k]) == v]
        assert ws and int(cost[p]) + min(ws) == int(cost[v])
        # (windowed: p may relax before it is fixed, and it is then fixed in
        # v's round at the latest -- v's bound needs lb(p) = D[p])
        if delta is None:
            assert r.fixed_round[p] < r.fixed_round[v]
        else:
            assert r.fixed_round[p] <= r.fixed_round[v]
    return r


@pytest.mark.parametrize("case", SMALL_CASES)
@pytest.mark.parametrize("mode", [oracle.RULE_THR, oracle.RULE_MIND])
def test_round_invariants(case, mode):
    n, d, wmax, seed = case
    g = random_small(n, d, wmax, seed)
    for s in range(min(n, 3)):
        check_round_invariants(g, s, mode)


def test_round_invariants_skewed():
    g = gg.rmat(10, 8, 1, 255, 3)
    s = int(np.argmax(g.out_degree()))
    check_round_invariants(g, s)


def test_threshold_rule_fixes_at_least_as_fast_as_mind_rule():
    """min(D, threshold) >= minD, so the THR clamp never fixes later."""
    for seed in range(5):
        g = random_small(200, 4, 100, seed)
        a = oracle.round_r(g, 0, mode=oracle.RULE_THR)
        b = oracle.round_r(g, 0, mode=oracle.RULE_MIND)
        ok = (a.fixed_round >= 0)
        assert np.all(a.fixed_round[ok] <= b.fixed_round[ok])


# ------------------------------------------------------------- closed forms

@pytest.mark.parametrize("seed", range(4))
def test_unit_weights_is_bfs(seed):
    """Unit weights: the vertex at BFS depth k is fixed in round k and the
    number of rounds is the eccentricity plus one (the last round relaxes the
    deepest layer and finds nothing)."""
    g = gg.random_graph(500, 3, 1, 1, seed)
    for s in (0, 7):
        depth = bfs_depth(g, s)
        r = oracle.round_r(g, s)
        reach = depth >= 0
        assert np.array_equal(r.dist[reach], depth[reach].astype(np.uint64))
        assert np.array_equal(r.fixed_round[reach], depth[reach])
        assert r.rounds == int(depth.max()) + 1


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 9), (7, 5), (16, 16), (33, 20)])
def test_unit_grid_closed_form(rows, cols):
    g = gg.grid(rows, cols, 1, 1, 0)
    r = oracle.round_r(g, 0)
    i, j = np.divmod(np.arange(rows * cols), cols)
    assert np.array_equal(r.dist, (i + j).astype(np.uint64))
    assert r.rounds == (rows - 1) + (cols - 1) + 1


def test_weighted_grid_distances():
    g = gg.grid(20, 30, 1, 10000, 5)
    dj, _ = oracle.dijkstra(g, 0)
    assert np.array_equal(oracle.bellman_ford(g, 0), dj)
    check_round_invariants(g, 0)


# -------------------------------------------------- SP_1 / SP_2 heap claims

@pytest.mark.parametrize("seed", range(4))
def test_sp1_dag_needs_no_heap_operation(seed):
    """Theorem 2: on a DAG in which only the source lacks in-edges (after the
    Sec. III pruning), SP_1 inserts only the source and never adjusts."""
    g = gg.dag(30, 40, 4, 4, 1, 1000, seed)
    dist, ops = oracle.sp1(g, 0, prune_first=True)
    assert np.array_equal(dist, oracle.dijkstra(g, 0)[0])
    assert ops["inserts"] + ops["adjusts"] == 1
    d2, ops2 = oracle.sp2(g, 0, prune_first=True)
    assert np.array_equal(d2, dist) and ops2["inserts"] + ops2["adjusts"] == 1


def test_prune_removes_exactly_the_vertices_without_paths_from_in_degree_zero():
    g = gg.from_edges(6, [(0, 1, 1), (2, 3, 1), (3, 4, 1), (4, 1, 1), (5, 5, 1)])
    removed = oracle.prune(g, 0)
    # 2 has no in-edge -> removed, then 3, then 4; 5 only has a self-loop
    # (stripped, Sec. II) -> removed; 1 keeps the edge from 0.
    assert removed.tolist() == [0, 0, 1, 1, 1, 1]


@pytest.mark.parametrize("seed", range(6))
def test_sp1_sp2_use_no_more_heap_operations_than_dijkstra(seed):
    """Sec. I / Sec. III: SP_1 and SP_2 never perform more heap inserts and
    adjusts than Dijkstra's algorithm."""
    g = gg.random_graph(300, 3, 1, 20, seed)
    _, dj = oracle.dijkstra(g, 0)
    _, o1 = oracle.sp1(g, 0)
    _, o2 = oracle.sp2(g, 0)
    base = dj["inserts"] + dj["adjusts"]
    assert o1["inserts"] + o1["adjusts"] <= base
    assert o2["inserts"] + o2["adjusts"] <= base


def test_sp2_unweighted_counterexample():
    """Theorem 3 claims SP_2 is O(e) (no heap use) on unweighted graphs.  With
    d read as the key of the last removeMin, unit weights s->a->b->x->b force
    a heap insert: when b is discovered, D[b] = 2 > d + inWeight[b] = 0 + 1."""
    g = gg.from_edges(4, [(0, 1, 1), (1, 2, 1), (2, 3, 1), (3, 2, 1)])
    dist, ops = oracle.sp2(g, 0)
    assert dist.tolist() == [0, 1, 2, 3]
    assert ops["inserts"] >= 2


def test_reduction_after_relaxation_reading():
    """SP_4 as printed computes threshold before relaxing; if the vertices
    fixed in the previous step are not yet explored this fixes b with
    D[b] = 5 > cost 2.  The oracle takes the minima after the relaxation."""
    g = gg.from_edges(5, [(0, 1, 1), (0, 2, 5), (1, 2, 1), (2, 3, 1), (3, 4, 100)])
    for mode in (oracle.RULE_THR, oracle.RULE_MIND, oracle.LABEL_CORRECT):
        assert oracle.round_r(g, 0, mode=mode).dist.tolist() == [0, 1, 2, 3, 103]


def test_termination_reading():
    """SP_4's printed loop test (some discovered vertex unfixed) would stop
    after s->a if a is fixed at once; the oracle runs while a frontier is
    left, so b is still reached."""
    g = gg.from_edges(3, [(0, 1, 1), (1, 2, 1)])
    r = oracle.round_r(g, 0)
    assert r.dist.tolist() == [0, 1, 2] and r.rounds == 3


def test_unreachable_and_isolated():
    g = gg.from_edges(4, [(1, 2, 3), (2, 1, 3)])
    r = oracle.round_r(g, 0)
    assert r.dist.tolist() == [0, INF, INF, INF]
    assert r.fixed_round.tolist() == [0, -1, -1, -1]
    assert r.rounds == 1


def test_multi_edges_and_self_loops():
    g = gg.from_edges(3, [(0, 1, 5), (0, 1, 2), (1, 1, 1), (1, 2, 4), (1, 2, 9)])
    assert oracle.round_r(g, 0).dist.tolist() == [0, 2, 6]
    with pytest.raises(ValueError):
        oracle.round_r(gg.from_edges(2, [(0, 1, 0)]), 0)


# ------------------------------------------------ single-target query (Sec. I)

def test_single_target_query_is_the_full_run_cut_at_the_targets_round():
    """Stopping when the target is fixed gives exactly the state of the full
    run after round fixed_round[target], and the target's distance is the
    textbook one (Dijkstra); a target equal to the source needs no round; an
    unreachable target runs to completion."""
    g = gg.random_var_graph(1500, 1, 7, 1, 90, 77)
    snaps = []
    full = oracle.round_r(g, 0, on_round=lambda r, thr, mD, D, C, F: snaps.append(
        (D.copy(), C.copy(), F.copy())))
    dj, _ = oracle.dijkstra(g, 0)
    reach = np.flatnonzero(full.fixed_round >= 0)
    assert len(reach) > 100
    for t in [int(x) for x in reach[:: max(1, len(reach) // 25)]] + [int(reach[-1])]:
        res = oracle.round_r(g, 0, target=t)
        k = int(full.fixed_round[t])
        assert res.rounds == k
        assert res.dist[t] == dj[t]
        if k > 0:
            D, C, F = snaps[k - 1]
            assert np.array_equal(res.dist, D)
            assert np.array_equal(res.C, C)
            assert np.array_equal(res.fixed_round, F)
    src = oracle.round_r(g, 0, target=0)
    assert src.rounds == 0 and src.dist[0] == 0
    assert np.count_nonzero(src.dist != INF) == 1
    unreach = np.flatnonzero(full.fixed_round < 0)
    if len(unreach):
        res = oracle.round_r(g, 0, target=int(unreach[0]))
        assert res.rounds == full.rounds and np.array_equal(res.dist, full.dist)


# ------------------------------------- cheaper fixing rules first (SP_2 / Lemma 8)

@pytest.mark.parametrize("base", [oracle.RULE_THR, oracle.RULE_MIND, oracle.LABEL_CORRECT])
def test_cheap_rules_first_change_only_the_scan_count(base):
    """The in-version rule D[y] <= minD + inWeight[y] and D[y] <= threshold
    imply Eq. (1)'s bound reaches D[y]; fixing such y without reading its
    in-edges leaves every state and round count unchanged and scans fewer
    in-edges.  A vertex the cheap rules fix is one the full rule fixes in
    the same round."""
    for g, s in ((gg.rmat(12, 8, 1, 255, 4), 0), (gg.random_var_graph(3000, 1, 9, 1, 60, 8), 2),
                 (gg.grid(40, 30, 1, 50, 1), 0)):
        if g.out_degree()[s] == 0:
            s = int(np.argmax(g.out_degree()))
        a = oracle.round_r(g, s, mode=base)
        b = oracle.round_r(g, s, mode=base | oracle.CHEAP_FIRST)
        assert np.array_equal(a.dist, b.dist) and np.array_equal(a.parent, b.parent)
        assert np.array_equal(a.C, b.C) and np.array_equal(a.fixed_round, b.fixed_round)
        assert a.rounds == b.rounds
        for k in ("out_scanned", "active_visits", "front_visits", "reached"):
            assert a.stats[k] == b.stats[k]
        assert b.stats["in_scanned"] < a.stats["in_scanned"]


@pytest.mark.parametrize("base", [oracle.RULE_THR, oracle.RULE_MIND, oracle.CHEAP_FIRST],
                         ids=["thr", "mind", "cheap"])
def test_pred_counts_change_only_the_scan_count(base):
    """SP_1's predecessor counts (Sec. III): a vertex all of whose in-edges
    have been relaxed by fixed sources has its final D, and Eq. (1) fixes it
    in that same round; fixing it without reading its in-edges leaves every
    state, round count and counter but in_scanned unchanged."""
    for g, s in ((gg.rmat(12, 8, 1, 255, 4), None), (gg.random_var_graph(3000, 1, 9, 1, 60, 8), 2),
                 (gg.grid(40, 30, 1, 50, 1), 0), (gg.dag(20, 64, 5, 3, 1, 100, 7), 0)):
        if s is None or g.out_degree()[s] == 0:
            s = int(np.argmax(g.out_degree()))
        a = oracle.round_r(g, s, mode=base)
        b = oracle.round_r(g, s, mode=base | oracle.PRED_COUNT)
        assert np.array_equal(a.dist, b.dist) and np.array_equal(a.parent, b.parent)
        assert np.array_equal(a.C, b.C) and np.array_equal(a.fixed_round, b.fixed_round)
        assert a.rounds == b.rounds
        for k in ("out_scanned", "active_visits", "front_visits", "reached"):
            assert a.stats[k] == b.stats[k]
        assert b.stats["in_scanned"] <= a.stats["in_scanned"]


def test_pred_counts_on_an_out_tree():
    """On an out-tree every discovered vertex's only in-neighbour has been
    fixed and has relaxed it: with the counts no in-edge is read, without
    them each reached vertex but the root reads its one in-edge once."""
    for n, seed in ((50, 1), (2000, 2)):
        g = gg.out_tree(n, 1, 50, seed)
        a = oracle.round_r(g, 0)
        b = oracle.round_r(g, 0, mode=oracle.PRED_COUNT)
        assert a.stats["reached"] == n
        assert a.stats["in_scanned"] == n - 1
        assert b.stats["in_scanned"] == 0
        assert np.array_equal(a.dist, b.dist) and a.rounds == b.rounds
        assert np.array_equal(b.dist, oracle.dijkstra(g, 0)[0])


def test_pred_counts_refused_with_label_correcting_or_window():
    g = gg.random_graph(50, 3, 1, 9, 1)
    for kw in (dict(mode=oracle.PRED_COUNT | oracle.LABEL_CORRECT),
               dict(mode=oracle.PRED_COUNT, delta=5)):
        with pytest.raises(Exception):
            oracle.round_r(g, 0, **kw)


# --------------------------------------------- stored minimum witnesses (R22)

def witness_scan_count(g, s, mode, wdeg):
    """in_scanned of the witness mode, recomputed in plain Python from the
    per-round state of the run without witnesses (which the witness mode must
    reproduce exactly): the terms of round r come from the C of round r - 1,
    the D and threshold / minD of round r and the fixing rounds before r."""
    snaps = []
    oracle.round_r(g, s, mode=mode, on_round=lambda r, thr, mD, D, C, F: snaps.append(
        (thr, mD, D.copy(), C.copy(), F.copy())))
    n = g.n
    ins = [[] for _ in range(n)]
    for u, v, w in edges_of(g):
        ins[v].append((u, w))                 # CSC order: by source, then CSR order
    inw = [min((w for _, w in e), default=None) for e in ins]
    Cpre = [0] * n
    Fpre = [-1] * n
    Fpre[s] = 0
    witness = {}
    count = 0
    for r, (thr, mD, D, C, F) in enumerate(snaps, start=1):
        def term(u, w):
            if mode & oracle.RULE_MIND:
                lb = Cpre[u] if Fpre[u] >= 0 else max(Cpre[u], mD)
            else:
                lb = max(Cpre[u], min(int(D[u]), thr))
            return lb + w
        for y in range(n):
            if y == s or int(D[y]) == INF or not (F[y] == -1 or F[y] == r):
                continue
            dy = int(D[y])
            if mode & oracle.CHEAP_FIRST and ((inw[y] is not None and dy <= mD + inw[y])
                                              or dy <= thr):
                continue
            if mode & oracle.PRED_COUNT and all(0 <= Fpre[u] for u, _ in ins[y]):
                continue
            if len(ins[y]) <= wdeg and Cpre[y] != 0:
                count += 1
                k, m2 = witness[y]
                if term(*ins[y][k]) <= m2:
                    continue
            count += len(ins[y])
            if len(ins[y]) <= wdeg:
                terms = [term(u, w) for u, w in ins[y]]
                k = min(range(len(terms)), key=lambda i: (terms[i], ins[y][i][0], ins[y][i][1]))
                others = terms[:k] + terms[k + 1:]
                witness[y] = (k, min(others) if others else INF)
        Cpre = [int(c) for c in C]
        Fpre = [int(f) for f in F]
    return count


@pytest.mark.parametrize("base", [oracle.RULE_THR, oracle.RULE_MIND, oracle.CHEAP_FIRST,
                                  oracle.CHEAP_FIRST | oracle.PRED_COUNT],
                         ids=["thr", "mind", "cheap", "cheap-pred"])
def test_witness_changes_only_the_scan_count(base):
    """Every Eq. (1) term is non-decreasing across rounds, so a stored argmin
    whose term is still <= the other terms' old minimum is the exact minimum:
    every state, round count and counter but in_scanned is unchanged."""
    for g, s in ((gg.rmat(12, 8, 1, 255, 4), None), (gg.random_var_graph(3000, 1, 9, 1, 60, 8), 2),
                 (gg.grid(40, 30, 1, 50, 1), 0), (gg.dag(20, 64, 5, 3, 1, 100, 7), 0),
                 (gg.random_var_graph(2000, 1, 30, 1, 3, 9), 0)):
        if s is None or g.out_degree()[s] == 0:
            s = int(np.argmax(g.out_degree()))
        a = oracle.round_r(g, s, mode=base)
        for wdeg in (4, 256, 2**32 - 1):
            b = oracle.round_r(g, s, mode=base, witness_deg=wdeg)
            assert np.array_equal(a.dist, b.dist) and np.array_equal(a.parent, b.parent)
            assert np.array_equal(a.C, b.C) and np.array_equal(a.fixed_round, b.fixed_round)
            assert a.rounds == b.rounds
            for k in ("out_scanned", "active_visits", "front_visits", "reached"):
                assert a.stats[k] == b.stats[k]
        assert oracle.round_r(g, s, mode=base, witness_deg=0).stats == a.stats


@pytest.mark.parametrize("base", [oracle.RULE_THR, oracle.RULE_MIND, oracle.CHEAP_FIRST,
                                  oracle.CHEAP_FIRST | oracle.PRED_COUNT],
                         ids=["thr", "mind", "cheap", "cheap-pred"])
def test_witness_scan_count_matches_a_python_count(base):
    """The in-edges the witness mode reads, counted independently in Python
    (small weights, so that equal terms and ties for the minimum are common)."""
    for g, s, wdeg in ((gg.random_var_graph(300, 1, 12, 1, 4, 21), 0, 2**32 - 1),
                       (gg.random_var_graph(300, 1, 12, 1, 40, 22), 0, 6),
                       (gg.rmat(8, 8, 1, 3, 23), None, 2**32 - 1)):
        if s is None:
            s = int(np.argmax(g.out_degree()))
        got = oracle.round_r(g, s, mode=base, witness_deg=wdeg).stats["in_scanned"]
        assert got == witness_scan_count(g, s, base, wdeg)


def test_witness_refused_with_other_rounds():
    g = gg.random_graph(50, 3, 1, 9, 1)
    for kw in (dict(mode=oracle.LABEL_CORRECT), dict(mode=oracle.RULE_THR, delta=5),
               dict(mode=oracle.ALL_UNFIXED)):
        with pytest.raises(Exception):
            oracle.round_r(g, 0, witness_deg=8, **kw)


# ------------------------------------------- ablation: C for all unfixed vertices

def test_all_unfixed_ablation_is_sound_and_never_slower_in_rounds():
    """Raising C of undiscovered vertices too (step 4 "for all unfixed") keeps
    every lower bound valid (C <= cost <= D after every round, distances the
    textbook ones) and fixes no later: never more rounds than the active-only
    update."""
    for g, s in ((gg.rmat(12, 16, 1, 255, 3), None), (gg.random_graph(800, 6, 1, 50, 4), 0),
                 (gg.grid(20, 15, 1, 100, 5), 0), (gg.dag(16, 64, 6, 3, 1, 100, 6), 0)):
        if s is None:
            s = int(np.argmax(g.out_degree()))
        cost, _ = oracle.dijkstra(g, s)
        for base in (oracle.RULE_THR, oracle.RULE_MIND):
            checks = []

            def cb(r, thr, mD, D, C, F):
                finite = cost != INF
                checks.append(bool(np.all(C[finite] <= cost[finite]) and np.all(cost <= D)))

            a = oracle.round_r(g, s, mode=base)
            b = oracle.round_r(g, s, mode=base | oracle.ALL_UNFIXED, on_round=cb)
            assert all(checks)
            assert np.array_equal(b.dist, cost)
            assert b.rounds <= a.rounds


# ------------------------------------------- windowed relaxation (Delta-stepping)

def window_graphs():
    """Graphs of every shape the windowed mode meets: random, skewed (hubs),
    grids, layered DAGs, some unreachable vertices, multi-edges."""
    out = [(gg.random_graph(600, 6, 1, 50, 21), 0), (gg.grid(24, 18, 1, 1000, 22), 0),
           (gg.dag(12, 40, 5, 3, 1, 300, 23), 0), (gg.random_var_graph(500, 0, 7, 1, 90, 24), 3),
           (gg.from_edges(4, [(0, 1, 2), (0, 1, 1), (1, 2, 5), (0, 2, 9), (2, 3, 1)]), 0)]
    g = gg.rmat(11, 12, 1, 255, 25)
    out.append((g, int(np.argmax(g.out_degree()))))
    return out


@pytest.mark.parametrize("variant", ["window9", "window10"])
def test_windowed_hand_derived_trace(variant):
    """The window bound is minD + delta, strict: on the hand-derived example
    delta = 9 keeps v3 waiting (the label-setting run, 4 rounds) and delta =
    10 lets it relax one round before it is fixed (3 rounds)."""
    ex = worked_example()[variant]
    g = gg.from_edges(ex["n"], ex["edges"])
    r = oracle.round_r(g, ex["source"], delta=ex["delta"])
    assert r.dist.tolist() == ex["dist"]
    assert r.fixed_round.tolist() == ex["fixed_round"]
    assert r.parent.tolist() == ex["parent"]
    assert r.rounds == ex["rounds"]
    for k in ("out_scanned", "front_visits", "active_visits"):
        assert r.stats[k] == ex[k]


@pytest.mark.parametrize("base", [oracle.RULE_THR, oracle.RULE_MIND, oracle.CHEAP_FIRST,
                                  oracle.RULE_MIND | oracle.CHEAP_FIRST],
                         ids=["thr", "mind", "cheap", "mind-cheap"])
def test_windowed_zero_is_the_label_setting_round(base):
    """delta = 0: no active vertex is below minD, so only fixed vertices
    relax, each once -- the label-setting round, state and counters alike."""
    for g, s in window_graphs():
        a = oracle.round_r(g, s, mode=base)
        b = oracle.round_r(g, s, mode=base, delta=0)
        for f in ("dist", "parent", "C", "fixed_round"):
            assert np.array_equal(getattr(a, f), getattr(b, f)), f
        assert a.rounds == b.rounds and a.stats == b.stats


@pytest.mark.parametrize("base", [oracle.RULE_THR, oracle.RULE_MIND], ids=["thr", "mind"])
def test_windowed_unbounded_is_label_correcting_round_by_round(base):
    """delta above every distance: every changed vertex relaxes the next
    round, as SP_4 step 3 prints it.  The state after each round equals the
    label-correcting run's for as long as that runs; the windowed run then
    goes on until the active set is empty, so every reachable vertex ends
    fixed."""
    for g, s in window_graphs():
        lc, win = [], []
        a = oracle.round_r(g, s, mode=base | oracle.LABEL_CORRECT,
                           on_round=lambda r, t, m, D, C, F: lc.append((D.copy(), C.copy(),
                                                                        F.copy())))
        b = oracle.round_r(g, s, mode=base, delta=2**64 - 1,
                           on_round=lambda r, t, m, D, C, F: win.append((D.copy(), C.copy(),
                                                                         F.copy())))
        assert b.rounds >= a.rounds
        for r, (x, y) in enumerate(zip(lc, win), start=1):
            for u, v in zip(x, y):
                assert np.array_equal(u, v), f"round {r}"
        cost = oracle.dijkstra(g, s)[0]
        assert np.array_equal(b.dist, cost)
        assert np.array_equal(b.fixed_round >= 0, cost != INF)


@pytest.mark.parametrize("delta", [1, 6, 40, 300, 5000])
@pytest.mark.parametrize("mode", [oracle.RULE_THR, oracle.RULE_MIND], ids=["thr", "mind"])
def test_windowed_round_invariants(delta, mode):
    """Any window: C <= cost <= D after every round, fixed vertices at their
    cost, textbook distances, tight parent edges, every reachable vertex
    fixed, every round but the last fixes something."""
    for n, d, wmax, seed in SMALL_CASES[::3]:
        check_round_invariants(random_small(n, d, wmax, seed), 0, mode, delta=delta)
    for g, s in window_graphs():
        check_round_invariants(g, s, mode, delta=delta)


def test_windowed_and_label_correcting_do_not_combine():
    g = gg.random_graph(50, 3, 1, 9, 1)
    with pytest.raises(RuntimeError):
        oracle.round_r(g, 0, mode=oracle.LABEL_CORRECT, delta=5)
